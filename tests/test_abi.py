"""The C-ABI library builds, loads without a GPU, and exports every function
that include/cutqc.h declares.  No compute calls here."""
import ctypes
import subprocess

import pytest


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_05836_gb300 import cutqc
    return cutqc


def test_exports_every_declared_symbol(built):
    cutqc = built
    declared = cutqc.declared_symbols()
    assert len(declared) >= 12
    L = cutqc.lib()
    for name in declared:
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", cutqc.LIB_PATH], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert set(declared) <= exported


def test_version_and_error_text(built):
    cutqc = built
    assert "sm_103a" in cutqc.cutqc_version()
    assert isinstance(cutqc.cutqc_last_error(), str)


def test_host_validation_without_gpu(built):
    """Descriptor checks run on the host before any CUDA call."""
    cutqc = built

    class S:
        w = 3
        in_local = [2, 1]          # not ascending: rejected
        out_local = []
        in_edge = [0, 1]
        out_edge = []
        out_qubit = [0, 1, 2]
    with pytest.raises(cutqc.CutqcError) as e:
        cutqc.cutqc_attribute_workspace_size(S)
    assert e.value.code == cutqc.EINVAL

    class T:
        w = 4
        in_local = [0]
        out_local = [3]
        in_edge = [0]
        out_edge = [1]
        out_qubit = [0, 1, 2]
    # the measured side's result: 2^o rows x 4^k columns of float32
    assert cutqc.cutqc_attribute_workspace_size(T) == 2 ** 3 * 4 ** 2 * 4

    class U:
        w = 3
        in_local = []
        out_local = [2]
        in_edge = []
        out_edge = [0]
        out_qubit = [0, 1]

    class V:
        w = 3
        in_local = [0]
        out_local = []
        in_edge = [0]
        out_edge = []
        out_qubit = [2, 3, 4]
    assert cutqc.cutqc_fd_shape([U, V]) == (4, 8)
    with pytest.raises(cutqc.CutqcError):      # edge 0 measured twice
        cutqc.cutqc_fd_shape([U, U])


def _sub(w, in_local=(), out_local=(), in_edge=(), out_edge=(), out_qubit=None):
    class S:
        pass
    s = S()
    s.w, s.in_local, s.out_local, s.in_edge, s.out_edge = w, list(in_local), list(out_local), list(in_edge), list(out_edge)
    s.out_qubit = list(out_qubit) if out_qubit is not None else list(range(w - len(out_local)))
    return s


def test_validation_error_codes(built):
    """Shape, size and workspace queries reject malformed descriptors with the
    documented codes, on the host."""
    cq = built
    # an initialised edge with no measured partner
    with pytest.raises(cq.CutqcError) as e:
        cq.cutqc_fd_shape([_sub(3, in_local=[0], in_edge=[5])])
    assert e.value.code == cq.EINVAL
    # width beyond the limit
    with pytest.raises(cq.CutqcError) as e:
        cq.cutqc_attribute_workspace_size(_sub(31))
    assert e.value.code == cq.EINVAL
    # unknown precision
    a = _sub(3, out_local=[2], out_edge=[0], out_qubit=[0, 1])
    b = _sub(3, in_local=[0], in_edge=[0], out_qubit=[2, 3, 4])
    with pytest.raises(cq.CutqcError) as e:
        cq.cutqc_reconstruct_fd_workspace_size([a, b], 7)
    assert e.value.code == cq.EINVAL
    assert cq.cutqc_reconstruct_fd_workspace_size([a, b], cq.PREC_FP16X3_TC) > 0
    # DD: outputs must cover n, M and T within limits
    with pytest.raises(cq.CutqcError) as e:
        cq.cutqc_dd_run_workspace_size([a, b], 6, 2, 2)
    assert e.value.code == cq.EINVAL
    with pytest.raises(cq.CutqcError) as e:
        cq.cutqc_dd_run_workspace_size([a, b], 5, 31, 2)
    assert e.value.code == cq.EUNSUPPORTED
    with pytest.raises(cq.CutqcError) as e:
        cq.cutqc_dd_run_workspace_size([a, b], 5, 2, 33)
    assert e.value.code == cq.EUNSUPPORTED
    assert cq.cutqc_dd_run_workspace_size([a, b], 5, 2, 2) > 0


def test_mlp_queries(built):
    cq = built
    n = ctypes.c_int64(0)
    assert cq.lib().cutqc_mlp_param_count(ctypes.byref(n)) == 0
    assert n.value == 64 * 256 + 256 + 256 * 256 + 256 + 256 + 1
    b = ctypes.c_size_t(0)
    assert cq.lib().cutqc_mlp_workspace_size(0, ctypes.byref(b)) == cq.EINVAL
    assert cq.lib().cutqc_mlp_workspace_size(100, ctypes.byref(b)) == 0 and b.value > 0


def test_dd_batch_validation_without_gpu(built):
    """The persistent DD batch sizes its workspace and rejects bad runs and
    options on the host (the device pointers are only recorded, never read)."""
    import torch
    cq = built
    a = _sub(3, out_local=[2], out_edge=[0], out_qubit=[0, 1])
    b = _sub(3, in_local=[0], in_edge=[0], out_qubit=[2, 3, 4])
    att = [torch.zeros(4, 4), torch.zeros(8, 4)]       # host stand-ins: not dereferenced here

    def run(subs=(a, b), n=5, M=2, R=3, T=2, max_jobs=8, bins=64):
        return dict(subs=list(subs), attributed=att, n_qubits=n, M=M, R=R, T=T,
                    jobs=torch.zeros(max_jobs * ctypes.sizeof(cq.DDJob), dtype=torch.uint8),
                    n_jobs=torch.zeros(1, dtype=torch.int32), bins=torch.zeros(bins))
    one = cq.cutqc_dd_batch_workspace_size([run()])
    two = cq.cutqc_dd_batch_workspace_size([run(), run(T=1)])
    assert one > 0 and two > one
    cases = [
        ([run(subs=(_sub(3, out_qubit=[0, 1, 2]),), n=3)], None, cq.EUNSUPPORTED),   # nothing to contract
        ([run(max_jobs=2)], None, cq.ENOMEM),          # 1 + 2 + 1 records needed
        ([run(bins=8)], None, cq.ENOMEM),
        ([run(n=6)], None, cq.EINVAL),                 # outputs do not cover n
        ([run(T=33)], None, cq.EUNSUPPORTED),
        ([run()], {"topk_chunk": 300}, cq.EINVAL),     # not a power of two
        ([run()], {"topk_chunk": 128}, cq.EINVAL),
        ([run()], {"merge_ctas": 5000}, cq.EINVAL),
        ([run()], {"ctas": -1}, cq.EINVAL),
        ([run()], {"ctas_per_sm": 5}, cq.EINVAL),
        ([run()], {"ctas_per_sm": 1}, cq.EINVAL),
        ([], None, cq.EINVAL),
    ]
    for runs, opt, code in cases:
        if not runs:
            n = ctypes.c_size_t(0)
            rc = cq.lib().cutqc_dd_batch_workspace_size(0, None, None, ctypes.byref(n))
            assert rc == code
            continue
        with pytest.raises(cq.CutqcError) as e:
            cq.cutqc_dd_batch_workspace_size(runs, opt)
        assert e.value.code == code, (opt, cq.cutqc_last_error())


def test_dd_batch_program_shape_without_gpu(built):
    """The batch program's structure, counted by hand on a two-subcircuit
    circuit (5 outputs, one cut, no merge split at these sizes): per level
    one merge phase (the bin totals' zeroing and one merge per subcircuit),
    one contraction phase (one step), the chunked top-T phase when T > 0 and
    the selection phase; levels = min(R, ceil(n / M)), one when T = 0.  Runs
    share phases (the phase count is the largest run's), ops add up."""
    import torch
    cq = built
    a = _sub(3, out_local=[2], out_edge=[0], out_qubit=[0, 1])
    b = _sub(3, in_local=[0], in_edge=[0], out_qubit=[2, 3, 4])
    att = [torch.zeros(4, 4), torch.zeros(8, 4)]

    def run(M, R, T):
        return dict(subs=[a, b], attributed=att, n_qubits=5, M=M, R=R, T=T,
                    jobs=torch.zeros(16 * ctypes.sizeof(cq.DDJob), dtype=torch.uint8),
                    n_jobs=torch.zeros(1, dtype=torch.int32), bins=torch.zeros(256))
    # T = 0: one level: merge, contraction, selection; ops: zero + 2 merges + step + selection
    assert {k: v for k, v in cq.cutqc_dd_batch_shape([run(2, 3, 0)]).items() if k != "tasks"} == \
        {"phases": 3, "ops": 5}
    # T = 2, M = 2: 3 levels x (merge, contraction, top-T, selection); 6 ops per level
    s = cq.cutqc_dd_batch_shape([run(2, 3, 2)])
    assert (s["phases"], s["ops"]) == (12, 18)
    # R caps the levels; M = 5 gives one level holding every qubit
    assert cq.cutqc_dd_batch_shape([run(2, 2, 2)])["phases"] == 8
    assert cq.cutqc_dd_batch_shape([run(5, 3, 2)])["phases"] == 4
    # runs share phases, ops add up
    both = cq.cutqc_dd_batch_shape([run(2, 3, 2), run(5, 3, 2)])
    assert (both["phases"], both["ops"]) == (12, 18 + 6)
    assert both["tasks"] == s["tasks"] + cq.cutqc_dd_batch_shape([run(5, 3, 2)])["tasks"]


def test_dd_batch_many_runs_shape(built):
    """Ninety runs in one program (a merge phase of 270 ops, beyond the
    kernel's shared-memory op table): the builder's counts still add up."""
    import torch
    cq = built
    a = _sub(3, out_local=[2], out_edge=[0], out_qubit=[0, 1])
    b = _sub(3, in_local=[0], in_edge=[0], out_qubit=[2, 3, 4])
    att = [torch.zeros(4, 4), torch.zeros(8, 4)]
    run = dict(subs=[a, b], attributed=att, n_qubits=5, M=2, R=3, T=2,
               jobs=torch.zeros(16 * ctypes.sizeof(cq.DDJob), dtype=torch.uint8),
               n_jobs=torch.zeros(1, dtype=torch.int32), bins=torch.zeros(256))
    one = cq.cutqc_dd_batch_shape([run])
    many = cq.cutqc_dd_batch_shape([run] * 90)
    assert many["phases"] == one["phases"] == 12
    assert many["ops"] == 90 * one["ops"] and many["tasks"] == 90 * one["tasks"]
    assert cq.cutqc_dd_batch_workspace_size([run] * 90) > 90 * cq.cutqc_dd_batch_workspace_size([run]) // 2


def test_fd_input_events_host_checks(built):
    """cutqc_fd_input_events: argument checks, and a count that does not
    match the next reconstruction's subcircuits fails that call (then the
    setting is gone).  Every call here fails on the host: null tensors and an
    invalid output order, so nothing can reach a kernel launch."""
    cutqc = built
    L = cutqc.lib()
    assert L.cutqc_fd_input_events(ctypes.c_int(-1), None) == cutqc.EINVAL
    assert L.cutqc_fd_input_events(ctypes.c_int(4097), None) == cutqc.EINVAL
    assert L.cutqc_fd_input_events(ctypes.c_int(2), None) == cutqc.EINVAL
    assert L.cutqc_fd_input_events(ctypes.c_int(0), None) == cutqc.OK

    class U:
        w = 3
        in_local = []
        out_local = [2]
        in_edge = []
        out_edge = [0]
        out_qubit = [0, 1]

    class V:
        w = 3
        in_local = [0]
        out_local = []
        in_edge = [0]
        out_edge = []
        out_qubit = [2, 3, 4]
    arr, keep = cutqc._subs([U, V])
    ptrs = (ctypes.c_void_p * 2)(None, None)
    none3 = (ctypes.c_void_p * 3)(None, None, None)
    assert L.cutqc_fd_input_events(ctypes.c_int(3), none3) == cutqc.OK

    def call():
        return L.cutqc_reconstruct_fd(ctypes.c_int(2), arr, ptrs, ctypes.c_int(7),
                                      ctypes.c_int(cutqc.PREC_FP32_SIMT), ctypes.c_int64(0), ctypes.c_int64(-1),
                                      None, None, None, ctypes.c_size_t(0), None)
    assert call() == cutqc.EINVAL
    assert "input events" in cutqc.cutqc_last_error()
    # cleared by that call: the next one fails on the output order instead
    assert call() == cutqc.EINVAL
    assert "out_order" in cutqc.cutqc_last_error()
