"""GPU parity of the dynamic-definition path (merge, bin reconstruction,
top-T selection, Algorithm 1 end to end) against the FP64 oracle."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_05836_gb300 import cutqc
    return cutqc


def _setup(cut):
    import torch
    from oracle import attribution
    from workloads.simulate import simulate_variants
    subs = cut.subcircuits
    var = [simulate_variants(s) for s in subs]
    A = [attribution.attribute(v, s.w, s.in_local, s.out_local, s.in_edge, s.out_edge) for s, v in zip(subs, var)]
    return subs, A, [torch.from_numpy(a.astype(np.float32)).cuda() for a in A]


def _cut(kind):
    from workloads import circuits as C
    from workloads.cutting import search_cut
    if kind == "brickwall":
        return search_cut(C.brickwall(10, 4, 11), 7, 2, restarts=4)
    if kind == "aqft":
        return search_cut(C.aqft(12, 2, max_dist=2), 5, 4, restarts=4)
    return search_cut(C.bv(14, 9), 5, 5, restarts=4)


TV_GATE = 1e-6      # the metric's gate: total variation and total per job


def _gate_job(b, ref_bins, bin_sum):
    """A job's bins against the FP64 oracle's: total variation
    0.5 sum |b - ref| <= 1e-6 and |float64 total - oracle total| <= 1e-6."""
    tv = 0.5 * float(np.abs(b - ref_bins).sum())
    assert tv <= TV_GATE, f"TV {tv:.3e} > {TV_GATE}"
    err = abs(bin_sum - float(ref_bins.sum()))
    assert err <= TV_GATE, f"bin total error {err:.3e} > {TV_GATE}"
    return tv


@pytest.mark.parametrize("kind", ["brickwall", "aqft", "bv"])
def test_merge_matches_oracle(cq, kind):
    import torch
    from oracle import dd
    cut = _cut(kind)
    subs, A, At = _setup(cut)
    rng = np.random.default_rng(0)
    for s, a64, at in zip(subs, A, At):
        o = s.o
        for _ in range(3):
            role = rng.integers(0, 4, size=o)
            got = cq.cutqc_dd_merge(s, at, role)
            active = {q for q, r in zip(s.out_qubit, role) if r == 0}
            zoom = {q: int(r - 2) for q, r in zip(s.out_qubit, role) if r >= 2}
            ref = dd.merge(a64, s.out_qubit, active, zoom)
            torch.cuda.synchronize()
            g = got.cpu().numpy().astype(np.float64)
            assert g.shape == ref.shape
            assert np.abs(g - ref).max() <= 1e-6 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("strategy", [0, 1], ids=["dfs", "bfs"])
@pytest.mark.parametrize("kind", ["brickwall", "aqft", "bv"])
def test_dd_run_matches_oracle(cq, kind, strategy):
    import torch
    from oracle import dd
    cut = _cut(kind)
    subs, A, At = _setup(cut)
    n = cut.circuit.n
    # a BV output is one basis state: its other bins are all zero and their
    # order is decided by rounding noise, so only the top bin is expanded
    M, R, T = 4, 6, (1 if kind == "bv" else 3)
    jobs, bins = cq.cutqc_dd_run(subs, At, n, M, R, T, strategy)
    torch.cuda.synchronize()
    ref = dd.run(A, [s.out_qubit for s in subs], [s.edges for s in subs], cut.K, n, M, R, T,
                 strategy="dfs" if strategy == 0 else "bfs")
    assert len(jobs) == len(ref)
    for J, rj in zip(jobs, ref):
        assert list(J.active[:J.n_active]) == rj["active"]
        assert J.zoom() == rj["zoom"]
        b = bins[J.bins_offset:J.bins_offset + (1 << J.n_active)].cpu().numpy().astype(np.float64)
        assert np.abs(b - rj["bins"]).max() <= 1e-6
        _gate_job(b, rj["bins"], J.bin_sum)
        # selection: same bins (values may tie within float32 rounding)
        top = [i for i in J.top_idx[:T] if i >= 0]
        if rj["top"]:
            assert len(top) == len(rj["top"])
            np.testing.assert_allclose(sorted(rj["bins"][top]), sorted(rj["bins"][rj["top"]]), atol=1e-6)


def test_dd_bv_finds_hidden_string(cq):
    """DFS on a Bernstein-Vazirani circuit reaches the single solution state."""
    from workloads import circuits as C
    from workloads.cutting import search_cut
    n = 24
    c = C.bv(n, 3)
    cut = search_cut(c, 8, 4, restarts=4)
    subs, A, At = _setup(cut)
    M = 6
    jobs, bins = cq.cutqc_dd_run(subs, At, n, M, math.ceil(n / M), 2, 0)
    last = jobs[-1]
    assert last.depth * M + last.n_active == n
    b = bins[last.bins_offset:last.bins_offset + (1 << last.n_active)].cpu().numpy()
    top = int(np.argmax(b))
    bits = last.zoom()
    for j in range(last.n_active):
        bits[last.active[j]] = (top >> j) & 1
    assert [bits[q] for q in range(n - 1)] == c.meta["hidden"] and bits[n - 1] == 1
    assert abs(b[top] - 1) < 1e-5


@pytest.mark.parametrize("kind", ["aqft", "bv"])
def test_dd_step_any_bin_order(cq, kind):
    """One reconstruction with every output qubit active and the bin bits in
    a random order: bins[sum_q b_q 2^perm[q]] = p(b), with the workspace the
    size query reports."""
    import torch
    from oracle import fd
    cut = _cut(kind)
    subs, A, At = _setup(cut)
    n = cut.circuit.n
    p = fd.kron_to_original(fd.reconstruct_kron(A, [s.edges for s in subs], cut.K), [s.out_qubit for s in subs])
    rng = np.random.default_rng(5)
    for _ in range(3):
        perm = rng.permutation(n)
        merged = [cq.cutqc_dd_merge(s, at, np.zeros(s.o, dtype=np.int8)) for s, at in zip(subs, At)]
        active_bits = [s.o for s in subs]
        bin_bit = [int(perm[q]) for s in subs for q in s.out_qubit]
        bins = torch.empty((1, 1 << n), dtype=torch.float32, device="cuda")
        total = torch.zeros(1, dtype=torch.float64, device="cuda")
        cq.cutqc_dd_step(subs, active_bits, bin_bit, merged, bins, bin_sum=total)
        torch.cuda.synchronize()
        idx = np.zeros(1 << n, dtype=np.int64)
        for q in range(n):
            idx |= ((np.arange(1 << n) >> q) & 1) << perm[q]
        got = bins[0].cpu().numpy().astype(np.float64)[idx]
        assert np.abs(got - p).max() <= 1e-6
        assert abs(total.item() - 1.0) <= 1e-6


@pytest.mark.parametrize("kind,M,T", [("brickwall", 4, 3), ("aqft", 4, 2), ("bv", 5, 1)])
def test_dd_run_async_in_cuda_graph(cq, kind, M, T):
    """The enqueue-only level-by-level run, captured in a CUDA graph and
    replayed twice, gives the records and bins of the synchronous run."""
    import torch
    cut = _cut(kind)
    subs, A, At = _setup(cut)
    n = cut.circuit.n
    R = 6
    ref_jobs, ref_bins = cq.cutqc_dd_run(subs, At, n, M, R, T, 1)
    torch.cuda.synchronize()
    jobs, n_jobs, bins = cq.cutqc_dd_run_async(subs, At, n, M, R, T)   # first call outside capture
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        cq.cutqc_dd_run_async(subs, At, n, M, R, T, jobs=jobs, n_jobs=n_jobs, bins=bins)
    for _ in range(2):
        jobs.zero_()
        bins.zero_()
        g.replay()
        torch.cuda.synchronize()
        got = cq.dd_jobs_from_device(jobs, n_jobs)
        assert len(got) == len(ref_jobs)
        for J, Rj in zip(got, ref_jobs):
            assert (J.level, J.depth, J.parent, J.parent_bin, J.n_active) == \
                (Rj.level, Rj.depth, Rj.parent, Rj.parent_bin, Rj.n_active)
            assert J.zoom() == Rj.zoom()
            assert list(J.top_idx) == list(Rj.top_idx)
            assert abs(J.bin_sum - Rj.bin_sum) <= 1e-12   # float64 totals: atomic order may differ
            nb = 1 << J.n_active
            assert torch.equal(bins[J.bins_offset:J.bins_offset + nb], ref_bins[Rj.bins_offset:Rj.bins_offset + nb])
    assert cq.cutqc_device_status() == 0


def test_dd_single_subcircuit(cq):
    """Degenerate case K = 0: dynamic definition over one subcircuit gives the
    marginals of its own distribution."""
    from oracle import dd
    from workloads import circuits as C
    from workloads.cutting import Dag, build_cut
    c = C.brickwall(9, 3, 5)
    cut = build_cut(c, [0] * Dag(c).nv)
    subs, A, At = _setup(cut)
    n, M, R, T = c.n, 4, 4, 2
    jobs, bins = cq.cutqc_dd_run(subs, At, n, M, R, T, 1)
    ref = dd.run(A, [s.out_qubit for s in subs], [s.edges for s in subs], 0, n, M, R, T, strategy="bfs")
    assert len(jobs) == len(ref)
    for J, rj in zip(jobs, ref):
        b = bins[J.bins_offset:J.bins_offset + (1 << J.n_active)].cpu().numpy().astype(np.float64)
        assert np.abs(b - rj["bins"]).max() <= 1e-6
        _gate_job(b, rj["bins"], J.bin_sum)


def test_autotuned_dd_options_match_oracle(cq):
    """The autotuner returns one of its candidate launch shapes, and the run
    with it still matches the FP64 oracle."""
    from oracle import dd
    from paper_2205_05836_gb300.tune import CANDIDATES, tune_dd
    cut = _cut("brickwall")
    subs, A, At = _setup(cut)
    n, M, R, T = cut.circuit.n, 4, 6, 3
    best, trials = tune_dd(subs, At, n, M, R, T, reps=2)
    assert best.get("precision") == 0
    assert {k: v for k, v in best.items() if k != "precision"} in CANDIDATES
    assert len(trials) == len(CANDIDATES) and trials[0][2]
    jobs, n_jobs, bins = cq.cutqc_dd_run_async(subs, At, n, M, R, T, options=best)
    got = cq.dd_jobs_from_device(jobs, n_jobs)
    ref = dd.run(A, [s.out_qubit for s in subs], [s.edges for s in subs], cut.K, n, M, R, T, strategy="bfs")
    assert len(got) == len(ref)
    for J, rj in zip(got, ref):
        b = bins[J.bins_offset:J.bins_offset + (1 << J.n_active)].cpu().numpy().astype(np.float64)
        assert np.abs(b - rj["bins"]).max() <= 1e-6
        _gate_job(b, rj["bins"], J.bin_sum)


@pytest.mark.parametrize("precision", [1, 2], ids=["tc", "tc_prune"])
@pytest.mark.parametrize("kind,M,T", [("brickwall", 4, 3), ("aqft", 6, 1), ("brickwall", 10, 2), ("bv", 5, 1)])
def test_dd_split_precision_matches_oracle(cq, kind, M, T, precision):
    """Bin reconstruction on the tensor-core path (FP16 hi/lo split, the FD
    GEMM) inside the enqueue-only run, every step on the split path
    (tc_min_outputs = 1; by default steps this small take FP32): bins and
    totals against the FP64 oracle, and the same jobs (levels of fewer than
    4 bins per job take FP32).  The cases are ones whose expanded bins are
    separated from the next by far more than rounding (an AQFT level with
    exactly equal bins may expand either of them)."""
    import torch
    from oracle import dd
    cut = _cut(kind)
    subs, A, At = _setup(cut)
    n, R = cut.circuit.n, 6
    jobs, n_jobs, bins = cq.cutqc_dd_run_async(subs, At, n, M, R, T,
                                               options={"precision": precision, "tc_min_outputs": 1})
    got = cq.dd_jobs_from_device(jobs, n_jobs)
    ref = dd.run(A, [s.out_qubit for s in subs], [s.edges for s in subs], cut.K, n, M, R, T, strategy="bfs")
    assert len(got) == len(ref)
    for J, rj in zip(got, ref):
        assert list(J.active[:J.n_active]) == rj["active"]
        assert J.zoom() == rj["zoom"]
        b = bins[J.bins_offset:J.bins_offset + (1 << J.n_active)].cpu().numpy().astype(np.float64)
        assert np.abs(b - rj["bins"]).max() <= 1e-6
        _gate_job(b, rj["bins"], J.bin_sum)
        top = [i for i in J.top_idx[:T] if i >= 0]
        if rj["top"]:
            np.testing.assert_allclose(sorted(rj["bins"][top]), sorted(rj["bins"][rj["top"]]), atol=1e-6)
    assert cq.cutqc_device_status() == 0


@pytest.mark.parametrize("kind,M,T", [("brickwall", 10, 2), ("aqft", 6, 1)])
def test_dd_split_precision_small_steps_take_fp32(cq, kind, M, T):
    """Under the tensor-core precision with the default floor, a level whose
    contraction steps have fewer than 2^22 outputs runs them in FP32 on CUDA
    cores: the records and bins equal the FP32 run's bit for bit (the
    float64 totals to rounding)."""
    cut = _cut(kind)
    subs, A, At = _setup(cut)
    n, R = cut.circuit.n, 6
    runs = []
    for prec in (0, 1):
        jobs, n_jobs, bins = cq.cutqc_dd_run_async(subs, At, n, M, R, T, options={"precision": prec})
        js = cq.dd_jobs_from_device(jobs, n_jobs)
        runs.append([(list(j.active[:j.n_active]), j.zoom(), list(j.top_idx[:T]), j.bin_sum,
                      bins[j.bins_offset:j.bins_offset + (1 << j.n_active)].cpu().numpy()) for j in js])
    assert len(runs[0]) == len(runs[1])
    for a, b in zip(*runs):
        assert a[:3] == b[:3]
        assert np.array_equal(a[4], b[4])
        assert abs(a[3] - b[3]) <= 1e-12       # float64 totals: atomics add warps' sums in any order
    assert cq.cutqc_device_status() == 0


def test_dd_options_out_of_range(cq):
    """Options are checked before anything is enqueued: a size floor beyond
    2^61 or negative, an unknown precision and an oversized merge split are
    rejected with CUTQC_EINVAL."""
    cut = _cut("brickwall")
    subs, A, At = _setup(cut)
    n = cut.circuit.n
    for opt in ({"tc_min_outputs": 63}, {"tc_min_outputs": -1}, {"precision": 7}, {"merge_ctas": 5000}):
        with pytest.raises(cq.CutqcError) as e:
            cq.cutqc_dd_run_async(subs, At, n, 4, 2, 2, options=opt)
        assert e.value.code == cq.EINVAL, opt
    assert cq.cutqc_device_status() == 0


@pytest.mark.parametrize("T", [1, 4, 17])
def test_dd_topk_large_job_with_ties(cq, T):
    """Selection on jobs of more than 2^16 bins (chunked first pass, then the
    chunks' candidates): one subcircuit without cuts, so the bins are its
    merged tensor as given; values drawn from a few levels, so that ties
    cross chunk boundaries.  The T best must be exactly the first T of the
    order (value descending, index ascending)."""
    import torch
    from types import SimpleNamespace
    o = 19
    sub = SimpleNamespace(w=o, in_local=[], in_edge=[], out_local=[], out_edge=[], out_qubit=list(range(o)))
    rng = np.random.default_rng(T)
    n_jobs = 3
    vals = rng.integers(0, 40, size=(n_jobs, 1 << o)).astype(np.float32) / 8.0
    vals[1, :] = 1.0                        # one job: every bin ties
    vals[2, rng.integers(0, 1 << o, size=5)] = 99.0
    merged = torch.from_numpy(vals.reshape(n_jobs, 1 << o, 1)).cuda()
    bins = torch.empty((n_jobs, 1 << o), dtype=torch.float32, device="cuda")
    tidx = torch.empty((n_jobs, T), dtype=torch.int32, device="cuda")
    tval = torch.empty((n_jobs, T), dtype=torch.float32, device="cuda")
    cq.cutqc_dd_step([sub], [o], list(range(o)), [merged], bins, topk=T, top_idx=tidx, top_val=tval)
    torch.cuda.synchronize()
    assert torch.equal(bins.cpu(), torch.from_numpy(vals))
    for j in range(n_jobs):
        order = np.lexsort((np.arange(1 << o), -vals[j].astype(np.float64)))[:T]
        assert tidx[j].cpu().tolist() == [int(i) for i in order]
        assert np.array_equal(tval[j].cpu().numpy(), vals[j][order])


@pytest.mark.parametrize("precision", [1, 0], ids=["tc", "fp32"])
def test_dd_dense_recursion_full_size(cq, precision):
    """One dense recursion, the paper's per-recursion workload: 30 active
    qubits of the 60-qubit blocked brick-wall circuit (2^30 bins, 4 GiB),
    30 merged.  4096 seeded sampled bins against the FP64 oracle (merge,
    then Eq. 1 entry by entry), the float64 bin total against 1, and the
    top-4 selection against torch.topk on the same bins."""
    import torch
    from oracle import attribution, dd, fd
    from workloads.configs import dd_batched
    w = [x for x in dd_batched() if x.n == 60][0]
    subs = w.subcircuits
    var = w.variants()
    A64 = [attribution.attribute(v, s.w, s.in_local, s.out_local, s.in_edge, s.out_edge) for s, v in zip(subs, var)]
    att = [cq.cutqc_attribute(s, torch.from_numpy(v).cuda()) for s, v in zip(subs, var)]
    M, T = 30, 4
    bins = torch.empty(1 << M, dtype=torch.float32, device="cuda")
    jobs, n_jobs, _ = cq.cutqc_dd_run_async(subs, att, w.n, M, 1, T, max_jobs=4, bins=bins,
                                            options={"precision": precision})
    js = cq.dd_jobs_from_device(jobs, n_jobs)
    assert len(js) == 1 and js[0].n_active == M
    assert abs(js[0].bin_sum - 1.0) <= 1e-6
    active = list(range(M))
    merged = [dd.merge(a, s.out_qubit, set(active), {}) for a, s in zip(A64, subs)]
    rng = np.random.default_rng(30)
    idx = np.unique(rng.integers(0, 1 << M, size=4096))
    parts = fd.split_original_index(idx, [[q for q in s.out_qubit if q < M] for s in subs])
    ref = fd.entries(merged, [s.edges for s in subs], w.K, parts)
    got = bins[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.float64)
    err = np.abs(got - ref)
    assert err.max() <= 1e-6, err.max()
    assert 0.5 * (1 << M) * err.mean() <= 1e-6
    tv, ti = torch.topk(bins, T)
    top_idx = [int(i) for i in js[0].top_idx[:T]]
    top_val = [float(v) for v in js[0].top_val[:T]]
    assert top_val == tv.cpu().tolist()
    assert [float(bins[i]) for i in top_idx] == top_val
    assert cq.cutqc_device_status() == 0


@pytest.mark.parametrize("kind,M,T", [("brickwall", 4, 3), ("aqft", 6, 1)])
def test_sharded_dd_driver_on_one_gpu(cq, kind, M, T):
    """The multi-GPU breadth-first driver (a level's jobs split over ranks,
    one all-gather of candidates per level), run as a single rank on this
    GPU through cutqc_dd_merge_batch and cutqc_dd_step: the same jobs as the
    single-GPU level-synchronous run, bins within float32 rounding."""
    import torch
    from paper_2205_05836_gb300.shard import dd_run_sharded, gpu_level_executor
    cut = _cut(kind)
    subs, A, At = _setup(cut)
    n, R = cut.circuit.n, 6
    recs = dd_run_sharded(gpu_level_executor(cq, subs, At, n, M, T), n, M, R, T)
    ref_jobs, ref_bins = cq.cutqc_dd_run(subs, At, n, M, R, T, 1)
    torch.cuda.synchronize()
    assert len(recs) == len(ref_jobs)
    for r, J in zip(recs, ref_jobs):
        assert r["active"] == list(J.active[:J.n_active])
        assert r["zoom"] == J.zoom()
        assert (r["parent"], r["parent_bin"]) == (J.parent, J.parent_bin)
        nb = 1 << J.n_active
        assert torch.allclose(r["bins"], ref_bins[J.bins_offset:J.bins_offset + nb], atol=1e-7, rtol=0)
        assert abs(r["bin_sum"] - J.bin_sum) <= 1e-9
    assert cq.cutqc_device_status() == 0


@pytest.mark.parametrize("n_qubits,n_jobs", [(40, 9), (50, 13), (60, 13)])
def test_dd_batched_full_size(cq, n_qubits, n_jobs):
    """The bench's DD configuration at full size, each of its three blocked
    brick-wall circuits (40, 50 and 60 qubits, subcircuits <= 15 qubits), 16
    active qubits per level, breadth first, top 4 (3 or 4 levels, 9 or 13
    jobs), through the enqueue-only run with its default launch shapes:
    every job's active and zoomed qubits as the FP64 oracle's (the same bins
    expanded), and per job a total variation <= 1e-6 and a float64 total
    within 1e-6 of the oracle's."""
    import torch
    from oracle import attribution, dd
    from workloads.configs import dd_batched
    w = [x for x in dd_batched() if x.n == n_qubits][0]
    subs = w.subcircuits
    var = w.variants()
    A = [attribution.attribute(v, s.w, s.in_local, s.out_local, s.in_edge, s.out_edge) for s, v in zip(subs, var)]
    att = [cq.cutqc_attribute(s, torch.from_numpy(v).cuda()) for s, v in zip(subs, var)]
    M, R, T = 16, 6, 4
    jobs, n_jobs, bins = cq.cutqc_dd_run_async(subs, att, w.n, M, R, T, max_jobs=64)
    got = cq.dd_jobs_from_device(jobs, n_jobs)
    ref = dd.run(A, [s.out_qubit for s in subs], [s.edges for s in subs], w.K, w.n, M, R, T, strategy="bfs")
    assert len(got) == len(ref) == n_jobs
    for J, rj in zip(got, ref):
        assert list(J.active[:J.n_active]) == rj["active"]
        assert J.zoom() == rj["zoom"]
        b = bins[J.bins_offset:J.bins_offset + (1 << J.n_active)].cpu().numpy().astype(np.float64)
        _gate_job(b, rj["bins"], J.bin_sum)
    assert cq.cutqc_device_status() == 0


@pytest.mark.parametrize("T", [1, 4])
def test_dd_dense_topk_candidates_with_ties(cq, T):
    """One dense job (every output active, 2^20 bins: the selection takes
    the chunked two-pass route) on the tensor-core path: two synthetic
    subcircuits joined by one cut, attributed entries small integers (the
    FP16 hi/lo products and sums are then exact), so many bins tie.  The T
    selected bins must be exactly the first T of the order (value
    descending, bin index ascending) over the bins written."""
    import torch
    from types import SimpleNamespace
    o0, o1 = 10, 10
    s0 = SimpleNamespace(w=o0 + 1, in_local=[], in_edge=[], out_local=[o0], out_edge=[0],
                         out_qubit=list(range(o1, o1 + o0)), edges=[0], o=o0)
    s1 = SimpleNamespace(w=o1, in_local=[0], in_edge=[0], out_local=[], out_edge=[],
                         out_qubit=list(range(o1)), edges=[0], o=o1)
    rng = np.random.default_rng(40 + T)
    att = [torch.from_numpy(rng.integers(0, 3, size=(1 << s.o, 4)).astype(np.float32)).cuda() for s in (s0, s1)]
    n = o0 + o1
    jobs, n_jobs, bins = cq.cutqc_dd_run_async([s0, s1], att, n, n, 1, T, max_jobs=2,
                                               options={"precision": 1, "tc_min_outputs": 1})
    js = cq.dd_jobs_from_device(jobs, n_jobs)
    assert len(js) == 1 and js[0].n_active == n
    b = bins[:1 << n].cpu().numpy().astype(np.float64)
    A0, A1 = (a.cpu().numpy().astype(np.float64) for a in att)
    # bin index: bit j = active qubit j; s1 owns qubits 0..9, s0 owns 10..19
    ref = (A0 @ A1.T).reshape(-1) * 0.5
    assert np.array_equal(b, ref)
    order = np.lexsort((np.arange(1 << n), -b))[:T]
    assert list(js[0].top_idx[:T]) == [int(i) for i in order]
    assert [float(v) for v in js[0].top_val[:T]] == [float(b[i]) for i in order]
    assert len(np.unique(b)) < (1 << n) // 100          # ties are plentiful
    assert cq.cutqc_device_status() == 0


def _two_sub_dense_job(cq, o0, o1, T, A0, A1):
    """A dense job of two synthetic subcircuits joined by one cut (every
    output active, 2^(o0+o1) bins) on the tensor-core path.  Returns the
    job record and the bins written."""
    import torch
    from types import SimpleNamespace
    s0 = SimpleNamespace(w=o0 + 1, in_local=[], in_edge=[], out_local=[o0], out_edge=[0],
                         out_qubit=list(range(o1, o1 + o0)), edges=[0], o=o0)
    s1 = SimpleNamespace(w=o1, in_local=[0], in_edge=[0], out_local=[], out_edge=[],
                         out_qubit=list(range(o1)), edges=[0], o=o1)
    att = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda() for a in (A0, A1)]
    n = o0 + o1
    jobs, n_jobs, bins = cq.cutqc_dd_run_async([s0, s1], att, n, n, 1, T, max_jobs=2, options={"precision": 1})
    js = cq.dd_jobs_from_device(jobs, n_jobs)
    assert len(js) == 1 and js[0].n_active == n
    return js[0], bins[:1 << n].cpu().numpy().astype(np.float64)


@pytest.mark.gpu
@pytest.mark.parametrize("case,T", [("uniform", 1), ("uniform", 4), ("uniform", 32), ("planted", 4),
                                    ("planted", 8), ("small_ints", 4)])
def test_dd_topk_from_block_maxima(cq, case, T):
    """Jobs of 2^24 bins on the tensor-core path, where the final GEMM also
    writes the largest value of each 32 x 64 block of its output and the
    selection reads again only the blocks whose maximum reaches the T-th
    largest block maximum.  Cases: distinct uniform values (exactly T
    blocks); five planted bins of one top value in separate blocks (T = 4:
    five blocks tie at the threshold; T = 8: the threshold value is held by
    about a hundred bins, more blocks than are read again, so the full scan
    runs); small-integer entries (every top value tied across many blocks).
    The T selected bins must be exactly the first T of the order (value
    descending, bin index ascending) over the bins written."""
    o0 = o1 = 12
    rng = np.random.default_rng(700 + T + len(case))
    if case == "uniform":
        A0 = rng.random((1 << o0, 4))
        A1 = rng.random((1 << o1, 4))
    else:
        A0 = rng.integers(0, 3, size=(1 << o0, 4)).astype(np.float64)
        A1 = rng.integers(0, 3, size=(1 << o1, 4)).astype(np.float64)
        if case == "planted":
            r = int(rng.integers(0, 1 << o0))
            cols = rng.choice(1 << o1, size=5, replace=False)
            A0[r] = 3.0
            A1[cols] = 3.0
            assert len(set(int(c) // 64 for c in cols)) == 5      # five separate blocks
    job, b = _two_sub_dense_job(cq, o0, o1, T, A0, A1)
    if case != "uniform":
        assert np.array_equal(b, (A0 @ A1.T).reshape(-1) * 0.5)   # exact: small integers
    order = np.lexsort((np.arange(b.size), -b))[:T]
    assert list(job.top_idx[:T]) == [int(i) for i in order]
    assert [float(v) for v in job.top_val[:T]] == [float(b[i]) for i in order]
    if case == "planted":
        assert np.sum(b == b.max()) == 5
    assert cq.cutqc_device_status() == 0


@pytest.mark.gpu
def test_dd_topk_from_block_maxima_batched_level(cq):
    """A second level of four jobs of 2^22 bins each (two synthetic
    subcircuits of 22 outputs joined by one cut, M = 22): the level's GEMM
    runs once per job with each job's block maxima at its own offset.  Each
    job's T selected bins must be the first T of the order (value
    descending, index ascending) over that job's bins."""
    import torch
    from types import SimpleNamespace
    o0 = o1 = 22
    T = 4
    s0 = SimpleNamespace(w=o0 + 1, in_local=[], in_edge=[], out_local=[o0], out_edge=[0],
                         out_qubit=list(range(o1, o1 + o0)), edges=[0], o=o0)
    s1 = SimpleNamespace(w=o1, in_local=[0], in_edge=[0], out_local=[], out_edge=[],
                         out_qubit=list(range(o1)), edges=[0], o=o1)
    rng = np.random.default_rng(722)
    att = [torch.from_numpy(rng.random((1 << o, 4), dtype=np.float32)).cuda() for o in (o0, o1)]
    n = o0 + o1
    jobs, n_jobs, bins = cq.cutqc_dd_run_async([s0, s1], att, n, 22, 2, T, max_jobs=1 + T,
                                               options={"precision": 1})
    js = cq.dd_jobs_from_device(jobs, n_jobs)
    level1 = [j for j in js if j.level == 1]
    assert len(level1) == T
    for j in level1:
        assert j.n_active == 22
        b = bins[j.bins_offset:j.bins_offset + (1 << 22)].cpu().numpy().astype(np.float64)
        order = np.lexsort((np.arange(b.size), -b))[:T]
        assert list(j.top_idx[:T]) == [int(i) for i in order]
        assert [float(v) for v in j.top_val[:T]] == [float(b[i]) for i in order]
    assert cq.cutqc_device_status() == 0
