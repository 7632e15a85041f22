"""Python binding of libcutqc (include/cutqc.h): argument marshalling only.

Every function here has the name of the C entry point it calls and forwards
to it through ctypes; torch tensors are used only to own device memory and to
name the CUDA stream.  There is no fallback: if the shared library is missing
the import of a compute function raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_float, c_int, c_int8, c_int32, c_int64, c_size_t, c_uint64, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libcutqc.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "cutqc.h")
HEADERS = [HEADER, os.path.join(os.path.dirname(HERE), "include", "cutqc_mlp.h")]

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = 0, -1, -2, -3, -4, -5
F64, F32 = 0, 1
ORDER_KRON, ORDER_ORIGINAL = 0, 1
PREC_FP32_SIMT, PREC_FP16X3_TC, PREC_FP16X3_TC_PRUNE = 0, 1, 2
PRUNE_TOL = 2.0 ** -30   # L1 bound of the cut terms the pruned precision may skip


class CutqcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"cutqc error {code}: {msg}")
        self.code = code


class _Sub(ctypes.Structure):
    _fields_ = [("w", c_int32), ("k_in", c_int32), ("k_out", c_int32),
                ("in_local", POINTER(c_int32)), ("out_local", POINTER(c_int32)),
                ("in_edge", POINTER(c_int32)), ("out_edge", POINTER(c_int32)),
                ("out_qubit", POINTER(c_int32))]


_lib = None


def lib():
    """Load libcutqc.so (built by paper_2205_05836_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libcutqc.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.cutqc_last_error.restype = c_char_p
        L.cutqc_version.restype = c_char_p
        _lib = L
    return _lib


def _check(rc):
    if rc != OK:
        raise CutqcError(rc, lib().cutqc_last_error().decode())


def _arr(xs):
    xs = [int(x) for x in xs]
    a = (c_int32 * max(1, len(xs)))(*xs)
    return a


def make_sub(s):
    """ctypes descriptor from any object with w, in_local, out_local,
    in_edge, out_edge, out_qubit (e.g. workloads.cutting.Subcircuit).  The
    returned tuple keeps the arrays alive."""
    arrays = [_arr(s.in_local), _arr(s.out_local), _arr(s.in_edge), _arr(s.out_edge), _arr(s.out_qubit)]
    d = _Sub(int(s.w), len(s.in_local), len(s.out_local),
             ctypes.cast(arrays[0], POINTER(c_int32)), ctypes.cast(arrays[1], POINTER(c_int32)),
             ctypes.cast(arrays[2], POINTER(c_int32)), ctypes.cast(arrays[3], POINTER(c_int32)),
             ctypes.cast(arrays[4], POINTER(c_int32)))
    return d, arrays


def _subs(subs):
    keep, arr = [], (_Sub * len(subs))()
    for i, s in enumerate(subs):
        d, a = make_sub(s)
        arr[i] = d
        keep.append(a)
    return arr, keep


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return c_void_p(stream.cuda_stream)


def _ptr(t):
    return c_void_p(0 if t is None else t.data_ptr())


# ------------------------------------------------------------------ misc

def cutqc_version():
    return lib().cutqc_version().decode()


def cutqc_last_error():
    return lib().cutqc_last_error().decode()


def cutqc_device_status():
    v = c_int32(0)
    _check(lib().cutqc_device_status(ctypes.byref(v)))
    return v.value


def cutqc_kernel_launches():
    """Kernels the library has enqueued (or captured) in this process."""
    v = c_int64(0)
    _check(lib().cutqc_kernel_launches(ctypes.byref(v)))
    return v.value


def cutqc_selftest_wait_timeout(waited=None, stream=None):
    """Launches the bounded-wait self test (a wait nothing satisfies); the
    device status word then reads CUTQC_ETIMEOUT (cutqc_device_status)."""
    _check(lib().cutqc_selftest_wait_timeout(_ptr(waited), _stream(stream)))
    return waited


def cutqc_sum_f64(x, out=None, stream=None):
    import torch
    if out is None:
        out = torch.zeros(1, dtype=torch.float64, device=x.device)
    _check(lib().cutqc_sum_f64(_ptr(x), c_int64(x.numel()), _ptr(out), _stream(stream)))
    return out


# ------------------------------------------------------------ attribution

def cutqc_attribute_workspace_size(sub):
    d, keep = make_sub(sub)
    n = c_size_t(0)
    _check(lib().cutqc_attribute_workspace_size(ctypes.byref(d), ctypes.byref(n)))
    return n.value


def cutqc_attribute(sub, variants, out=None, ws=None, stream=None):
    """variants: device tensor [4^k_in, 3^k_out, 2^w] (float64 or float32).
    Returns the attributed tensor [2^o, 4^k] float32."""
    import torch
    d, keep = make_sub(sub)
    kin, kout = len(sub.in_local), len(sub.out_local)
    o = int(sub.w) - kout
    if out is None:
        out = torch.empty((1 << o, 4 ** (kin + kout)), dtype=torch.float32, device=variants.device)
    need = cutqc_attribute_workspace_size(sub)
    if ws is None and need:
        ws = torch.empty(need, dtype=torch.uint8, device=variants.device)
    dtype = F64 if variants.dtype == torch.float64 else F32
    _check(lib().cutqc_attribute(ctypes.byref(d), _ptr(variants), c_int(dtype), _ptr(out), _ptr(ws),
                                 c_size_t(0 if ws is None else ws.numel()), _stream(stream)))
    return out


def cutqc_attribute_noalloc(sub, variants, out, stream=None):
    """cutqc_attribute without any device allocation: the caller passes the
    output tensor; the library's static scratch array is used."""
    import torch
    d, keep = make_sub(sub)
    kin, kout = len(sub.in_local), len(sub.out_local)
    shape = (1 << (int(sub.w) - kout), 4 ** (kin + kout))
    if variants.dtype not in (torch.float64, torch.float32):
        raise TypeError("variants must be float64 or float32")
    if not variants.is_contiguous() or variants.numel() != 4 ** kin * 3 ** kout * (1 << int(sub.w)):
        raise ValueError("variants must be a contiguous [4^k_in, 3^k_out, 2^w] tensor")
    if (out.dtype != torch.float32 or not out.is_contiguous() or out.device != variants.device
            or tuple(out.shape) != shape):
        raise ValueError(f"out must be a contiguous float32 tensor of shape {shape} on {variants.device}")
    dtype = F64 if variants.dtype == torch.float64 else F32
    _check(lib().cutqc_attribute_noalloc(ctypes.byref(d), _ptr(variants), c_int(dtype), _ptr(out), _stream(stream)))
    return out


# --------------------------------------------------------------------- FD

def cutqc_fd_shape(subs):
    arr, keep = _subs(subs)
    r, c = c_int64(0), c_int64(0)
    _check(lib().cutqc_fd_shape(c_int(len(subs)), arr, ctypes.byref(r), ctypes.byref(c)))
    return r.value, c.value


def cutqc_fd_timing_events(start=None, stop=None):
    """The next cutqc_reconstruct_fd on this thread records the two
    torch.cuda.Event objects (created with enable_timing=True) around its
    last contraction's GEMM launch; None, None cancels."""
    if start is None and stop is None:
        _check(lib().cutqc_fd_timing_events(None, None))
        return
    for e in (start, stop):
        if not e.cuda_event:          # torch creates the CUDA event on first record
            e.record()
    _check(lib().cutqc_fd_timing_events(c_void_p(start.cuda_event), c_void_p(stop.cuda_event)))


def cutqc_fd_input_events(events=None):
    """The next cutqc_reconstruct_fd on this thread waits, in each step that
    reads subcircuit i's tensor, for events[i] (a recorded torch.cuda.Event,
    or None: ready at the call) instead of needing every input written when
    it is issued; None or [] clears."""
    events = list(events or [])
    for e in events:
        if e is not None and not e.cuda_event:
            raise ValueError("record each input event before passing it")
    arr = (c_void_p * max(1, len(events)))(*[None if e is None else e.cuda_event for e in events])
    _check(lib().cutqc_fd_input_events(c_int(len(events)), arr if events else None))


def cutqc_fd_set_tiles_per_item(tiles_per_item=0):
    """Work-item size of the tensor-core contraction (0: automatic)."""
    _check(lib().cutqc_fd_set_tiles_per_item(c_int(int(tiles_per_item))))


def cutqc_reconstruct_fd_workspace_size(subs, precision):
    arr, keep = _subs(subs)
    n = c_size_t(0)
    _check(lib().cutqc_reconstruct_fd_workspace_size(c_int(len(subs)), arr, c_int(precision), ctypes.byref(n)))
    return n.value


def cutqc_reconstruct_fd(subs, attributed, out_order=ORDER_KRON, precision=PREC_FP16X3_TC, row_begin=0,
                         row_end=-1, out=None, sum_out=None, ws=None, stream=None, input_events=None):
    """Eq. 1 over the subcircuits.  Returns (out, sum_out).  input_events:
    optional recorded torch.cuda.Event per subcircuit (None = ready), see
    cutqc_fd_input_events."""
    import torch
    arr, keep = _subs(subs)
    dev = attributed[0].device
    n = sum(int(s.w) - len(s.out_local) for s in subs)
    if out is None:
        if row_begin == 0 and row_end == -1:
            numel = 1 << n
        else:
            rows, cols = cutqc_fd_shape(subs)
            numel = ((rows if row_end < 0 else row_end) - row_begin) * cols
        out = torch.empty(numel, dtype=torch.float32, device=dev)
    need = cutqc_reconstruct_fd_workspace_size(subs, precision)
    if ws is None and need:
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
    ptrs = (c_void_p * len(attributed))(*[t.data_ptr() for t in attributed])
    if input_events is not None:
        cutqc_fd_input_events(input_events)
    _check(lib().cutqc_reconstruct_fd(c_int(len(subs)), arr, ptrs, c_int(out_order), c_int(precision),
                                      c_int64(row_begin), c_int64(row_end), _ptr(out), _ptr(sum_out), _ptr(ws),
                                      c_size_t(0 if ws is None else ws.numel()), _stream(stream)))
    return out, sum_out


# --------------------------------------------------------------------- DD

def cutqc_dd_merge(sub, attributed, role, out=None, stream=None):
    """role: per output qubit 0 active, 1 merged, 2 zoom->0, 3 zoom->1."""
    import torch
    d, keep = make_sub(sub)
    a = sum(1 for r in role if r == 0)
    k = len(sub.in_local) + len(sub.out_local)
    if out is None:
        out = torch.empty((1 << a, 4 ** k), dtype=torch.float32, device=attributed.device)
    roles = (c_int8 * max(1, len(role)))(*[int(r) for r in role])
    _check(lib().cutqc_dd_merge(ctypes.byref(d), _ptr(attributed), roles, _ptr(out), _stream(stream)))
    return out


def cutqc_dd_merge_batch(sub, attributed, active_mask, zoom_mask, zoom_dev, out, stream=None):
    d, keep = make_sub(sub)
    _check(lib().cutqc_dd_merge_batch(ctypes.byref(d), _ptr(attributed), c_uint64(active_mask), c_uint64(zoom_mask),
                                      c_int(zoom_dev.numel()), _ptr(zoom_dev), _ptr(out), _stream(stream)))
    return out


def cutqc_dd_step_workspace_size(subs, active_bits, n_jobs):
    arr, keep = _subs(subs)
    ab = _arr(active_bits)
    n = c_size_t(0)
    _check(lib().cutqc_dd_step_workspace_size(c_int(len(subs)), arr, ab, c_int(n_jobs), ctypes.byref(n)))
    return n.value


def cutqc_dd_step(subs, active_bits, bin_bit, merged, bins, bin_sum=None, topk=0, top_idx=None, top_val=None,
                  ws=None, stream=None):
    """merged: per subcircuit a device tensor holding the jobs' merged tensors
    back to back ([n_jobs, 2^a_i, 4^k_i]); bins: device tensor [n_jobs, 2^sum(a)]."""
    import torch
    arr, keep = _subs(subs)
    n_jobs = bins.shape[0]
    ab, bb = _arr(active_bits), _arr(bin_bit)
    mp = (c_void_p * len(merged))(*[t.data_ptr() for t in merged])
    need = cutqc_dd_step_workspace_size(subs, active_bits, n_jobs)
    if ws is None and need:
        ws = torch.empty(need, dtype=torch.uint8, device=bins.device)
    _check(lib().cutqc_dd_step(c_int(len(subs)), arr, ab, bb, c_int(n_jobs), mp, _ptr(bins), _ptr(bin_sum),
                               c_int(topk), _ptr(top_idx), _ptr(top_val), _ptr(ws),
                               c_size_t(0 if ws is None else ws.numel()), _stream(stream)))
    return bins


class DDJob(ctypes.Structure):
    _fields_ = [("level", c_int32), ("depth", c_int32), ("parent", c_int32), ("parent_bin", c_int32),
                ("n_active", c_int32), ("active", c_int32 * 32), ("zoom_mask", c_uint64 * 2),
                ("zoom_val", c_uint64 * 2), ("bin_sum", c_double), ("top_idx", c_int32 * 32),
                ("top_val", c_float * 32), ("bins_offset", c_int64)]

    def zoom(self):
        z = {}
        for q in range(128):
            if (self.zoom_mask[q >> 6] >> (q & 63)) & 1:
                z[q] = int((self.zoom_val[q >> 6] >> (q & 63)) & 1)
        return z


def cutqc_dd_run_workspace_size(subs, n_qubits, M, T):
    arr, keep = _subs(subs)
    n = c_size_t(0)
    _check(lib().cutqc_dd_run_workspace_size(c_int(len(subs)), arr, c_int(n_qubits), c_int(M), c_int(T), ctypes.byref(n)))
    return n.value


def cutqc_dd_run(subs, attributed, n_qubits, M, R, T, strategy, max_jobs=256, bins=None, ws=None, stream=None):
    """Algorithm 1 on the device.  strategy 0 = DFS, 1 = BFS.  Returns
    (list of DDJob, bins tensor); job j's bins are
    bins[job.bins_offset : job.bins_offset + 2**job.n_active]."""
    import torch
    arr, keep = _subs(subs)
    dev = attributed[0].device
    if bins is None:
        bins = torch.empty(max_jobs << min(M, n_qubits), dtype=torch.float32, device=dev)
    need = cutqc_dd_run_workspace_size(subs, n_qubits, M, T)
    if ws is None:
        ws = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    jobs = (DDJob * max_jobs)()
    nj = c_int(0)
    ptrs = (c_void_p * len(attributed))(*[t.data_ptr() for t in attributed])
    _check(lib().cutqc_dd_run(c_int(len(subs)), arr, ptrs, c_int(n_qubits), c_int(M), c_int(R), c_int(T),
                              c_int(strategy), c_int(max_jobs), jobs, ctypes.byref(nj), _ptr(bins),
                              c_int64(bins.numel()), _ptr(ws), c_size_t(ws.numel()), _stream(stream)))
    return [jobs[i] for i in range(nj.value)], bins


class DDOptions(ctypes.Structure):
    _fields_ = [("merge_ctas", c_int32), ("topk_threads", c_int32), ("precision", c_int32),
                ("tc_min_outputs", c_int32)]


def cutqc_dd_run_async(subs, attributed, n_qubits, M, R, T, max_jobs=256, jobs=None, n_jobs=None, bins=None, ws=None,
                       stream=None, options=None):
    """Level-by-level Algorithm 1 enqueued without host synchronisation (CUDA
    graph capturable).  jobs: device uint8 tensor of max_jobs records, n_jobs:
    device int32[1]; returns (jobs, n_jobs, bins).  Use dd_jobs_from_device to
    read the records."""
    import torch
    arr, keep = _subs(subs)
    dev = attributed[0].device
    rec = ctypes.sizeof(DDJob)
    if jobs is None:
        jobs = torch.empty(max_jobs * rec, dtype=torch.uint8, device=dev)
    if n_jobs is None:
        n_jobs = torch.zeros(1, dtype=torch.int32, device=dev)
    if bins is None:
        bins = torch.empty(max_jobs << min(M, n_qubits), dtype=torch.float32, device=dev)
    need = cutqc_dd_run_workspace_size(subs, n_qubits, M, T)
    if ws is None:
        ws = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    ptrs = (c_void_p * len(attributed))(*[t.data_ptr() for t in attributed])
    opt = None
    if options is not None:
        opt = ctypes.byref(DDOptions(int(options.get("merge_ctas", 0)), int(options.get("topk_threads", 0)),
                                     int(options.get("precision", 0)), int(options.get("tc_min_outputs", 0))))
    _check(lib().cutqc_dd_run_async(c_int(len(subs)), arr, ptrs, c_int(n_qubits), c_int(M), c_int(R), c_int(T),
                                    c_int(jobs.numel() // rec), _ptr(jobs), _ptr(n_jobs), _ptr(bins),
                                    c_int64(bins.numel()), opt, _ptr(ws), c_size_t(ws.numel()), _stream(stream)))
    return jobs, n_jobs, bins


def dd_jobs_from_device(jobs, n_jobs):
    """Records written by cutqc_dd_run_async (placeholders dropped, parents
    re-indexed into the returned list)."""
    n = int(n_jobs.item())
    raw = jobs.cpu().numpy().tobytes()
    rec = ctypes.sizeof(DDJob)
    allj = [DDJob.from_buffer_copy(raw[i * rec:(i + 1) * rec]) for i in range(n)]
    keep = [i for i, J in enumerate(allj) if J.level >= 0]
    remap = {r: k for k, r in enumerate(keep)}
    out = []
    for r in keep:
        J = allj[r]
        if J.parent >= 0:
            J.parent = remap[J.parent]
        out.append(J)
    return out


class _DDRunDesc(ctypes.Structure):
    _fields_ = [("n_sub", c_int32), ("subcircuits", POINTER(_Sub)), ("attributed_dev", POINTER(c_void_p)),
                ("n_qubits", c_int32), ("M", c_int32), ("R", c_int32), ("T", c_int32), ("max_jobs", c_int32),
                ("jobs_dev", c_void_p), ("n_jobs_dev", c_void_p), ("bins_dev", c_void_p),
                ("bins_capacity", c_int64)]


class DDBatchOptions(ctypes.Structure):
    _fields_ = [("merge_ctas", c_int32), ("topk_chunk", c_int32), ("ctas", c_int32), ("ctas_per_sm", c_int32),
                ("narrow_max_n", c_int32)]


def _batch_descs(runs):
    """runs: dicts with subs, attributed, n_qubits, M, R, T, jobs, n_jobs,
    bins (device tensors as cutqc_dd_run_async takes them)."""
    keep, descs = [], (_DDRunDesc * len(runs))()
    rec = ctypes.sizeof(DDJob)
    for i, r in enumerate(runs):
        arr, k = _subs(r["subs"])
        ptrs = (c_void_p * len(r["attributed"]))(*[t.data_ptr() for t in r["attributed"]])
        keep += [arr, k, ptrs]
        descs[i] = _DDRunDesc(len(r["subs"]), ctypes.cast(arr, POINTER(_Sub)), ctypes.cast(ptrs, POINTER(c_void_p)),
                              int(r["n_qubits"]), int(r["M"]), int(r["R"]), int(r["T"]), r["jobs"].numel() // rec,
                              r["jobs"].data_ptr(), r["n_jobs"].data_ptr(), r["bins"].data_ptr(), r["bins"].numel())
    return descs, keep


def _batch_opts(options):
    if options is None:
        return None
    return ctypes.byref(DDBatchOptions(int(options.get("merge_ctas", 0)), int(options.get("topk_chunk", 0)),
                                       int(options.get("ctas", 0)), int(options.get("ctas_per_sm", 0)),
                                       int(options.get("narrow_max_n", 0))))


def cutqc_dd_batch_workspace_size(runs, options=None):
    descs, keep = _batch_descs(runs)
    n = c_size_t(0)
    _check(lib().cutqc_dd_batch_workspace_size(c_int(len(runs)), descs, _batch_opts(options), ctypes.byref(n)))
    return n.value


def cutqc_dd_batch_shape(runs, options=None):
    """Phases, ops and total tasks of the batch program (host only)."""
    descs, keep = _batch_descs(runs)
    p, o, t = c_int32(0), c_int32(0), c_int64(0)
    _check(lib().cutqc_dd_batch_shape(c_int(len(runs)), descs, _batch_opts(options), ctypes.byref(p), ctypes.byref(o),
                                      ctypes.byref(t)))
    return {"phases": p.value, "ops": o.value, "tasks": t.value}


class DDBatch:
    """Handle of cutqc_dd_batch_create: the runs' program, written into `ws`
    (a device uint8 tensor this object keeps alive).  launch() enqueues the
    persistent launch; the records land in each run's jobs / n_jobs / bins."""

    def __init__(self, runs, options=None, ws=None):
        import torch
        descs, keep = _batch_descs(runs)
        need = cutqc_dd_batch_workspace_size(runs, options)
        dev = runs[0]["bins"].device
        if ws is None:
            ws = torch.empty(need + 256, dtype=torch.uint8, device=dev)
            off = (-ws.data_ptr()) % 256
            ws = ws[off:off + need]
        self.ws = ws
        self.runs = runs
        self._h = c_void_p(0)
        _check(lib().cutqc_dd_batch_create(c_int(len(runs)), descs, _batch_opts(options), _ptr(ws),
                                           c_size_t(ws.numel()), ctypes.byref(self._h)))

    def launch(self, stream=None):
        _check(lib().cutqc_dd_batch_launch(self._h, _stream(stream)))

    def info(self):
        p, o, g = c_int32(0), c_int32(0), c_int32(0)
        _check(lib().cutqc_dd_batch_info(self._h, ctypes.byref(p), ctypes.byref(o), ctypes.byref(g)))
        return {"phases": p.value, "ops": o.value, "ctas": g.value}

    KINDS = ("zero", "merge", "reduce", "contract", "topk", "select")

    def phases(self, cycles=True):
        """Per phase: op kinds, tasks, contraction multiply-adds and
        (cycles=True: synchronous read) the SM cycles it took in the last
        completed launch."""
        n = self.info()["phases"]
        k, t = (c_int32 * max(1, n))(), (c_int32 * max(1, n))()
        f, c = (c_int64 * max(1, n))(), (c_int64 * max(1, n))()
        _check(lib().cutqc_dd_batch_phases(self._h, k, t, f, c if cycles else None, c_int(n)))
        return [{"kinds": [name for b, name in enumerate(self.KINDS) if (k[p] >> b) & 1], "tasks": t[p],
                 "fma": f[p], "cycles": c[p] if cycles else None} for p in range(n)]

    def close(self):
        if self._h and self._h.value:
            lib().cutqc_dd_batch_destroy(self._h)
            self._h = c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cutqc_dd_batch_create(runs, options=None, ws=None):
    """Several circuits' Algorithm 1 (BFS) as one persistent launch; returns a
    DDBatch (call .launch(stream))."""
    return DDBatch(runs, options, ws)


def cutqc_dd_batch_launch(batch, stream=None):
    batch.launch(stream)


def cutqc_dd_batch_info(batch):
    return batch.info()


def cutqc_dd_batch_phases(batch, cycles=True):
    return batch.phases(cycles)


def cutqc_dd_batch_destroy(batch):
    batch.close()


def dd_batch_run(subs, attributed, n_qubits, M, R, T, max_jobs=256):
    """Device buffers of one run of a batch (dict for cutqc_dd_batch_create)."""
    import torch
    dev = attributed[0].device
    return dict(subs=subs, attributed=attributed, n_qubits=n_qubits, M=M, R=R, T=T,
                jobs=torch.empty(max_jobs * ctypes.sizeof(DDJob), dtype=torch.uint8, device=dev),
                n_jobs=torch.zeros(1, dtype=torch.int32, device=dev),
                bins=torch.empty(max_jobs << min(M, n_qubits), dtype=torch.float32, device=dev))


def declared_symbols(headers=None):
    """Function names declared in include/*.h."""
    import re
    names = set()
    for h in headers or HEADERS:
        text = open(h).read()
        names.update(re.findall(r"^\s*(?:int|const char\*)\s+(cutqc_\w+)\s*\(", text, re.M))
    return sorted(names)


# -------------------------------------------------------------------- MLP

class MLP:
    """Device-resident cut-scoring network: FP32 master parameters, BF16
    copy, Adam moments; every step runs in the library's kernels."""

    def __init__(self, params=None, device="cuda", seed=0):
        import torch
        n = c_int64(0)
        _check(lib().cutqc_mlp_param_count(ctypes.byref(n)))
        self.n = n.value
        self.device = torch.device(device)
        if params is None:
            params = init_params(seed)
        self.p = torch.as_tensor(params, dtype=torch.float32).to(self.device).contiguous()
        assert self.p.numel() == self.n
        self.pb = torch.empty(self.n, dtype=torch.bfloat16, device=self.device)
        self.grad = torch.zeros(self.n, dtype=torch.float32, device=self.device)
        self.m = torch.zeros_like(self.grad)
        self.v = torch.zeros_like(self.grad)
        self.loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        self.step = 0
        self._ws = None
        _check(lib().cutqc_mlp_sync_bf16(_ptr(self.p), _ptr(self.pb), _stream(None)))

    def _work(self, batch):
        import torch
        b = c_size_t(0)
        _check(lib().cutqc_mlp_workspace_size(c_int(batch), ctypes.byref(b)))
        if self._ws is None or self._ws.numel() < b.value:
            self._ws = torch.empty(b.value, dtype=torch.uint8, device=self.device)
        return self._ws

    def _rows(self, x, t=None):
        import torch
        if x.dim() != 2 or x.shape[1] != SIZES[0] or x.dtype != torch.float32 or not x.is_contiguous():
            raise ValueError("x must be a contiguous float32 [batch, 64] device tensor")
        if t is not None and (t.shape != (x.shape[0],) or t.dtype != torch.float32 or not t.is_contiguous()):
            raise ValueError("t must be a contiguous float32 [batch] device tensor")
        return x.shape[0]

    def forward(self, x):
        import torch
        B = self._rows(x)
        y = torch.empty(B, dtype=torch.float32, device=self.device)
        ws = self._work(B)
        _check(lib().cutqc_mlp_forward(_ptr(self.p), _ptr(self.pb), _ptr(x), c_int(B), _ptr(y), _ptr(ws),
                                       c_size_t(ws.numel()), _stream(None)))
        return y

    def gradients(self, x, t):
        B = self._rows(x, t)
        ws = self._work(B)
        _check(lib().cutqc_mlp_gradients(_ptr(self.p), _ptr(self.pb), _ptr(x), _ptr(t), c_int(B), _ptr(self.grad),
                                         _ptr(self.loss), _ptr(ws), c_size_t(ws.numel()), _stream(None)))
        return self.grad, self.loss

    def adam(self, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        """Adam update of the parameters from ``self.grad`` (step >= 1)."""
        _check(lib().cutqc_mlp_adam(_ptr(self.p), _ptr(self.pb), _ptr(self.grad), _ptr(self.m), _ptr(self.v),
                                    c_int(step), c_float(lr), c_float(beta1), c_float(beta2), c_float(eps),
                                    _stream(None)))

    def train_step(self, x, t, lr=1e-3):
        B = self._rows(x, t)
        ws = self._work(B)
        self.step += 1
        _check(lib().cutqc_mlp_train_step(_ptr(self.p), _ptr(self.pb), _ptr(self.grad), _ptr(self.m), _ptr(self.v),
                                          c_int(self.step), c_float(lr), _ptr(x), _ptr(t), c_int(B),
                                          _ptr(self.loss), _ptr(ws), c_size_t(ws.numel()), _stream(None)))
        return self.loss


    def fit(self, x, t, steps, batch=512, lr=1e-3, seed=0):
        """``steps`` Adam steps over contiguous minibatches of (x, t), both
        device tensors; the rows are put in a seeded random order once per
        pass over the data.  Returns the device loss tensor of the last step."""
        import numpy as np
        import torch
        N = x.shape[0]
        batch = min(batch, N)
        rng = np.random.default_rng(seed)
        done = 0
        while done < steps:
            perm = torch.from_numpy(rng.permutation(N)).to(x.device)
            xp, tp = x[perm].contiguous(), t[perm].contiguous()
            for b0 in range(0, N - batch + 1, batch):
                if done == steps:
                    break
                self.train_step(xp[b0:b0 + batch], tp[b0:b0 + batch], lr)
                done += 1
        return self.loss

    def params_numpy(self):
        """FP32 master parameters split into (W1, b1, W2, b2, W3, b3)."""
        return split_params(self.p.cpu().numpy())


SIZES = (64, 256, 256, 1)


def split_params(flat):
    """Flat parameter vector -> [W1, b1, W2, b2, W3, b3] ([in][out] weights)."""
    out, o = [], 0
    for a, b in zip(SIZES[:-1], SIZES[1:]):
        out.append(flat[o:o + a * b].reshape(a, b))
        o += a * b
        out.append(flat[o:o + b])
        o += b
    assert o == flat.size
    return out


def init_params(seed=0):
    """He-style initial weights (numpy, float32), layout of cutqc_mlp.h."""
    import numpy as np
    rng = np.random.default_rng(seed)
    parts = []
    for a, b in ((64, 256), (256, 256), (256, 1)):
        parts.append((rng.standard_normal((a, b)) * np.sqrt(2.0 / a)).astype(np.float32).reshape(-1))
        parts.append(np.zeros(b, dtype=np.float32))
    return np.concatenate(parts)
