"""Autotuner for the enqueue-only dynamic-definition run.

`cutqc_dd_run_async` takes launch-shape options (how many CTAs share one
subcircuit's merge, threads per job of the top-T pass).  The best setting
depends on the subcircuits' sizes and on how many active, merged and zoomed
qubits each level gives them, so it is chosen per workload shape: each
candidate runs the caller's own data as a captured CUDA graph, its bins and
job records are checked against the default setting's, and the fastest
matching one is cached under the shape key.
"""
from __future__ import annotations

from . import cutqc as cq

CANDIDATES = [dict(merge_ctas=m, topk_threads=t) for m in (1024, 256, 4096) for t in (1024, 256)]
_CACHE = {}


def shape_key(subs, n, M, R, T, precision=0):
    return (n, M, R, T, precision,
            tuple((int(s.w), len(s.in_local), len(s.out_local), tuple(s.out_qubit)) for s in subs))


def _time_graph(run, reps):
    import torch
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        run()
    g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_dd(subs, attributed, n, M, R, T, max_jobs=64, reps=5, candidates=None, atol=1e-6, precision=0):
    """Returns (best options dict, [(ms, options, matches_default), ...]).
    ``precision`` (0 FP32, 1 split-precision tensor cores) is fixed; only the
    launch shapes are searched."""
    import torch
    key = shape_key(subs, n, M, R, T, precision)
    if key in _CACHE:
        return _CACHE[key]
    dev = attributed[0].device
    ws = torch.empty(max(1, cq.cutqc_dd_run_workspace_size(subs, n, M, T)), dtype=torch.uint8, device=dev)
    ref = None
    results = []
    for opt in candidates or CANDIDATES:
        opt = dict(opt, precision=precision)
        jobs, n_jobs, bins = cq.cutqc_dd_run_async(subs, attributed, n, M, R, T, max_jobs=max_jobs, ws=ws,
                                                   options=opt)
        torch.cuda.synchronize()

        def run(jobs=jobs, n_jobs=n_jobs, bins=bins, opt=opt):
            cq.cutqc_dd_run_async(subs, attributed, n, M, R, T, jobs=jobs, n_jobs=n_jobs, bins=bins, ws=ws,
                                  options=opt)
        ms = _time_graph(run, reps)
        recs = cq.dd_jobs_from_device(jobs, n_jobs)
        if ref is None:
            ref = (recs, bins.clone())
            ok = True
        else:
            rrecs, rbins = ref
            ok = len(recs) == len(rrecs) and all(
                (a.parent, a.parent_bin, a.n_active) == (b.parent, b.parent_bin, b.n_active) and
                bool(torch.allclose(bins[a.bins_offset:a.bins_offset + (1 << a.n_active)],
                                    rbins[b.bins_offset:b.bins_offset + (1 << b.n_active)], atol=atol, rtol=0))
                for a, b in zip(recs, rrecs))
        results.append((ms, dict(opt), ok))
    best = min((r for r in results if r[2]), key=lambda r: r[0])[1]
    _CACHE[key] = (best, results)
    return best, results


# ------------------------------------------------- the persistent DD batch
# One launch for several circuits (cutqc_dd_batch_*): the shape options are
# the merge slicing (merge_ctas), the bins per top-T task (topk_chunk), the
# grid (ctas, 0 = every CTA that fits at once), the CTAs per SM the
# kernel's registers are budgeted for (ctas_per_sm) and the GEMM tile shape of
# the contraction steps (narrow_max_n).  Each candidate builds the
# batch over the caller's runs (fresh output buffers), replays it as a
# captured graph, and is kept only if its records and bins match the first
# candidate's.

# tile shapes: narrow_max_n = the most columns a contraction step may have
# and still take 256 x 16 tiles (-1: every step takes 64 x 64 tiles)
BATCH_CANDIDATES = [dict(merge_ctas=1024, topk_chunk=c, ctas=0, ctas_per_sm=r, narrow_max_n=nm)
                    for r in (3, 2, 4) for c in (2048, 4096) for nm in (16, -1, 64)]


def batch_shape_key(runs):
    return tuple(shape_key(r["subs"], r["n_qubits"], r["M"], r["R"], r["T"]) for r in runs)


def tune_dd_batch(runs, reps=5, candidates=None, atol=1e-6):
    """runs: dicts for cq.cutqc_dd_batch_create (their buffers are not
    touched: each candidate gets its own).  Returns (best options dict,
    [(ms, options, matches_first), ...])."""
    import torch
    key = batch_shape_key(runs)
    if key in _CACHE:
        return _CACHE[key]
    ref = None
    results = []
    for opt in candidates or BATCH_CANDIDATES:
        mine = [cq.dd_batch_run(r["subs"], r["attributed"], r["n_qubits"], r["M"], r["R"], r["T"],
                                max_jobs=r["jobs"].numel() // cq.ctypes.sizeof(cq.DDJob)) for r in runs]
        batch = cq.cutqc_dd_batch_create(mine, opt)
        ms = _time_graph(lambda b=batch: b.launch(torch.cuda.current_stream()), reps)
        recs = [cq.dd_jobs_from_device(m["jobs"], m["n_jobs"]) for m in mine]
        if ref is None:
            ref = (recs, [m["bins"].clone() for m in mine])
            ok = True
        else:
            ok = all(
                len(rs) == len(rr) and all(
                    (a.parent, a.parent_bin, a.n_active) == (b.parent, b.parent_bin, b.n_active) and
                    bool(torch.allclose(mb[a.bins_offset:a.bins_offset + (1 << a.n_active)],
                                        rb[b.bins_offset:b.bins_offset + (1 << b.n_active)], atol=atol, rtol=0))
                    for a, b in zip(rs, rr))
                for rs, rr, mb, rb in zip(recs, ref[0], [m["bins"] for m in mine], ref[1]))
        results.append((ms, dict(opt), ok))
        batch.close()
    best = min((r for r in results if r[2]), key=lambda r: r[0])[1]
    _CACHE[key] = (best, results)
    return best, results


# ---------------------------------------------------------------- FD
# The tensor-core contraction on SM pairs: the work-item size (consecutive
# 128-column tiles per 256-row block of the row operand; 0 = chosen per launch
# to balance the pairs).  Each candidate reconstructs the caller's own
# subcircuits as a captured graph; its output must equal the default's bit
# for bit (the tiling changes no output, only the float64 total's order).

FD_CANDIDATES = [0, 16, 32, 48, 64, 96, 128]


def tune_fd(subs, attributed, precision=1, reps=5, candidates=None, out=None, ws=None):
    """Returns (best tiles_per_item, [(ms, tiles_per_item, identical), ...])
    and leaves the best one set (cutqc_fd_set_tiles_per_item).  out / ws:
    optional buffers for the trial reconstructions (2^n floats; the FD
    workspace)."""
    import torch
    key = ("fd", precision, tuple((int(s.w), len(s.in_local), len(s.out_local), tuple(s.out_qubit)) for s in subs))
    if key in _CACHE:
        best, results = _CACHE[key]
        cq.cutqc_fd_set_tiles_per_item(best)
        return best, results
    dev = attributed[0].device
    n = sum(int(s.w) - len(s.out_local) for s in subs)
    if out is None:
        out = torch.empty(1 << n, dtype=torch.float32, device=dev)
    ref = None
    if ws is None:
        ws = torch.empty(max(1, cq.cutqc_reconstruct_fd_workspace_size(subs, precision)), dtype=torch.uint8,
                         device=dev)
    results = []
    for t in candidates or FD_CANDIDATES:
        cq.cutqc_fd_set_tiles_per_item(t)
        cq.cutqc_reconstruct_fd(subs, attributed, cq.ORDER_KRON, precision, out=out, ws=ws)
        torch.cuda.synchronize()
        ms = _time_graph(lambda: cq.cutqc_reconstruct_fd(subs, attributed, cq.ORDER_KRON, precision, out=out, ws=ws),
                         reps)
        if ref is None:
            ref = out.clone()
            same = True
        else:
            same = bool(torch.equal(out, ref))
        results.append((ms, t, same))
    del ref
    best = min((r for r in results if r[2]), key=lambda r: r[0])[1]
    cq.cutqc_fd_set_tiles_per_item(best)
    _CACHE[key] = (best, results)
    return best, results
