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
