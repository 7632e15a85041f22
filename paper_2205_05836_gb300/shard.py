"""Sharding of one reconstruction over several GPUs (one process each).

The final contraction's rows are the high output bits (Kronecker order), so
a rank that writes rows [r0, r1) writes the contiguous output range
[r0 * cols, r1 * cols): no exchange is needed on the data path.  The only
collective is the max-over-ranks of the step time (and, if wanted, the sum of
the per-rank totals)."""
from __future__ import annotations


def row_range(rows: int, world: int, rank: int):
    """Contiguous, balanced split of `rows` rows: the first rows % world ranks
    get one extra row."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    base, extra = divmod(rows, world)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, group=None):
    """Max of a per-rank float over the process group (CPU tensor for gloo,
    device tensor for nccl)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return float(value)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


# ------------------------------------------------------------------ DD
# Algorithm 1 breadth first over several GPUs.  The bin jobs of a level are
# independent: each rank reconstructs a contiguous share of them, and the one
# exchange per level is an all-gather of every job's T best (value, bin)
# candidates, from which every rank picks the same T jobs of the next level
# (Algorithm 1's list L, truncated to T).


def merge_level_candidates(tops, T):
    """tops: per job of the level, in job order, its candidates [(value,
    bin), ...] in the job's own order.  Returns the T best (job, bin) pairs
    by value, larger first; equal values keep job order, then each job's own
    order (the order the single-GPU selection uses)."""
    flat = [(-float(v), j, t, int(b)) for j, lst in enumerate(tops) for t, (v, b) in enumerate(lst)]
    flat.sort(key=lambda x: (x[0], x[1], x[2]))
    return [(j, b) for _, j, _, b in flat[:T]]


def _gather(obj, group):
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return [obj]
    out = [None] * dist.get_world_size(group)
    dist.all_gather_object(out, obj, group=group)
    return out


def dd_run_sharded(execute_level, n, M, R, T, group=None):
    """Breadth-first Algorithm 1 with the jobs of each level split over the
    ranks of `group` (all ranks call it with the same arguments).

    execute_level(level, jobs) reconstructs this rank's jobs -- each a dict
    with `active` (qubits, ascending) and `zoom` (qubit -> bit) -- and returns
    per job a dict with `bin_sum` and `top` ([(value, bin)], the job's T best
    bins, empty when no merged qubit remains).  Returns the records of all
    jobs in level order, on every rank: active, zoom, level, parent,
    parent_bin, bin_sum, top (and `bins`, where the executor returns them,
    on the rank that reconstructed the job)."""
    import torch.distributed as dist
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    records = []
    level_jobs = [dict(zoom={}, parent=-1, parent_bin=-1)]
    for level in range(max(1, min(R, -(-n // M)))):
        lo = level * M
        active = list(range(lo, min(n, lo + M)))
        for jb in level_jobs:
            jb["active"] = active
            jb["level"] = level
        j0, j1 = row_range(len(level_jobs), world, rank)
        mine = execute_level(level, level_jobs[j0:j1]) if j1 > j0 else []
        # only the totals and candidates travel; the bins stay on their rank
        payload = [dict(bin_sum=float(r["bin_sum"]), top=[(float(v), int(b)) for v, b in r["top"]]) for r in mine]
        results = [r for part in _gather(payload, group) for r in part]
        base = len(records)
        for j, (jb, res) in enumerate(zip(level_jobs, results)):
            rec = dict(jb, bin_sum=res["bin_sum"], top=list(res["top"]))
            if j0 <= j < j1 and "bins" in mine[j - j0]:
                rec["bins"] = mine[j - j0]["bins"]
            records.append(rec)
        sel = merge_level_candidates([r["top"] for r in results], T)
        if not sel:
            break
        nxt = []
        for j, b in sel:
            parent = records[base + j]
            z = dict(parent["zoom"])
            for a, q in enumerate(parent["active"]):
                z[q] = (b >> a) & 1
            nxt.append(dict(zoom=z, parent=base + j, parent_bin=b))
        level_jobs = nxt
    return records


def gpu_level_executor(cq, subs, attributed, n, M, T, stream=None):
    """execute_level for dd_run_sharded on this process's GPU: per subcircuit
    one merge launch for the rank's jobs (zoom values per job from the host),
    then one batched bin reconstruction with the top-T selection."""
    import torch

    def run(level, jobs):
        dev = attributed[0].device
        active = jobs[0]["active"]
        rank_of = {q: j for j, q in enumerate(active)}
        nj = len(jobs)
        merged, active_bits, bin_bit = [], [], []
        for s, att in zip(subs, attributed):
            amask = zmask = 0
            zvals = [0] * nj
            a = 0
            for t, q in enumerate(s.out_qubit):
                if q in rank_of:
                    amask |= 1 << t
                    bin_bit.append(rank_of[q])
                    a += 1
                elif q in jobs[0]["zoom"]:
                    zmask |= 1 << t
                    for j, jb in enumerate(jobs):
                        zvals[j] |= jb["zoom"][q] << t
            k = len(s.in_local) + len(s.out_local)
            out = torch.empty((nj, 1 << a, 4 ** k), dtype=torch.float32, device=dev)
            zdev = torch.tensor(zvals, dtype=torch.int64).to(dev)
            cq.cutqc_dd_merge_batch(s, att, amask, zmask, zdev, out, stream=stream)
            merged.append(out)
            active_bits.append(a)
        na = len(active)
        bins = torch.empty((nj, 1 << na), dtype=torch.float32, device=dev)
        bsum = torch.zeros(nj, dtype=torch.float64, device=dev)
        Tk = max(1, T)
        tidx = torch.empty((nj, Tk), dtype=torch.int32, device=dev)
        tval = torch.empty((nj, Tk), dtype=torch.float32, device=dev)
        cq.cutqc_dd_step(subs, active_bits, bin_bit, merged, bins, bin_sum=bsum, topk=T, top_idx=tidx, top_val=tval,
                         stream=stream)
        has_merged = active[-1] + 1 < n
        ti, tv, bs = tidx.cpu().tolist(), tval.cpu().tolist(), bsum.cpu().tolist()
        out = []
        for j in range(nj):
            top = [(tv[j][t], ti[j][t]) for t in range(T) if ti[j][t] >= 0] if (has_merged and T > 0) else []
            out.append(dict(bin_sum=bs[j], top=top, bins=bins[j]))
        return out
    return run


# ------------------------------------------------- DD batches over ranks
# Several circuits' runs are independent: each rank builds one persistent
# batch (cutqc_dd_batch_*) over its share of the runs, with no collective on
# the data path.  Shares are balanced by the runs' bin counts (longest first
# to the least-loaded rank), the same on every rank.


def dd_run_bins(n, M, R, T):
    """Bins a breadth-first run reconstructs: level 0 one job, every later
    level T jobs, 2^(active qubits) bins each; min(R, ceil(n / M)) levels
    (one when T = 0)."""
    depths = -(-n // M)
    levels = min(R, depths) if T > 0 else 1
    return sum((1 if lv == 0 else T) << (min(n, lv * M + M) - lv * M) for lv in range(levels))


def assign_runs(work, world):
    """Rank of each run: runs in decreasing work (index order for equal
    work) each go to the rank with the least work so far (lowest rank for
    equal loads)."""
    if world < 1:
        raise ValueError("bad world")
    load = [0] * world
    rank_of = [0] * len(work)
    for i in sorted(range(len(work)), key=lambda i: (-work[i], i)):
        r = min(range(world), key=lambda r: (load[r], r))
        rank_of[i] = r
        load[r] += work[i]
    return rank_of


def my_runs(runs, world, rank):
    """Indices of the runs (dicts with n_qubits, M, R, T) this rank builds
    its batch from."""
    work = [dd_run_bins(r["n_qubits"], r["M"], r["R"], r["T"]) for r in runs]
    return [i for i, r in enumerate(assign_runs(work, world)) if r == rank]
