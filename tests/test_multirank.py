"""Two-rank (gloo, CPU) coverage of the multi-GPU path: the output-row split
of one FD reconstruction reassembles the whole distribution, and the step time
reported is the max over ranks."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q, case):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import attribution, fd
        from paper_2205_05836_gb300 import cutqc
        from paper_2205_05836_gb300.shard import max_over_ranks, row_range
        from workloads import circuits as C
        from workloads.cutting import search_cut
        from workloads.simulate import simulate_variants
        cut = search_cut(*case, restarts=4)
        subs = cut.subcircuits
        A = [attribution.attribute(simulate_variants(s), s.w, s.in_local, s.out_local, s.in_edge, s.out_edge)
             for s in subs]
        # the library's own split (host-side planner, no device): rows of its
        # last contraction = the high output bits in Kronecker order
        rows, cols = cutqc.cutqc_fd_shape(subs)
        assert rows * cols == 2 ** cut.circuit.n
        r0, r1 = row_range(rows, world, rank)
        # this rank's outputs [r0 * cols, r1 * cols): Eq. 1 at each of them
        idx = np.arange(r0 * cols, r1 * cols, dtype=np.int64)
        part = fd.entries(A, [s.edges for s in subs], cut.K, fd.split_kron_index(idx, [s.o for s in subs]))
        t = torch.from_numpy(np.ascontiguousarray(part))
        sizes = [None] * world
        dist.all_gather_object(sizes, t.numel())
        bufs = [torch.zeros(n, dtype=t.dtype) for n in sizes]
        dist.all_gather(bufs, t)
        tmax = max_over_ranks(1.0 + rank)
        if rank == 0:
            whole = torch.cat(bufs).numpy()
            ref = fd.reconstruct_kron(A, [s.edges for s in subs], cut.K)
            q.put((float(np.abs(whole - ref).max()), tmax, sizes))
    finally:
        dist.destroy_process_group()


def _cases():
    from workloads import circuits as C
    return [(C.supremacy(3, 4, 8, 1), 8, 2), (C.aqft(10, 6, max_dist=2), 5, 4)]


@pytest.mark.parametrize("ci", [0, 1], ids=["two_sub", "four_sub"])
def test_two_rank_row_split(ci):
    """Each rank computes the outputs of its rows of the library's last
    contraction (cutqc_fd_shape, shard.row_range) with the FP64 oracle; the
    gathered ranks equal the single-process reconstruction."""
    import __graft_entry__
    __graft_entry__.build()
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q, _cases()[ci])) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
        assert p.exitcode == 0
    err, tmax, sizes = q.get(timeout=10)
    assert err < 1e-15
    assert tmax == 2.0
    assert len(sizes) == 2 and abs(sizes[0] - sizes[1]) <= max(sizes) // 2


def test_row_range_covers_rows():
    from paper_2205_05836_gb300.shard import row_range
    for rows in (1, 7, 8192):
        for world in (1, 2, 3, 8):
            got = [row_range(rows, world, r) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == rows
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            assert max(b - a for a, b in got) - min(b - a for a, b in got) <= 1


def _oracle_level_executor(A, subs, K):
    """execute_level for the sharded DD driver built on the FP64 oracle (the
    CPU stand-in for a rank's GPU in these tests)."""
    from oracle import dd

    def run(level, jobs):
        out = []
        for jb in jobs:
            bins = dd.reconstruct_bins(A, [s.out_qubit for s in subs], [s.edges for s in subs], K, jb["active"],
                                       jb["zoom"])
            n = sum(s.o for s in subs)
            has_merged = jb["active"][-1] + 1 < n
            top = [(float(bins[b]), int(b)) for b in dd._top(bins, _T, has_merged)]
            out.append(dict(bin_sum=float(bins.sum()), top=top))
        return out
    return run


_T = 3


def _dd_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import attribution
        from paper_2205_05836_gb300.shard import dd_run_sharded
        from workloads import circuits as C
        from workloads.cutting import search_cut
        from workloads.simulate import simulate_variants
        cut = search_cut(C.brickwall(10, 4, 11), 7, 2, restarts=4)
        subs = cut.subcircuits
        A = [attribution.attribute(simulate_variants(s), s.w, s.in_local, s.out_local, s.in_edge, s.out_edge)
             for s in subs]
        recs = dd_run_sharded(_oracle_level_executor(A, subs, cut.K), cut.circuit.n, 4, 6, _T)
        q.put((rank, [(r["level"], r["parent"], r["parent_bin"], sorted(r["zoom"].items()), r["bin_sum"],
                       r["top"]) for r in recs]))
    finally:
        dist.destroy_process_group()


def test_two_rank_dd_levels_match_single_process():
    """Breadth-first Algorithm 1 with each level's jobs split over two gloo
    ranks (one all-gather of (value, bin) candidates per level): both ranks
    get the job records of the single-process FP64 oracle run."""
    import torch.multiprocessing as mp
    from oracle import attribution, dd
    from workloads import circuits as C
    from workloads.cutting import search_cut
    from workloads.simulate import simulate_variants
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dd_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    cut = search_cut(C.brickwall(10, 4, 11), 7, 2, restarts=4)
    subs = cut.subcircuits
    A = [attribution.attribute(simulate_variants(s), s.w, s.in_local, s.out_local, s.in_edge, s.out_edge)
         for s in subs]
    ref = dd.run(A, [s.out_qubit for s in subs], [s.edges for s in subs], cut.K, cut.circuit.n, 4, 6, _T,
                 strategy="bfs")
    assert got[0] == got[1]
    assert len(got[0]) == len(ref) > 1
    for (lvl, parent, pbin, zoom, bsum, top), r in zip(got[0], ref):
        assert zoom == sorted(r["zoom"].items())
        assert abs(bsum - r["bins"].sum()) <= 1e-12
        assert [b for _, b in top] == r["top"]


def test_merge_level_candidates_order():
    """The next level's jobs: larger values first; equal values keep job
    order, then each job's own order."""
    from paper_2205_05836_gb300.shard import merge_level_candidates
    tops = [[(0.5, 7), (0.25, 3)], [(0.5, 1), (0.75, 9)], [], [(0.25, 0)]]
    assert merge_level_candidates(tops, 4) == [(1, 9), (0, 7), (1, 1), (0, 3)]
    assert merge_level_candidates(tops, 10)[-1] == (3, 0)
    assert merge_level_candidates([[], []], 3) == []


def test_dd_run_bins_and_assignment():
    """Bin counts of breadth-first runs (the bench's three DD circuits: 9/13/13
    jobs of up to 2^16 bins) and the balanced, deterministic split of runs
    over ranks: every run on exactly one rank, the largest load no more than
    the largest run above the average."""
    from paper_2205_05836_gb300.shard import assign_runs, dd_run_bins, my_runs
    assert dd_run_bins(40, 16, 6, 4) == (1 << 16) + 4 * (1 << 16) + 4 * (1 << 8)
    assert dd_run_bins(60, 16, 6, 4) == (1 << 16) + 2 * 4 * (1 << 16) + 4 * (1 << 12)   # 4 levels, the last 12 wide
    assert dd_run_bins(60, 16, 6, 0) == 1 << 16
    assert dd_run_bins(8, 4, 1, 2) == 1 << 4
    work = [5, 1, 9, 9, 2, 7, 3]
    for world in (1, 2, 3, 8):
        ranks = assign_runs(work, world)
        assert ranks == assign_runs(work, world)
        loads = [sum(w for w, r in zip(work, ranks) if r == k) for k in range(world)]
        assert sum(loads) == sum(work)
        assert max(loads) <= sum(work) / world + max(work)
    assert assign_runs([4, 4], 2) == [0, 1]
    runs = [dict(n_qubits=n, M=16, R=6, T=4) for n in (40, 50, 60)]
    shares = [my_runs(runs, 2, r) for r in range(2)]
    assert sorted(shares[0] + shares[1]) == [0, 1, 2]


def _batch_split_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import attribution, dd
        from paper_2205_05836_gb300.shard import my_runs
        from workloads import circuits as C
        from workloads.cutting import search_cut
        from workloads.simulate import simulate_variants
        cuts = [search_cut(C.brickwall(10, 4, 11), 7, 2, restarts=4), search_cut(C.bv(12, 9), 5, 5, restarts=4),
                search_cut(C.aqft(10, 2, max_dist=2), 5, 4, restarts=4)]
        runs = [dict(n_qubits=c.circuit.n, M=4, R=6, T=2) for c in cuts]
        out = {}
        for i in my_runs(runs, world, rank):      # this rank's batch: the FP64 oracle stands in for its GPU
            c = cuts[i]
            A = [attribution.attribute(simulate_variants(s), s.w, s.in_local, s.out_local, s.in_edge, s.out_edge)
                 for s in c.subcircuits]
            recs = dd.run(A, [s.out_qubit for s in c.subcircuits], [s.edges for s in c.subcircuits], c.K,
                          c.circuit.n, 4, 6, 2, strategy="bfs")
            out[i] = [(sorted(r["zoom"].items()), float(r["bins"].sum())) for r in recs]
        parts = [None] * world
        dist.all_gather_object(parts, out)
        if rank == 0:
            q.put(parts)
    finally:
        dist.destroy_process_group()


def test_two_rank_dd_batch_split():
    """Three DD runs split over two gloo ranks by my_runs: each run is
    computed by exactly one rank, and the gathered records equal the
    single-process FP64 oracle runs."""
    import torch.multiprocessing as mp
    from oracle import attribution, dd
    from workloads import circuits as C
    from workloads.cutting import search_cut
    from workloads.simulate import simulate_variants
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batch_split_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
        assert p.exitcode == 0
    parts = q.get(timeout=10)
    assert not set(parts[0]) & set(parts[1]) and sorted(set(parts[0]) | set(parts[1])) == [0, 1, 2]
    got = {**parts[0], **parts[1]}
    cuts = [search_cut(C.brickwall(10, 4, 11), 7, 2, restarts=4), search_cut(C.bv(12, 9), 5, 5, restarts=4),
            search_cut(C.aqft(10, 2, max_dist=2), 5, 4, restarts=4)]
    for i, c in enumerate(cuts):
        A = [attribution.attribute(simulate_variants(s), s.w, s.in_local, s.out_local, s.in_edge, s.out_edge)
             for s in c.subcircuits]
        ref = dd.run(A, [s.out_qubit for s in c.subcircuits], [s.edges for s in c.subcircuits], c.K, c.circuit.n,
                     4, 6, 2, strategy="bfs")
        assert got[i] == [(sorted(r["zoom"].items()), float(r["bins"].sum())) for r in ref]
