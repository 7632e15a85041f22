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
        assert abs(J.bin_sum - rj["bins"].sum()) <= 1e-6
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


def test_autotuned_dd_options_match_oracle(cq):
    """The autotuner returns one of its candidate launch shapes, and the run
    with it still matches the FP64 oracle."""
    from oracle import dd
    from paper_2205_05836_gb300.tune import CANDIDATES, tune_dd
    cut = _cut("brickwall")
    subs, A, At = _setup(cut)
    n, M, R, T = cut.circuit.n, 4, 6, 3
    best, trials = tune_dd(subs, At, n, M, R, T, reps=2)
    assert best in CANDIDATES and len(trials) == len(CANDIDATES) and trials[0][2]
    jobs, n_jobs, bins = cq.cutqc_dd_run_async(subs, At, n, M, R, T, options=best)
    got = cq.dd_jobs_from_device(jobs, n_jobs)
    ref = dd.run(A, [s.out_qubit for s in subs], [s.edges for s in subs], cut.K, n, M, R, T, strategy="bfs")
    assert len(got) == len(ref)
    for J, rj in zip(got, ref):
        b = bins[J.bins_offset:J.bins_offset + (1 << J.n_active)].cpu().numpy().astype(np.float64)
        assert np.abs(b - rj["bins"]).max() <= 1e-6
