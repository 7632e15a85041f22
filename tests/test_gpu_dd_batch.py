"""GPU parity of the persistent DD batch (several circuits' Algorithm 1 in
one cooperative launch) against the level-by-level run and the FP64 oracle."""
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


def _cuts():
    from workloads import circuits as C
    from workloads.cutting import search_cut
    # (cut, M, T): three shapes of different depth and job counts
    return [(search_cut(C.brickwall(10, 4, 11), 7, 2, restarts=4), 4, 3),
            (search_cut(C.aqft(12, 2, max_dist=2), 5, 4, restarts=4), 4, 2),
            (search_cut(C.bv(14, 9), 5, 5, restarts=4), 5, 1)]


def _same_records(cq, got, ref, bins, ref_bins):
    import torch
    assert len(got) == len(ref)
    for J, Rj in zip(got, ref):
        assert (J.level, J.depth, J.parent, J.parent_bin, J.n_active) == \
            (Rj.level, Rj.depth, Rj.parent, Rj.parent_bin, Rj.n_active)
        assert J.zoom() == Rj.zoom()
        assert list(J.top_idx) == list(Rj.top_idx)
        assert list(J.top_val) == list(Rj.top_val)
        nb = 1 << J.n_active
        b = bins[J.bins_offset:J.bins_offset + nb]
        # same merge slices and the same fmaf chain over k per bin: identical bins
        assert torch.equal(b, ref_bins[Rj.bins_offset:Rj.bins_offset + nb])
        # the float64 totals add float partials of 4 (persistent tile) or 8 bins
        # (level-by-level tile), each rounded by at most 3 * 2^-24 of its size,
        # in atomic order: they agree within that bound on both sides
        mass = float(b.double().abs().sum())
        assert abs(J.bin_sum - Rj.bin_sum) <= 6 * 2.0 ** -24 * mass + 1e-12


def _reference(cq, subs, At, n, M, R, T, options=None):
    import torch
    jobs, n_jobs, bins = cq.cutqc_dd_run_async(subs, At, n, M, R, T, options=options)
    torch.cuda.synchronize()
    return cq.dd_jobs_from_device(jobs, n_jobs), bins


@pytest.mark.parametrize("options", [None, {"topk_chunk": 256}, {"ctas": 7}, {"merge_ctas": 64, "topk_chunk": 512},
                                     {"ctas_per_sm": 2}, {"ctas_per_sm": 4}, {"ctas": 3, "ctas_per_sm": 3},
                                     {"narrow_max_n": -1}, {"narrow_max_n": 64}],
                         ids=["default", "chunk256", "ctas7", "merge64", "per_sm2", "per_sm4", "ctas3",
                              "tiles64x64", "narrow64"])
def test_batch_matches_level_by_level_and_oracle(cq, options):
    """Three circuits in one persistent launch: every run's records, bins and
    selections equal those of its own level-by-level run (same merge slicing),
    and its bins match the FP64 oracle, whatever the grid and chunk sizes."""
    import torch
    from oracle import dd
    R = 6
    runs, refs, oracle = [], [], []
    for cut, M, T in _cuts():
        subs, A, At = _setup(cut)
        n = cut.circuit.n
        mc = (options or {}).get("merge_ctas", 0)
        refs.append(_reference(cq, subs, At, n, M, R, T, options={"merge_ctas": mc} if mc else None))
        runs.append(cq.dd_batch_run(subs, At, n, M, R, T, max_jobs=64))
        oracle.append(dd.run(A, [s.out_qubit for s in subs], [s.edges for s in subs], cut.K, n, M, R, T,
                             strategy="bfs"))
    batch = cq.cutqc_dd_batch_create(runs, options)
    info = batch.info()
    assert info["ops"] > 0 and info["phases"] > 0 and info["ctas"] >= 1
    if options and options.get("ctas"):
        assert info["ctas"] == options["ctas"]
    batch.launch()
    torch.cuda.synchronize()
    assert cq.cutqc_device_status() == 0
    for r, (ref_jobs, ref_bins), rj in zip(runs, refs, oracle):
        got = cq.dd_jobs_from_device(r["jobs"], r["n_jobs"])
        _same_records(cq, got, ref_jobs, r["bins"], ref_bins)
        assert len(got) == len(rj)
        for J, o in zip(got, rj):
            assert list(J.active[:J.n_active]) == o["active"]
            assert J.zoom() == o["zoom"]
            b = r["bins"][J.bins_offset:J.bins_offset + (1 << J.n_active)].cpu().numpy().astype(np.float64)
            assert np.abs(b - o["bins"]).max() <= 1e-6
            assert 0.5 * float(np.abs(b - o["bins"]).sum()) <= 1e-6       # total variation per job
            assert abs(J.bin_sum - o["bins"].sum()) <= 1e-6


@pytest.mark.parametrize("topk_chunk", [256, 2048])
def test_batch_wide_selection(cq, topk_chunk):
    """T = 6 (each chunk's list wider than 4) on two circuits: records and
    bins equal the level-by-level run's."""
    import torch
    runs, refs = [], []
    for cut, M, _ in _cuts()[:2]:
        subs, A, At = _setup(cut)
        n = cut.circuit.n
        refs.append(_reference(cq, subs, At, n, M, 4, 6))
        runs.append(cq.dd_batch_run(subs, At, n, M, 4, 6, max_jobs=64))
    batch = cq.cutqc_dd_batch_create(runs, {"topk_chunk": topk_chunk})
    batch.launch()
    torch.cuda.synchronize()
    for r, (ref_jobs, ref_bins) in zip(runs, refs):
        _same_records(cq, cq.dd_jobs_from_device(r["jobs"], r["n_jobs"]), ref_jobs, r["bins"], ref_bins)
    assert cq.cutqc_device_status() == 0


def test_batch_in_cuda_graph_replays(cq):
    """The launch captures in a CUDA graph (one memset, one cooperative
    kernel); replays after clearing the outputs give the same records."""
    import torch
    R = 6
    runs, refs = [], []
    for cut, M, T in _cuts():
        subs, A, At = _setup(cut)
        n = cut.circuit.n
        refs.append(_reference(cq, subs, At, n, M, R, T))
        runs.append(cq.dd_batch_run(subs, At, n, M, R, T, max_jobs=64))
    batch = cq.cutqc_dd_batch_create(runs)
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        batch.launch(stream)
    for _ in range(2):
        for r in runs:
            r["jobs"].zero_()
            r["bins"].zero_()
            r["n_jobs"].zero_()
        g.replay()
        torch.cuda.synchronize()
        for r, (ref_jobs, ref_bins) in zip(runs, refs):
            _same_records(cq, cq.dd_jobs_from_device(r["jobs"], r["n_jobs"]), ref_jobs, r["bins"], ref_bins)
    assert cq.cutqc_device_status() == 0


def test_batch_single_level_and_no_selection(cq):
    """Edge cases: one level (R = 1: no next-level records) and T = 0 (no
    selection at all), beside a normal run in the same launch."""
    import torch
    cut, M, T = _cuts()[0]
    subs, A, At = _setup(cut)
    n = cut.circuit.n
    cases = [(M, 1, T), (M, 6, 0), (n, 3, 2)]      # M = n: one level holding every qubit
    runs, refs = [], []
    for m, R, t in cases:
        refs.append(_reference(cq, subs, At, n, m, R, t))
        runs.append(cq.dd_batch_run(subs, At, n, m, R, t, max_jobs=64))
    batch = cq.cutqc_dd_batch_create(runs)
    batch.launch()
    torch.cuda.synchronize()
    for r, (ref_jobs, ref_bins) in zip(runs, refs):
        got = cq.dd_jobs_from_device(r["jobs"], r["n_jobs"])
        assert len(got) == 1
        _same_records(cq, got, ref_jobs, r["bins"], ref_bins)
    assert cq.cutqc_device_status() == 0


def test_batch_three_dd_circuits_full_size(cq):
    """The bench's DD configuration at full size (40-, 50- and 60-qubit
    blocked brick-wall circuits, 16 active qubits per level, top 4, up to 6
    levels) in one persistent launch: each run equals its level-by-level run
    exactly (records, bins, selections), and every run matches the FP64
    oracle: the same bins expanded, and per job a total variation <= 1e-6
    and a float64 total within 1e-6 of the oracle's."""
    import torch
    from oracle import attribution, dd
    from workloads.configs import dd_batched
    M, R, T = 16, 6, 4
    runs, refs, ws = [], [], []
    for w in dd_batched():
        subs = w.subcircuits
        var = w.variants()
        att = [cq.cutqc_attribute(s, torch.from_numpy(v).cuda()) for s, v in zip(subs, var)]
        refs.append(_reference(cq, subs, att, w.n, M, R, T))
        runs.append(cq.dd_batch_run(subs, att, w.n, M, R, T, max_jobs=64))
        ws.append((w, var))
    batch = cq.cutqc_dd_batch_create(runs)
    batch.launch()
    torch.cuda.synchronize()
    assert cq.cutqc_device_status() == 0
    for r, (ref_jobs, ref_bins) in zip(runs, refs):
        _same_records(cq, cq.dd_jobs_from_device(r["jobs"], r["n_jobs"]), ref_jobs, r["bins"], ref_bins)
    assert [w.n for w, _ in ws] == [40, 50, 60]
    for run, (w, var) in zip(runs, ws):
        subs = w.subcircuits
        A = [attribution.attribute(v, s.w, s.in_local, s.out_local, s.in_edge, s.out_edge) for s, v in zip(subs, var)]
        ref = dd.run(A, [s.out_qubit for s in subs], [s.edges for s in subs], w.K, w.n, M, R, T, strategy="bfs")
        got = cq.dd_jobs_from_device(run["jobs"], run["n_jobs"])
        assert len(got) == len(ref)
        for J, rj in zip(got, ref):
            assert list(J.active[:J.n_active]) == rj["active"]
            assert J.zoom() == rj["zoom"]
            b = run["bins"][J.bins_offset:J.bins_offset + (1 << J.n_active)].cpu().numpy().astype(np.float64)
            tv = 0.5 * float(np.abs(b - rj["bins"]).sum())
            assert tv <= 1e-6, (w.n, tv)
            assert abs(J.bin_sum - float(rj["bins"].sum())) <= 1e-6, w.n


def test_tuned_batch_options_match_oracle(cq):
    """The persistent batch's autotuner (launch shapes and GEMM tile shapes)
    returns one of its candidates, every candidate it kept reproduced the
    first one's records and bins, and the batch built with the tuned options
    matches the FP64 oracle (TV <= 1e-6 per job)."""
    import torch
    from oracle import dd
    from paper_2205_05836_gb300.tune import BATCH_CANDIDATES, tune_dd_batch
    R = 6
    runs, oracle = [], []
    for cut, M, T in _cuts():
        subs, A, At = _setup(cut)
        n = cut.circuit.n
        runs.append(cq.dd_batch_run(subs, At, n, M, R, T, max_jobs=64))
        oracle.append(dd.run(A, [s.out_qubit for s in subs], [s.edges for s in subs], cut.K, n, M, R, T,
                             strategy="bfs"))
    best, trials = tune_dd_batch(runs, reps=2)
    assert best in BATCH_CANDIDATES and len(trials) == len(BATCH_CANDIDATES)
    assert all(ok for _, _, ok in trials)
    batch = cq.cutqc_dd_batch_create(runs, best)
    batch.launch()
    torch.cuda.synchronize()
    assert cq.cutqc_device_status() == 0
    for r, rj in zip(runs, oracle):
        got = cq.dd_jobs_from_device(r["jobs"], r["n_jobs"])
        assert len(got) == len(rj)
        for J, o in zip(got, rj):
            b = r["bins"][J.bins_offset:J.bins_offset + (1 << J.n_active)].cpu().numpy().astype(np.float64)
            assert 0.5 * float(np.abs(b - o["bins"]).sum()) <= 1e-6
