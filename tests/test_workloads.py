"""Input generators: gate matrices, variant tensors, cut structure, and the
shapes of the benchmark workloads."""
import math

import numpy as np
import pytest

from workloads import circuits as C
from workloads import configs
from workloads.cutting import build_cut, contraction_plan, search_cut
from workloads.simulate import simulate_variants


@pytest.mark.parametrize("name", ["h", "x", "s", "sdg", "sx", "sy", "sw"])
def test_gates_unitary(name):
    U = C.gate_matrix(name)
    np.testing.assert_allclose(U @ U.conj().T, np.eye(2), atol=1e-14)


def test_square_roots():
    X = C.gate_matrix("x")
    Y = np.array([[0, -1j], [1j, 0]])
    W = (X + Y) / math.sqrt(2)
    for name, P in (("sx", X), ("sy", Y), ("sw", W)):
        U = C.gate_matrix(name)
        np.testing.assert_allclose(U @ U, P, atol=1e-14)


@pytest.mark.parametrize("name", ["cz", "cx", "cp"])
def test_two_qubit_unitary(name):
    U = C.gate_matrix(name, (0.4,))
    np.testing.assert_allclose(U @ U.conj().T, np.eye(4), atol=1e-14)


def test_variants_are_distributions():
    c = C.brickwall(8, 6, 0)
    cut = search_cut(c, 7, 2, restarts=4)
    for s in cut.subcircuits:
        v = simulate_variants(s)
        assert v.shape == (4 ** s.k_in, 3 ** s.k_out, 2 ** s.w)
        np.testing.assert_allclose(v.sum(axis=2), 1.0, atol=1e-12)
        assert v.min() >= 0


def test_cut_structure_invariants():
    c = C.aqft(12, 2, max_dist=3)
    cut = search_cut(c, 7, 3, restarts=4)
    assert sum(s.w for s in cut.subcircuits) == c.n + cut.K
    ins = sorted(e for s in cut.subcircuits for e in s.in_edge)
    outs = sorted(e for s in cut.subcircuits for e in s.out_edge)
    assert ins == outs == list(range(cut.K))
    qs = sorted(q for s in cut.subcircuits for q in s.out_qubit)
    assert qs == list(range(c.n))


def test_contraction_plan_meets_in_the_middle():
    # chain 0-1-2-3 with 4 edges per boundary
    e = [{0, 1, 2, 3}, {0, 1, 2, 3, 4, 5, 6, 7}, {4, 5, 6, 7, 8, 9, 10, 11}, {8, 9, 10, 11}]
    steps, _ = contraction_plan([7, 7, 7, 11], e)
    assert steps == [(0, 1), (2, 3), (4, 5)]


def test_benchmark_shapes():
    w1 = configs.fd_plain()
    assert w1.n == 8 and len(w1.subcircuits) == 2 and max(s.w for s in w1.subcircuits) <= 7
    w2 = configs.fd_two_sub()
    assert w2.n == 30 and w2.K == 4
    assert [(s.w, s.k_in, s.k_out, s.o) for s in w2.subcircuits] == [(17, 0, 4, 13), (17, 4, 0, 17)]
    w3 = configs.fd_chain()
    assert w3.n == 32 and len(w3.subcircuits) == 4 and all(s.w <= 11 for s in w3.subcircuits)
    assert sum(s.o for s in w3.subcircuits) == 32
    for w in configs.dd_batched():
        assert all(s.w <= 15 for s in w.subcircuits) and len(w.subcircuits) in (4, 5)
        assert all(1 <= s.k_in + s.k_out <= 3 for s in w.subcircuits)


def test_candidate_structure_matches_built_cut():
    """The array-derived widths, output counts, cut count and exact cost of
    candidate clusterings equal those of the subcircuits build_cut makes."""
    from workloads.cutting import Dag, build_cut, contraction_cost
    from workloads.features import CandidateSet, candidates
    rng = np.random.default_rng(1)
    checked = 0
    for _ in range(30):
        n = int(rng.integers(12, 40))
        c = C.random_family_circuit(rng, n)
        dag = Dag(c)
        w_max = int(rng.integers(max(4, n // 6), max(5, n // 2) + 1))
        A = candidates(dag, w_max, 12, rng)
        cs = CandidateSet(dag, A, w_max)
        for i in range(len(A)):
            cut = build_cut(c, A[i], w_max=w_max)
            feasible = all(s.w <= w_max for s in cut.subcircuits)
            assert feasible == bool(cs.feasible[i])
            if not feasible:
                continue
            checked += 1
            assert sorted(s.w for s in cut.subcircuits) == sorted(cs.w[i][cs.used[i]].tolist())
            assert sorted(s.o for s in cut.subcircuits) == sorted(cs.o[i][cs.used[i]].tolist())
            assert cut.K == cs.K[i]
            assert contraction_cost(cut) == cs.exact_cost(i)
    assert checked >= 50


def test_features_shape_and_permutation_invariance():
    """64 finite features; relabelling the clusters changes none of them."""
    from workloads.cutting import Dag
    from workloads.features import N_FEATURES, CandidateSet, candidates
    rng = np.random.default_rng(2)
    c = C.brickwall(30, 6, 4)
    dag = Dag(c)
    A = candidates(dag, 12, 64, rng)
    f = CandidateSet(dag, A, 12).features()
    assert f.shape == (64, N_FEATURES) and np.isfinite(f).all()
    perm = rng.permutation(7)
    f2 = CandidateSet(dag, perm[A], 12).features()
    np.testing.assert_array_equal(f, f2)


def test_exact_cut_is_optimal_by_enumeration():
    """The branch-and-bound cut search against plain enumeration of every
    assignment of the two-qubit gates to 2 or 3 clusters under the width
    limit: the same minimal Eq. 2 cost, and among the clusterings of that
    cost the same minimal contraction cost; with and without the local
    search's cut as the starting incumbent."""
    import itertools
    from workloads import circuits as C
    from workloads.cutting import Dag, build_cut, contraction_cost, eq2_cost, exact_cut, search_cut
    for c, w, ns in ((C.brickwall(6, 3, 2), 4, 2), (C.aqft(6, 1, max_dist=2), 4, 3), (C.bv(7, 2), 4, 2),
                     (C.brickwall(6, 2, 5), 3, 3), (C.supremacy(2, 3, 4, 1), 3, 3)):
        nv = Dag(c).nv
        assert ns ** nv <= 200_000
        best = None
        for cl in itertools.product(range(ns), repeat=nv):
            cut = build_cut(c, list(cl), w_max=w)
            if all(s.w <= w for s in cut.subcircuits) and len(cut.subcircuits) <= ns + len(Dag(c).free_qubits):
                key = (eq2_cost(cut), contraction_cost(cut))
                best = key if best is None else min(best, key)
        for inc in (None, search_cut(c, w, ns, restarts=2)):
            ex, full = exact_cut(c, w, ns, incumbent=inc, max_ties=100_000)
            assert full and ex is not None
            assert (eq2_cost(ex), contraction_cost(ex)) == best, (c.name, eq2_cost(ex), best)
            assert all(s.w <= w for s in ex.subcircuits)


def test_exact_cut_bound_is_admissible():
    """The lookahead bound never prunes the optimum: with and without it the
    same Eq. 2 cost on small instances.  With the local search's cut as the
    incumbent the search finishes exhaustively on 20- to 40-qubit instances
    (their optimum is then proven), never returns a costlier cut than the
    incumbent, and on a 40-qubit BV instance finds a cut with fewer cuts than
    the local search."""
    from workloads import circuits as C
    from workloads.cutting import eq2_cost, exact_cut, search_cut
    for c, w, ns in ((C.brickwall(8, 4, 1), 6, 2), (C.aqft(8, 2, max_dist=2), 5, 2), (C.supremacy(2, 4, 5, 2), 5, 2)):
        a, fa = exact_cut(c, w, ns)
        b, fb = exact_cut(c, w, ns, lookahead=False)
        assert fa and fb and eq2_cost(a) == eq2_cost(b), c.name
    for c, w, ns in ((C.brickwall(20, 4, 3), 12, 2), (C.aqft(20, 1, max_dist=2), 11, 2),
                     (C.supremacy(4, 5, 6, 1), 12, 2), (C.aqft(40, 2, max_dist=2), 21, 2), (C.bv(40, 3), 11, 4)):
        ls = search_cut(c, w, ns, restarts=4)
        ex, full = exact_cut(c, w, ns, incumbent=ls, max_nodes=300_000)
        assert full, c.name
        assert eq2_cost(ex) <= eq2_cost(ls), c.name
        if c.name.startswith("bv"):
            assert ex.K < ls.K


def test_local_search_reaches_exact_optimum_on_small_circuits():
    """The simulated-annealing cut search finds the exact minimum number of
    cuts (branch and bound) on small instances of every benchmark family."""
    from workloads import circuits as C
    from workloads.cutting import exact_cut, search_cut
    for c, w, ns in ((C.brickwall(8, 6, 0), 7, 2), (C.aqft(8, 2, max_dist=2), 5, 2), (C.adder(10, 3), 6, 3),
                     (C.bv(10, 4), 5, 3), (C.supremacy(3, 3, 6, 1), 6, 2), (C.brickwall(10, 4, 11), 7, 2)):
        ex, full = exact_cut(c, w, ns)
        assert full
        assert search_cut(c, w, ns, restarts=4).K == ex.K, c.name


def test_scorer_falls_back_to_the_search_when_it_is_cheaper():
    """The learned proposal keeps the local search as its fallback: with a
    stand-in scorer that ranks the candidates worst first (by their Eq. 2
    feature, negated) the network's pick is costlier than the search's cut,
    so the search's cut is returned; with the check off the network's pick is
    returned as it is.  No GPU: the stand-in scores on the CPU."""
    import torch
    from paper_2205_05836_gb300.scorer import propose_cut
    from workloads import circuits as C
    from workloads.cutting import contraction_cost

    class WorstFirst:
        device = "cpu"

        def forward(self, x):
            return -x[:, 6]          # column 6: log2 Eq. 2 of the candidate (scaled)
    c, w = C.aqft(30, 1, max_dist=2), 11
    mlp_cut, info0 = propose_cut(c, w, WorstFirst(), n_candidates=512, n_exact=1, seed=0)
    assert info0["fallback"] is False and contraction_cost(mlp_cut) == info0["mlp_cost"]
    cut, info = propose_cut(c, w, WorstFirst(), n_candidates=512, n_exact=1, seed=0, check_restarts=2)
    assert info["fallback"] == "search cheaper"
    assert info["search_cost"] < info["mlp_cost"]
    assert contraction_cost(cut) == info["search_cost"] == info["exact_cost"]
