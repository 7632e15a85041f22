"""Pins of the FP64 oracle against things other than itself: closed forms,
brute-force state-vector simulation of the uncut circuit, invariants, the
paper's worked-example counts, and hand counts.  A planted mistake in the
oracle must fail at least one of them (see the planted-mistake tests)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import attribution, dd, fd, metrics, statevector
from oracle import mlp as omlp
from workloads import circuits as C
from workloads.cutting import build_cut, search_cut, eq2_cost, Dag
from workloads.simulate import simulate_variants


def _attr(subs, variants):
    return [attribution.attribute(v, s.w, s.in_local, s.out_local, s.in_edge, s.out_edge)
            for s, v in zip(subs, variants)]


def _reconstruct(cut, order="original"):
    subs = cut.subcircuits
    A = _attr(subs, [simulate_variants(s) for s in subs])
    pk = fd.reconstruct_kron(A, [s.edges for s in subs], cut.K)
    if order == "kron":
        return pk, A
    return fd.kron_to_original(pk, [s.out_qubit for s in subs]), A


# ---------------------------------------------------------------- closed forms

def _rand_rho(rng):
    g = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
    r = g @ g.conj().T
    return r / np.trace(r)


def _rand_unitary(rng):
    q, r = np.linalg.qr(rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2)))
    return q * (np.diag(r) / abs(np.diag(r)))


H = np.array([[1, 1], [1, -1]]) / math.sqrt(2)
SDG = np.diag([1, -1j])


@pytest.mark.parametrize("seed", range(5))
def test_single_cut_pauli_identity(seed):
    """One cut between a (mixed) one-qubit state rho and a unitary V: the
    reconstruction must give <b| V rho V^+ |b>.  Variants written from the
    closed forms, not from any simulator."""
    rng = np.random.default_rng(seed)
    rho, V = _rand_rho(rng), _rand_unitary(rng)
    up = np.zeros((1, 3, 2))       # upstream: w=1, the qubit is the measured cut
    for m, R in enumerate([np.eye(2), H, H @ SDG]):
        r = R @ rho @ R.conj().T
        up[0, m] = np.real(np.diag(r))
    states = [np.array([1, 0]), np.array([0, 1]),
              np.array([1, 1]) / math.sqrt(2), np.array([1, 1j]) / math.sqrt(2)]
    down = np.zeros((4, 1, 2))     # downstream: w=1, init cut, output
    for s, st in enumerate(states):
        down[s, 0] = np.abs(V @ st) ** 2
    A_up = attribution.attribute(up, 1, [], [0], [], [0])
    A_dn = attribution.attribute(down, 1, [0], [], [0], [])
    assert A_up.shape == (1, 4) and A_dn.shape == (2, 4)
    p = fd.reconstruct_kron([A_up, A_dn], [[0], [0]], 1)
    exact = np.real(np.diag(V @ rho @ V.conj().T))
    np.testing.assert_allclose(p, exact, atol=1e-14)


def test_attribution_bases_match_pauli_traces():
    """Upstream attributed entries are Tr(rho M) for M = I, X, Y, Z."""
    rng = np.random.default_rng(7)
    rho = _rand_rho(rng)
    up = np.zeros((1, 3, 2))
    for m, R in enumerate([np.eye(2), H, H @ SDG]):
        up[0, m] = np.real(np.diag(R @ rho @ R.conj().T))
    A = attribution.attribute(up, 1, [], [0], [], [0])[0]
    paulis = [np.eye(2), np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.diag([1, -1])]
    np.testing.assert_allclose(A, [np.real(np.trace(rho @ P)) for P in paulis], atol=1e-14)


def test_qft_of_zero_is_uniform():
    """AQFT on |0...0> (input angles 0) outputs |+>^n: uniform 2^-n."""
    c = C.aqft(9, 0, max_dist=3, input_scale=0.0)
    cut = search_cut(c, 6, 2, restarts=4)
    assert cut is not None and cut.K > 0
    p, _ = _reconstruct(cut)
    np.testing.assert_allclose(p, np.full(2 ** 9, 2.0 ** -9), atol=1e-14)


@pytest.mark.parametrize("n,seed", [(9, 1), (12, 4)])
def test_bv_single_bitstring(n, seed):
    c = C.bv(n, seed, hidden=[1, 0, 1, 1, 0, 1, 1, 0, 1, 1, 0][: n - 1])
    cut = search_cut(c, 4, 4, restarts=4)
    assert cut is not None and cut.K >= 1
    p, _ = _reconstruct(cut)
    hidden = c.meta["hidden"]
    x = sum(b << q for q, b in enumerate(hidden)) | (1 << (n - 1))
    assert np.argmax(p) == x
    assert abs(p[x] - 1) < 1e-12
    assert metrics.norm_error(p) < 1e-12


# ------------------------------------------------------------ worked example

def _worked_example_circuit():
    c = C.Circuit(5)
    for q in range(5):
        c.add("h", (q,))
    c.add("cz", (0, 1))
    c.add("rx", (2,), (0.3,))
    c.add("cz", (1, 2))       # first CZ on q2
    c.add("ry", (2,), (1.1,))
    c.add("cz", (2, 3))       # second CZ on q2
    c.add("cz", (3, 4))
    c.add("rz", (4,), (0.7,))
    return c


def test_worked_example_counts(repo_root):
    g = json.load(open(os.path.join(repo_root, "tests", "golden", "worked_example.json")))
    c = _worked_example_circuit()
    # cluster: gates on q0..q2 up to the first CZ on q2 -> 0, the rest -> 1
    cut = build_cut(c, [0, 0, 1, 1])
    assert cut.K == g["cuts"]
    assert [s.w for s in cut.subcircuits] == g["subcircuit_widths"]
    var = [simulate_variants(s) for s in cut.subcircuits]
    assert [v.shape[0] * v.shape[1] for v in var] == g["variants"]
    assert 4 ** cut.K == g["kronecker_terms"]
    p, _ = _reconstruct(cut)
    np.testing.assert_allclose(p, statevector.probabilities(c), atol=1e-14)


# ------------------------------------------------------------ brute force

def _cases():
    yield "brickwall8", C.brickwall(8, 6, 0), 7, 2
    yield "brickwall9_3sub", C.brickwall(9, 4, 3), 5, 3
    yield "supremacy3x3", C.supremacy(3, 3, 6, 2), 6, 2
    yield "aqft10_3sub", C.aqft(10, 5, max_dist=2), 6, 3
    yield "aqft10_4sub", C.aqft(10, 6, max_dist=2), 5, 4


@pytest.mark.parametrize("name,c,w,nsub", list(_cases()))
def test_fd_matches_bruteforce(name, c, w, nsub):
    cut = search_cut(c, w, nsub, restarts=4)
    assert cut is not None and cut.K > 0
    assert sum(s.w for s in cut.subcircuits) == c.n + cut.K
    assert sum(s.o for s in cut.subcircuits) == c.n
    p, A = _reconstruct(cut)
    exact = statevector.probabilities(c)
    assert metrics.max_abs(p, exact) < 1e-12
    assert metrics.tv(p, exact) < 1e-12
    # analytic total and sampled entries agree with the full vector
    edges = [s.edges for s in cut.subcircuits]
    assert abs(fd.total_probability(A, edges, cut.K) - 1) < 1e-12
    idx = np.random.default_rng(0).integers(0, 2 ** c.n, size=64)
    parts = fd.split_original_index(idx, [s.out_qubit for s in cut.subcircuits])
    np.testing.assert_allclose(fd.entries(A, edges, cut.K, parts), exact[idx], atol=1e-13)


@pytest.mark.parametrize("name,c,w,nsub", [x for x in _cases() if x[3] >= 3])
def test_contract_pair_entries_match_bruteforce(name, c, w, nsub):
    """Summing a pair's shared edges for all their outputs first
    (fd.contract_pair), then evaluating Eq. 1 over the remaining edges at
    every output, gives the uncut circuit's exact distribution; every pair of
    subcircuits is tried, sharing edges or not."""
    cut = search_cut(c, w, nsub, restarts=4)
    subs = cut.subcircuits
    A = _attr(subs, [simulate_variants(s) for s in subs])
    exact = statevector.probabilities(c)
    idx = np.arange(2 ** c.n)
    kparts = fd.split_kron_index(idx, [s.o for s in subs])
    # perm[original index] = Kronecker index
    perm = fd.kron_to_original(idx.astype(np.float64), [s.out_qubit for s in subs]).astype(np.int64)
    exact_kron = np.empty_like(exact)
    exact_kron[perm] = exact            # exact distribution in Kronecker order
    for i in range(len(subs)):
        j = i + 1
        if j >= len(subs):
            break
        T, open_e = fd.contract_pair(A[i], subs[i].edges, A[j], subs[j].edges)
        assert T.shape == (2 ** (subs[i].o + subs[j].o), 4 ** len(open_e))
        tensors = A[:i] + [T] + A[j + 1:]
        edges = [s.edges for s in subs[:i]] + [open_e] + [s.edges for s in subs[j + 1:]]
        parts = kparts[:i] + [(kparts[i] << subs[j].o) | kparts[j]] + kparts[j + 1:]
        got = fd.entries(tensors, edges, cut.K, parts)
        assert np.abs(got - exact_kron).max() < 1e-12, (name, i)


def test_contract_pair_hand_values():
    """Two one-output subcircuits sharing one edge and keeping one open edge
    each: T[x_i x_j, (d_a, d_b)] = sum_s A_i[x_i, d_a + 4 s] A_j[x_j, s + 4 d_b]
    written out for every entry (edges: i = {0 open, 1 shared}, j = {1 shared,
    2 open})."""
    rng = np.random.default_rng(3)
    Ai = rng.normal(size=(2, 16))
    Aj = rng.normal(size=(2, 16))
    T, open_e = fd.contract_pair(Ai, [0, 1], Aj, [1, 2])
    assert open_e == [0, 2] and T.shape == (4, 16)
    for xi in range(2):
        for xj in range(2):
            for da in range(4):
                for db in range(4):
                    want = sum(Ai[xi, da + 4 * sh] * Aj[xj, sh + 4 * db] for sh in range(4))
                    assert abs(T[xi * 2 + xj, da + 4 * db] - want) < 1e-12


def test_kron_order_is_numpy_kron():
    """'kron' order = np.kron of the per-subcircuit vectors for one term."""
    a0 = np.array([1.0, 2.0])[:, None]
    a1 = np.array([3.0, 5.0, 7.0, 11.0])[:, None]
    np.testing.assert_allclose(fd.reconstruct_kron([a0, a1], [[], []], 0), np.kron(a0[:, 0], a1[:, 0]))
    # original order: subcircuit 0 owns qubit 2, subcircuit 1 owns qubits 0, 1
    p = fd.kron_to_original(np.kron(a0[:, 0], a1[:, 0]), [[2], [0, 1]])
    for x in range(8):
        b0, b12 = (x >> 2) & 1, x & 3
        assert p[x] == a0[b0, 0] * a1[b12, 0]


# ------------------------------------------------------------ DD invariants

def _dd_setup(c, w, nsub):
    cut = search_cut(c, w, nsub, restarts=4)
    subs = cut.subcircuits
    A = _attr(subs, [simulate_variants(s) for s in subs])
    return cut, A, [s.out_qubit for s in subs], [s.edges for s in subs]


def _marginal(p, n, active, zoom):
    x = np.arange(2 ** n)
    keep = np.ones(2 ** n, bool)
    for q, b in zoom.items():
        keep &= ((x >> q) & 1) == b
    a = np.zeros(2 ** n, np.int64)
    for j, q in enumerate(active):
        a |= ((x >> q) & 1) << j
    out = np.zeros(2 ** len(active))
    np.add.at(out, a[keep], p[keep])
    return out


@pytest.mark.parametrize("strategy", ["dfs", "bfs"])
def test_dd_bins_are_marginals_and_children_sum_to_parent(strategy):
    c = C.brickwall(10, 4, 11)
    cut, A, oq, edges = _dd_setup(c, 7, 2)
    exact = statevector.probabilities(c)
    jobs = dd.run(A, oq, edges, cut.K, c.n, M=3, R=5, T=2, strategy=strategy)
    assert len(jobs) >= 3
    assert abs(jobs[0]["bins"].sum() - 1) < 1e-12
    for j in jobs:
        np.testing.assert_allclose(j["bins"], _marginal(exact, c.n, j["active"], j["zoom"]), atol=1e-13)
    # each child job's bins sum to the parent bin it zooms into
    for j in jobs[1:]:
        parent = [p for p in jobs if set(p["zoom"]) < set(j["zoom"])
                  and all(j["zoom"][q] == v for q, v in p["zoom"].items())
                  and set(j["zoom"]) == set(p["zoom"]) | set(p["active"])]
        assert parent
        par = parent[-1]
        b = sum(j["zoom"][q] << k for k, q in enumerate(par["active"]))
        assert abs(j["bins"].sum() - par["bins"][b]) < 1e-13


def test_dd_dfs_finds_bv_string():
    n = 14
    c = C.bv(n, 9)
    cut, A, oq, edges = _dd_setup(c, 5, 5)
    M = 4
    jobs = dd.run(A, oq, edges, cut.K, n, M=M, R=math.ceil(n / M), T=2, strategy="dfs")
    last = jobs[-1]
    assert len(last["zoom"]) + len(last["active"]) == n
    b = int(np.argmax(last["bins"]))
    bits = dict(last["zoom"])
    for j, q in enumerate(last["active"]):
        bits[q] = (b >> j) & 1
    hidden = c.meta["hidden"]
    assert [bits[q] for q in range(n - 1)] == hidden and bits[n - 1] == 1
    assert abs(last["bins"][b] - 1) < 1e-12
    assert len(jobs) == math.ceil(n / M)


# ------------------------------------------------------------ metrics, costs

def test_metrics_hand_values():
    a = np.array([0.5, 0.5, 0.0])
    b = np.array([0.25, 0.5, 0.25])
    assert metrics.tv(a, b) == pytest.approx(0.25)
    # Eq. 3: (0.25^2 / 0.75) + 0 + (0.25^2 / 0.25)
    assert metrics.chi2(a, b) == pytest.approx(0.0625 / 0.75 + 0.25)
    assert metrics.norm_error(b) == 0.0


def test_eq2_hand_counts():
    c = _worked_example_circuit()
    cut = build_cut(c, [0, 0, 1, 1])
    # two subcircuits with 2 and 3 outputs, one cut: 4 * 2^2 * 2^3
    assert eq2_cost(cut) == 4 * 2 ** 5
    # three clusters: CZ(0,1) | CZ(1,2), CZ(2,3) | CZ(3,4): cuts on q1 and q3,
    # outputs 1 (q0), 2 (q1, q2), 2 (q3, q4): 4^2 * (2^(1+2) + 2^(1+2+2)) = 640
    cut3 = build_cut(c, [0, 1, 1, 2])
    assert cut3.K == 2 and [s.o for s in cut3.subcircuits] == [1, 2, 2]
    assert eq2_cost(cut3) == 640


def test_dag_counts():
    c = _worked_example_circuit()
    d = Dag(c)
    assert d.nv == 4
    assert [len(w) for w in d.wire] == [1, 2, 2, 2, 1]


# ------------------------------------------------------------ MLP reference

def test_mlp_gradients_finite_difference():
    rng = np.random.default_rng(3)
    sizes = (6, 5, 4, 1)
    params = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        params += [rng.normal(size=(a, b)) * 0.5, rng.normal(size=b) * 0.1]
    x = rng.normal(size=(7, 6))
    t = rng.normal(size=7)
    g = omlp.backward(params, x, t)
    eps = 1e-6
    for pi, p in enumerate(params):
        flat = p.reshape(-1)
        for k in range(0, flat.size, max(1, flat.size // 5)):
            old = flat[k]
            flat[k] = old + eps
            lp = omlp.loss(params, x, t)
            flat[k] = old - eps
            lm = omlp.loss(params, x, t)
            flat[k] = old
            assert abs((lp - lm) / (2 * eps) - g[pi].reshape(-1)[k]) < 1e-6


def test_adam_first_step_is_signed_lr():
    p = [np.array([1.0, -2.0])]
    g = [np.array([0.3, -4.0])]
    z = [np.zeros(2)]
    p2, _, _ = omlp.adam_step(p, g, z, z, 1, lr=0.1)
    np.testing.assert_allclose(p2[0], [0.9, -1.9], atol=1e-7)


def test_adam_three_steps_against_hand_derivation():
    """Three Adam steps (Kingma & Ba, bias-corrected; beta1 = 0.9, beta2 =
    0.999, eps = 1e-8, lr = 0.1), worked out by hand with exact fractions, so
    that beta2, the bias corrections and the moments carried between steps
    all matter.

    Element 0, gradients 1, -2, 0 from p = 1:
      step 1: m = 1/10,  v = 1/1000;          m^ = 1,       v^ = 1
              p = 1 - 0.1 / (1 + 1e-8)                      = 0.90000000099999999
      step 2: m = 0.09 - 0.2 = -11/100, v = 0.000999 + 0.004 = 4999/10^6
              m^ = (-11/100) / (1 - 0.81) = -11/19
              v^ = (4999/10^6) / (1 - 0.998001) = 4999/1999
              p -= 0.1 m^ / (sqrt(v^) + 1e-8)               = 0.93661035347207509
      step 3: m = 0.9 (-11/100) = -99/1000, v = 0.999 * 4999/10^6 = 4994001/10^9
              m^ = (-99/1000) / (1 - 0.729) = -99/271
              v^ = (4994001/10^9) / (1 - 0.997002999) = 4994001/2997001
              p -= 0.1 m^ / (sqrt(v^) + 1e-8)               = 0.96491026200093055
    (the zero gradient of step 3 still moves p: only the moments' history does.)
    Element 1, constant gradient 0.5 from p = -2: m^ = 0.5 and v^ = 0.25 at
    every step, so each step subtracts 0.1 * 0.5 / (0.5 + 1e-8)."""
    p = [np.array([1.0, -2.0])]
    m = [np.zeros(2)]
    v = [np.zeros(2)]
    for step, g in enumerate(([1.0, 0.5], [-2.0, 0.5], [0.0, 0.5]), start=1):
        p, m, v = omlp.adam_step(p, [np.array(g)], m, v, step, lr=0.1)
    np.testing.assert_allclose(m[0], [-99 / 1000, 0.5 * (1 - 0.9 ** 3)], rtol=1e-14)
    np.testing.assert_allclose(v[0], [4994001 / 10 ** 9, 0.25 * (1 - 0.999 ** 3)], rtol=1e-14)
    np.testing.assert_allclose(p[0], [0.96491026200093055, -2.299999994000000120], rtol=1e-14)


def test_adam_wrong_beta2_or_history_is_caught():
    """Planted mistakes in the update fail the three-step pin above: a
    different beta2, or moments restarted every step."""
    want = 0.96491026200093055

    def run(beta2=0.999, carry=True):
        p, m, v = [np.array([1.0])], [np.zeros(1)], [np.zeros(1)]
        for step, g in enumerate((1.0, -2.0, 0.0), start=1):
            p, m2, v2 = omlp.adam_step(p, [np.array([g])], m, v, step, lr=0.1, beta2=beta2)
            if carry:
                m, v = m2, v2
        return float(p[0][0])
    assert abs(run() - want) < 1e-12
    assert abs(run(beta2=0.99) - want) > 1e-5
    assert abs(run(carry=False) - want) > 1e-4


# ------------------------------------------------------------ planted mistakes

def test_planted_sign_error_is_caught(monkeypatch):
    """Flip the sign of the Y basis on the init side only: brute force fails."""
    bad = attribution.INIT_MAP.copy()
    bad[2] *= -1
    monkeypatch.setattr(attribution, "INIT_MAP", bad)
    c = C.brickwall(8, 6, 0)
    cut = search_cut(c, 7, 2, restarts=4)
    p, _ = _reconstruct(cut)
    assert metrics.max_abs(p, statevector.probabilities(c)) > 1e-4


def test_planted_swapped_meas_bases_is_caught(monkeypatch):
    """Use the Y-basis run for X and vice versa on the measured side."""
    bad = list(attribution.MEAS_MAP)
    bad[1], bad[2] = (2, 1.0, -1.0), (1, 1.0, -1.0)
    monkeypatch.setattr(attribution, "MEAS_MAP", tuple(bad))
    c = C.brickwall(8, 6, 0)
    cut = search_cut(c, 7, 2, restarts=4)
    p, _ = _reconstruct(cut)
    assert metrics.max_abs(p, statevector.probabilities(c)) > 1e-4


def test_planted_missing_scale_is_caught():
    c = C.brickwall(8, 6, 0)
    cut = search_cut(c, 7, 2, restarts=4)
    p, _ = _reconstruct(cut)
    assert metrics.norm_error(p * 2) > 0.5   # a dropped 1/2 per cut breaks sum p = 1


def test_planted_order_swap_is_caught():
    c = C.brickwall(8, 6, 0)
    cut = search_cut(c, 7, 2, restarts=4)
    pk, _ = _reconstruct(cut, order="kron")
    subs = cut.subcircuits
    wrong = fd.kron_to_original(pk, [s.out_qubit for s in reversed(subs)])
    assert metrics.max_abs(wrong, statevector.probabilities(c)) > 1e-4


def test_adder_closed_form():
    """The Adder benchmark (ripple-carry, one ancilla): register a in uniform
    superposition, b a seeded constant; the exact output is uniform over a of
    the basis state (a, a + b mod 2^m, carry), ancilla 0 -- the statevector
    simulator reproduces it to rounding."""
    from oracle import statevector
    from workloads import circuits as C
    for n, seed in ((6, 1), (10, 3)):
        c = C.adder(n, seed)
        m, b = c.meta["m"], c.meta["b"]
        ref = np.zeros(1 << n)
        for a in range(1 << m):
            s = a + b
            idx = (((s >> m) & 1) << c.meta["carry_qubit"])
            for i in range(m):
                idx |= ((a >> i) & 1) << c.meta["a_qubits"][i]
                idx |= ((s >> i) & 1) << c.meta["b_qubits"][i]
            ref[idx] = 2.0 ** -m
        assert np.abs(statevector.probabilities(c) - ref).max() < 1e-12
    with pytest.raises(ValueError):
        C.adder(7, 0)


def test_fd_oracle_on_cut_adder_matches_statevector():
    """A 12-qubit adder cut into a chain of three subcircuits (K = 4): the
    oracle's Eq. 1 reconstruction equals the uncut circuit's distribution."""
    from oracle import attribution, fd, metrics, statevector
    from workloads import circuits as C
    from workloads.cutting import search_cut
    from workloads.simulate import simulate_variants
    c = C.adder(12, 3)
    cut = search_cut(c, 7, 3, restarts=4)
    subs = cut.subcircuits
    assert len(subs) == 3 and cut.K >= 2
    A = [attribution.attribute(simulate_variants(s), s.w, s.in_local, s.out_local, s.in_edge, s.out_edge)
         for s in subs]
    p = fd.kron_to_original(fd.reconstruct_kron(A, [s.edges for s in subs], cut.K), [s.out_qubit for s in subs])
    assert metrics.tv(p, statevector.probabilities(c)) < 1e-12


def test_sampled_variants_are_distributions():
    """Finite-shot variants: every row sums to 1, seeded draws repeat, and
    their frequencies approach the exact outcome probabilities (within six
    binomial standard deviations at 10^6 shots)."""
    from workloads import circuits as C
    from workloads.cutting import search_cut
    from workloads.simulate import sample_variants, simulate_variants
    cut = search_cut(C.brickwall(8, 6, 0), 7, 2, restarts=4)
    v = simulate_variants(cut.subcircuits[0])
    s1 = sample_variants(v, 10 ** 6, 5)
    assert s1.shape == v.shape
    assert np.allclose(s1.sum(-1), 1.0)
    assert np.array_equal(s1, sample_variants(v, 10 ** 6, 5))
    assert not np.array_equal(s1, sample_variants(v, 10 ** 6, 6))
    sd = np.sqrt(v * (1 - v) / 1e6)
    assert (np.abs(s1 - v) <= 6 * sd + 1e-12).all()


def test_chi2_falls_with_shots():
    """Eq. 3 between the reconstruction from finite-shot variants (negative
    entries clipped, renormalised) and the exact distribution shrinks as the
    shots grow (about as 1 / shots; checked loosely: two decades of shots give
    at least a 20-fold drop), TV about as 1 / sqrt(shots), and chi^2 is 0 for
    exact variants."""
    from oracle import attribution, fd, metrics, statevector
    from workloads import circuits as C
    from workloads.cutting import search_cut
    from workloads.simulate import sample_variants, simulate_variants
    c = C.brickwall(8, 6, 0)
    cut = search_cut(c, 7, 2, restarts=4)
    subs = cut.subcircuits
    truth = statevector.probabilities(c)
    var = [simulate_variants(s) for s in subs]

    def rec(vs):
        A = [attribution.attribute(v, s.w, s.in_local, s.out_local, s.in_edge, s.out_edge) for s, v in zip(subs, vs)]
        return fd.kron_to_original(fd.reconstruct_kron(A, [s.edges for s in subs], cut.K), [s.out_qubit for s in subs])
    assert metrics.chi2(rec(var), truth) < 1e-20
    # Eq. 3 by hand: (0.5-1)^2/1.5 + (0.5-0)^2/0.5 = 1/6 + 1/2; the 0/0 term is left out
    assert abs(metrics.chi2([0.5, 0.5, 0.0], [1.0, 0.0, 0.0]) - (1 / 6 + 1 / 2)) < 1e-15
    recs = [rec([sample_variants(v, S, 11 + i) for i, v in enumerate(var)]) for S in (10 ** 3, 10 ** 5)]
    x = [metrics.chi2(metrics.clip_renormalise(r), truth) for r in recs]
    assert x[1] < x[0] / 20, x
    t = [metrics.tv(r, truth) for r in recs]
    assert t[1] < t[0] / 4, t       # TV falls about as 1 / sqrt(shots)
    # the clipped, renormalised reconstruction is a distribution
    q = metrics.clip_renormalise(recs[0])
    assert (q >= 0).all() and abs(q.sum() - 1) < 1e-12
