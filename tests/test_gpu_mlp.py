"""Cut-scoring MLP on the GPU: forward, gradients and Adam against the FP64
oracle (BF16-rounded weights, as the kernels read them), and what the trained
network gains when it picks among candidate cuts."""
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


def _bf16(a):
    import torch
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _oracle_params(cq, flat):
    """FP64 parameters as the kernels use them: weights rounded to BF16,
    biases FP32."""
    W1, b1, W2, b2, W3, b3 = cq.split_params(np.asarray(flat, dtype=np.float32))
    return [_bf16(W1), b1.astype(np.float64), _bf16(W2), b2.astype(np.float64), _bf16(W3), b3.astype(np.float64)]


def _random_net(cq, seed):
    rng = np.random.default_rng(seed)
    flat = cq.init_params(seed)
    flat += (rng.standard_normal(flat.size) * 0.05).astype(np.float32)   # non-zero biases
    return flat


@pytest.mark.parametrize("batch", [1, 63, 300, 1024])
def test_forward_matches_oracle(cq, batch):
    import torch
    from oracle import mlp as omlp
    flat = _random_net(cq, batch)
    net = cq.MLP(flat)
    x = np.random.default_rng(7).standard_normal((batch, 64)).astype(np.float32)
    y = net.forward(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    ref, _ = omlp.forward(_oracle_params(cq, flat), x.astype(np.float64))
    assert np.abs(y - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("batch", [5, 300, 1024])
def test_gradients_match_oracle(cq, batch):
    import torch
    from oracle import mlp as omlp
    flat = _random_net(cq, 100 + batch)
    net = cq.MLP(flat)
    rng = np.random.default_rng(batch)
    x = rng.standard_normal((batch, 64)).astype(np.float32)
    t = rng.standard_normal(batch).astype(np.float32)
    grad, loss = net.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    g = cq.split_params(grad.cpu().numpy().astype(np.float64))
    P = _oracle_params(cq, flat)
    ref = omlp.backward(P, x.astype(np.float64), t.astype(np.float64))
    names = ["W1", "b1", "W2", "b2", "W3", "b3"]
    for name, a, r in zip(names, g, ref):
        r = r.reshape(a.shape)
        assert np.abs(a - r).max() <= 1e-4 * np.abs(r).max(), name
    assert abs(loss.item() - omlp.loss(P, x.astype(np.float64), t.astype(np.float64))) <= 1e-5 * loss.item()


def test_adam_matches_oracle(cq):
    import torch
    from oracle import mlp as omlp
    flat = _random_net(cq, 5)
    net = cq.MLP(flat)
    rng = np.random.default_rng(11)
    p = [flat.astype(np.float64)]
    m = [np.zeros(flat.size)]
    v = [np.zeros(flat.size)]
    m_abs = np.zeros(flat.size)          # the first moment of |g|: its terms' magnitude
    B1, B2 = float(np.float32(0.9)), float(np.float32(0.999))
    for step in (1, 2, 3):
        g = (rng.standard_normal(flat.size) * 10.0 ** rng.integers(-4, 0, flat.size)).astype(np.float32)
        net.grad.copy_(torch.from_numpy(g))
        net.adam(step, 1e-3)
        # the kernel is given beta1 = 0.9f and beta2 = 0.999f: the oracle
        # takes the same float32 values (beta2 in float32 is 0.999 + 1.3e-8,
        # which moves 1 - beta2, and so v, by 1.3e-5 relatively)
        p, m, v = omlp.adam_step(p, [g.astype(np.float64)], m, v, step, 1e-3, beta1=B1, beta2=B2)
        m_abs = B1 * m_abs + (1 - B1) * np.abs(g.astype(np.float64))
    got = net.p.cpu().numpy().astype(np.float64)
    assert np.abs(got - p[0]).max() <= 1e-6 * max(1.0, np.abs(p[0]).max())
    assert torch.equal(net.pb.cpu(), net.p.cpu().to(torch.bfloat16))
    # the moments after three steps (their history and beta2 matter here,
    # which the parameters' float32 rounding could hide): float32 relative
    gm = net.m.cpu().numpy().astype(np.float64)
    gv = net.v.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(gm - m[0]) <= 1e-6 * m_abs)
    assert np.all(np.abs(gv - v[0]) <= 1e-6 * np.abs(v[0]) + 1e-30)
    # and the total update of three steps, per parameter, against the
    # oracle's: float32 rounding of p (~6e-8 relative) against steps of ~1e-3
    upd_ref = p[0] - flat.astype(np.float64)
    upd = got - flat.astype(np.float64)
    assert np.abs(upd - upd_ref).max() <= 1e-3 * np.abs(upd_ref).max()


@pytest.fixture(scope="module")
def trained(cq):
    """A network trained on the GPU by the library's kernels: 1500 seeded
    random circuits of 20-60 qubits, up to 4 feasible candidates each."""
    import torch
    from workloads.features import training_set
    x, t, _ = training_set(1500, 4, seed=0)
    net = cq.MLP(seed=0)
    X, T = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    l0 = float(((net.forward(X) - T) ** 2).mean())
    net.fit(X, T, steps=3000, batch=512, lr=1e-3, seed=0)
    return net, l0


def test_training_gain_over_unscored_pick(cq, trained):
    """Labels: exact contraction cost of each candidate cut.  On held-out
    circuits the trained network's pick among feasible candidates costs far
    less than a pick without a scorer (uniform over the candidates) and less
    than a pick by the Eq. 2 objective."""
    import torch
    from workloads.features import LABEL_SCALE, training_set
    net, l0 = trained
    xv, tv, gv = training_set(300, 32, seed=99)     # ~200 held-out circuits with >= 4 candidates
    pv = net.forward(torch.from_numpy(xv).cuda()).cpu().numpy()
    mse = float(((pv - tv) ** 2).mean())
    assert mse < 0.1 * float(tv.var()) and mse < 0.01 * l0, (mse, float(tv.var()), l0)
    reg_mlp, reg_rand, reg_eq2 = [], [], []
    for g in np.unique(gv):
        s = gv == g
        if s.sum() < 4:
            continue
        cost = tv[s] * LABEL_SCALE          # log2 cost, up to a per-circuit constant
        best = cost.min()
        reg_mlp.append(cost[pv[s].argmin()] - best)
        reg_rand.append(cost.mean() - best)
        reg_eq2.append(cost[xv[s][:, 6].argmin()] - best)
    assert len(reg_mlp) >= 150
    assert np.mean(reg_mlp) < 0.25 * np.mean(reg_rand), (np.mean(reg_mlp), np.mean(reg_rand))
    assert np.mean(reg_mlp) < np.mean(reg_eq2), (np.mean(reg_mlp), np.mean(reg_eq2))
    assert cq.cutqc_device_status() == 0


def test_bv100_proposed_cut_reaches_hidden_string(cq, trained):
    """100-qubit Bernstein-Vazirani circuit, subcircuits of <= 20 qubits: the
    network proposes the cut (checked against the width limit and against
    the local search's cost), and dynamic definition on that cut (16 active
    qubits per recursion, depth first) ends on the hidden string with
    probability 1."""
    import math
    import torch
    from paper_2205_05836_gb300.scorer import propose_cut
    from workloads import circuits as C
    from workloads.cutting import contraction_cost, search_cut
    from workloads.simulate import simulate_variants
    net, _ = trained
    n, w_max = 100, 20
    c = C.bv(n, 5)
    cut, info = propose_cut(c, w_max, net, n_candidates=4096, n_exact=8, seed=0)
    assert not info["fallback"] and all(s.w <= w_max for s in cut.subcircuits)
    assert all(4 ** s.k_in * 3 ** s.k_out * 2 ** s.w <= 2 ** 26 for s in cut.subcircuits)
    assert info["exact_cost"] == contraction_cost(cut)
    searched = search_cut(c, w_max, -(-(n + 8) // w_max), restarts=4, seed=5)
    assert contraction_cost(cut) <= 4 * contraction_cost(searched)
    subs = cut.subcircuits
    att = [cq.cutqc_attribute(s, torch.from_numpy(simulate_variants(s)).cuda()) for s in subs]
    M = 16
    jobs, bins = cq.cutqc_dd_run(subs, att, n, M, math.ceil(n / M), 1, 0)
    last = jobs[-1]
    assert last.depth * M + last.n_active == n
    b = bins[last.bins_offset:last.bins_offset + (1 << last.n_active)].cpu().numpy()
    top = int(np.argmax(b))
    bits = last.zoom()
    for j in range(last.n_active):
        bits[last.active[j]] = (top >> j) & 1
    assert [bits[q] for q in range(n - 1)] == c.meta["hidden"] and bits[n - 1] == 1
    assert abs(b[top] - 1) < 1e-5
    assert cq.cutqc_device_status() == 0
