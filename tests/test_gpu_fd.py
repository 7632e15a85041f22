"""GPU parity of attribution and FD reconstruction (through the C ABI)
against the FP64 oracle, on seeded inputs: small cases that span several
tiles and ragged tails, both output orders, both precisions, and the full
30-qubit two-subcircuit configuration."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TV_GATE = 1e-6      # total-variation gate of the reconstruction


@pytest.fixture(scope="module")
def cq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_05836_gb300 import cutqc
    return cutqc


def _oracle_att(subs, var):
    from oracle import attribution
    return [attribution.attribute(v, s.w, s.in_local, s.out_local, s.in_edge, s.out_edge) for s, v in zip(subs, var)]


def _gpu_att(cq, subs, var, dtype=None):
    import torch
    dev = torch.device("cuda")
    outs = []
    for s, v in zip(subs, var):
        t = torch.from_numpy(v).to(dev)
        if dtype is not None:
            t = t.to(dtype)
        outs.append(cq.cutqc_attribute(s, t))
    torch.cuda.synchronize()
    return outs


def _cases():
    from workloads import circuits as C
    from workloads.cutting import search_cut
    yield "brickwall8_k5", search_cut(C.brickwall(8, 6, 0), 7, 2, restarts=4)
    yield "aqft12_3sub", search_cut(C.aqft(12, 3, max_dist=3), 7, 3, restarts=4)
    yield "supremacy3x4", search_cut(C.supremacy(3, 4, 8, 1), 8, 2, restarts=4)
    yield "brickwall12_4sub", search_cut(C.brickwall(12, 3, 2), 5, 4, restarts=6)
    yield "bv13_chain", search_cut(C.bv(13, 4), 5, 4, restarts=4)
    yield "adder12_3sub", search_cut(C.adder(12, 3), 7, 3, restarts=4)


CASES = list(_cases())


@pytest.mark.parametrize("name,cut", CASES, ids=[c[0] for c in CASES])
def test_attribution_matches_oracle(cq, name, cut):
    import torch
    from workloads.simulate import simulate_variants
    subs = cut.subcircuits
    var = [simulate_variants(s) for s in subs]
    ref = _oracle_att(subs, var)
    for dtype in (None, torch.float32):
        got = _gpu_att(cq, subs, var, dtype)
        for g, r in zip(got, ref):
            g = g.cpu().numpy().astype(np.float64)
            assert g.shape == r.shape
            scale = np.abs(r).max()
            assert np.abs(g - r).max() <= 4e-7 * scale, name


@pytest.mark.parametrize("kout,w,aligned", [(1, 3, True), (2, 4, True), (3, 9, True), (4, 12, True),
                                             (5, 11, True), (5, 5, True), (4, 6, True), (2, 9, False),
                                             (4, 12, False)])
def test_attribution_measured_cuts_only(cq, kout, w, aligned):
    """Subcircuits with measured cuts only write the attributed layout
    directly: a CTA takes the group of runs that fills whole blocks of
    columns (the run-at-a-time kernel when the output is not 16-byte
    aligned).  Random variants, measured qubits anywhere, edge ids in any
    order, 2^o rows from 1 (fewer than one CTA's 32) to several CTAs;
    every entry written (NaN-filled output) and within the float32
    rounding of a k_out-level Walsh-Hadamard transform of the oracle."""
    import torch
    from types import SimpleNamespace
    from oracle import attribution
    rng = np.random.default_rng(1000 * kout + w)
    out_local = sorted(rng.choice(w, size=kout, replace=False).tolist())
    out_edge = rng.permutation(np.arange(3, 3 + 2 * kout, 2)).tolist()
    sub = SimpleNamespace(w=w, in_local=[], out_local=out_local, in_edge=[], out_edge=out_edge,
                          out_qubit=list(range(w - kout)))
    var = rng.uniform(0.0, 1.0, size=(1, 3 ** kout, 2 ** w))
    ref = attribution.attribute(var, w, [], out_local, [], out_edge)
    n = ref.size
    # inputs rounded once, then k_out add/subtract levels over 2^k_out values <= 1
    tol = (kout + 2) * 2.0 ** (kout - 24)
    for dtype in (torch.float64, torch.float32):
        buf = torch.full((n + 4,), float("nan"), dtype=torch.float32, device="cuda")
        out = buf[0 if aligned else 1:][:n].view(ref.shape)
        assert (out.data_ptr() % 16 == 0) == aligned
        cq.cutqc_attribute(sub, torch.from_numpy(var).cuda().to(dtype), out=out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= tol, (kout, w, dtype)
        lo = 0 if aligned else 1
        assert torch.isnan(buf[:lo]).all() and torch.isnan(buf[lo + n:]).all()     # nothing outside


def test_float64_loads_round_to_nearest_even(cq):
    """The attribution's FP64 loads convert to float32 on the integer pipes
    (binary64 -> binary32 round to nearest, ties to even, written out from
    the two formats).  A subcircuit without cuts is that conversion alone:
    bit-identical to the device's own conversion (torch float64 -> float32)
    on random bit patterns of every exponent, ties and near-ties, the float32
    subnormal and overflow edges, zeros and infinities; NaN stays NaN."""
    import torch
    from types import SimpleNamespace
    rng = np.random.default_rng(7)
    n = 1 << 20
    u = rng.integers(0, 1 << 62, size=n, dtype=np.uint64) * np.uint64(4) + rng.integers(0, 4, size=n, dtype=np.uint64)
    # a quarter of the patterns at exponents around the float32 range edges
    # (binary64 biased exponents 860..930 and 1140..1160, 0, 2047), their
    # dropped 29 bits a tie, just below one, or just above one
    m = n // 4
    exps = rng.choice(np.r_[np.arange(860, 931), np.arange(1140, 1161), [0, 1, 1023, 2046, 2047]], size=m)
    frac = rng.integers(0, 1 << 52, size=m, dtype=np.uint64)
    kind = rng.integers(0, 4, size=m)
    low29 = np.uint64((1 << 29) - 1)
    frac = np.where(kind == 0, (frac & ~low29) | np.uint64(1 << 28), frac)
    frac = np.where(kind == 1, (frac & ~low29) | np.uint64((1 << 28) - 1), frac)
    frac = np.where(kind == 2, (frac & ~low29) | np.uint64((1 << 28) + 1), frac)
    sgn = rng.integers(0, 2, size=m, dtype=np.uint64) << np.uint64(63)
    u[:m] = sgn | (exps.astype(np.uint64) << np.uint64(52)) | frac
    d = u.view(np.float64)
    sub = SimpleNamespace(w=20, in_local=[], out_local=[], in_edge=[], out_edge=[], out_qubit=list(range(20)))
    t = torch.from_numpy(d).cuda()
    got = cq.cutqc_attribute(sub, t).view(-1)
    ref = t.to(torch.float32)
    torch.cuda.synchronize()
    nan = torch.isnan(ref)
    assert torch.equal(torch.isnan(got), nan)
    assert torch.equal(got.view(torch.int32)[~nan], ref.view(torch.int32)[~nan])
    assert int(nan.sum()) > 0 and int(torch.isinf(ref).sum()) > 0 and int((ref == 0).sum()) > 0


@pytest.mark.parametrize("precision", [0, 1, 2], ids=["simt", "tc", "tc_prune"])
@pytest.mark.parametrize("order", [0, 1], ids=["kron", "original"])
@pytest.mark.parametrize("name,cut", CASES, ids=[c[0] for c in CASES])
def test_fd_matches_oracle(cq, name, cut, precision, order):
    import torch
    from oracle import fd, metrics, statevector
    from workloads.simulate import simulate_variants
    subs = cut.subcircuits
    var = [simulate_variants(s) for s in subs]
    A = _oracle_att(subs, var)
    pk = fd.reconstruct_kron(A, [s.edges for s in subs], cut.K)
    ref = pk if order == 0 else fd.kron_to_original(pk, [s.out_qubit for s in subs])
    att = _gpu_att(cq, subs, var)
    total = torch.zeros(1, dtype=torch.float64, device="cuda")
    out, _ = cq.cutqc_reconstruct_fd(subs, att, order, precision, sum_out=total)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    assert metrics.tv(got, ref) <= TV_GATE, (name, metrics.tv(got, ref))
    assert abs(total.item() - 1.0) <= 1e-6
    # the device sum adds pairwise float partials of <= 32 outputs in float64:
    # each partial is <= 5 roundings deep, so |error| <= 5 * 2^-24 * sum|p|
    assert abs(total.item() - got.sum()) <= 5 * 2.0 ** -24 * np.abs(got).sum()
    assert metrics.max_abs(got, ref) <= 1e-6
    if order == 1:
        assert metrics.tv(got, statevector.probabilities(cut.circuit)) <= TV_GATE
    assert cq.cutqc_device_status() == 0


def _synthetic_chain(o0, o1, o2, k01, k12, seed):
    """Three structural subcircuits in a chain, s0 -(k01 cuts)- s1 -(k12
    cuts)- s2, with seeded random attributed tensors (Eq. 1 is bilinear in
    them, so any values exercise the contraction).  s0 measures edges
    0..k01-1, s1 initialises them and measures the next k12, s2 initialises
    those; output qubits are a seeded permutation of 0..n-1."""
    from types import SimpleNamespace
    rng = np.random.default_rng(seed)
    n = o0 + o1 + o2
    perm = [int(q) for q in rng.permutation(n)]
    e01 = list(range(k01))
    e12 = list(range(k01, k01 + k12))
    s0 = SimpleNamespace(w=o0 + k01, in_local=[], in_edge=[], out_local=list(range(o0, o0 + k01)), out_edge=e01,
                         out_qubit=perm[:o0], edges=e01, o=o0)
    s1 = SimpleNamespace(w=o1 + k12, in_local=list(range(k01)), in_edge=e01,
                         out_local=list(range(o1, o1 + k12)), out_edge=e12, out_qubit=perm[o0:o0 + o1],
                         edges=e01 + e12, o=o1)
    s2 = SimpleNamespace(w=o2, in_local=list(range(k12)), in_edge=e12, out_local=[], out_edge=[],
                         out_qubit=perm[o0 + o1:], edges=e12, o=o2)
    subs = [s0, s1, s2]
    # magnitudes spread over a few decades per row, both signs
    A = [rng.standard_normal((1 << s.o, 4 ** len(s.edges))) * 10.0 ** rng.uniform(-3, 0, size=(1 << s.o, 1))
         for s in subs]
    return subs, A


_SYN_CACHE = {}


@pytest.mark.parametrize("precision", [0, 1], ids=["simt", "tc"])
@pytest.mark.parametrize("order", [0, 1], ids=["kron", "original"])
@pytest.mark.parametrize("shape", [(5, 6, 4, 3, 3), (5, 5, 4, 3, 4), (6, 5, 3, 2, 3)],
                         ids=["open3", "open4", "open3_k2"])
def test_fd_synthetic_chain_layouts(cq, shape, order, precision):
    """Chains whose middle tensor is contracted first over its high cut
    digits, its open digits lowest (operand rows gathered through the
    shared-memory transpose, intermediate rows stored column by column),
    then joined with the first: every output against the FP64 oracle, to a
    bound relative to the sum of |terms| (the oracle on |A|)."""
    import torch
    from oracle import fd
    if shape not in _SYN_CACHE:
        o0, o1, o2, k01, k12 = shape
        subs, A = _synthetic_chain(o0, o1, o2, k01, k12, seed=sum(shape))
        # the float32 copy of A is the kernels' input: the oracle runs on it
        A = [a.astype(np.float32).astype(np.float64) for a in A]
        edges = [s.edges for s in subs]
        K = k01 + k12
        _SYN_CACHE[shape] = (subs, A, fd.reconstruct_kron(A, edges, K),
                             fd.reconstruct_kron([np.abs(a) for a in A], edges, K))
    subs, A, ref, bound = _SYN_CACHE[shape]
    if order == 1:
        ref = fd.kron_to_original(ref, [s.out_qubit for s in subs])
        bound = fd.kron_to_original(bound, [s.out_qubit for s in subs])
    att = [torch.from_numpy(a.astype(np.float32)).cuda() for a in A]
    total = torch.zeros(1, dtype=torch.float64, device="cuda")
    out, _ = cq.cutqc_reconstruct_fd(subs, att, order, precision, sum_out=total)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    err = np.abs(got - ref)
    assert (err <= 2.0 ** -16 * bound + 1e-30).all(), (err / (bound + 1e-300)).max()
    assert abs(total.item() - got.sum()) <= 2.0 ** -20 * np.abs(got).sum()
    assert cq.cutqc_device_status() == 0


def _wide_range(rng, rows, cols, decades):
    """Attributed-tensor stand-in whose entries span `decades` decades inside
    every row and 4 more across rows, both signs, 3% of rows and 5% of
    entries exactly zero."""
    a = rng.choice([-1.0, 1.0], size=(rows, cols)) * 10.0 ** rng.uniform(-decades, 0, size=(rows, cols))
    a *= 10.0 ** rng.uniform(-4, 0, size=(rows, 1))
    a[rng.random((rows, cols)) < 0.05] = 0.0
    a[rng.random(rows) < 0.03] = 0.0
    return a.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("precision", [0, 1, 2], ids=["simt", "tc", "tc_prune"])
@pytest.mark.parametrize("k,order", [(0, 0), (1, 0), (2, 0), (1, 1), (2, 1)])
def test_fd_last_step_over_few_terms(cq, k, order, precision):
    """A last step over 4^k <= 16 cut terms whose output is row-major in the
    column index runs FP32 outer products (outer.cu) under every precision:
    two synthetic subcircuits (2^9 x 2^13 outputs, k cuts, values spread over
    three decades with both signs), every output against the FP64 oracle to
    2^-20 of the sum of |terms|, in Kronecker order and in a permuted
    original qubit order (the row operand's bits reordered), and the float64
    total against the outputs' own sum."""
    import torch
    from types import SimpleNamespace
    from oracle import fd
    oA, oB = 9, 13
    rng = np.random.default_rng(300 + 10 * k + order)
    e = list(range(k))
    qa = [int(q) for q in oB + rng.permutation(oA)] if order else list(range(oB, oB + oA))
    sA = SimpleNamespace(w=oA + k, in_local=[], in_edge=[], out_local=list(range(oA, oA + k)), out_edge=e,
                         out_qubit=qa, edges=e, o=oA)
    sB = SimpleNamespace(w=oB, in_local=list(range(k)), in_edge=e, out_local=[], out_edge=[],
                         out_qubit=list(range(oB)), edges=e, o=oB)
    A = [(rng.standard_normal((1 << s.o, 4 ** k)) * 10.0 ** rng.uniform(-3, 0, size=(1 << s.o, 1)))
         .astype(np.float32).astype(np.float64) for s in (sA, sB)]
    ref = fd.reconstruct_kron(A, [e, e], k)
    bound = fd.reconstruct_kron([np.abs(a) for a in A], [e, e], k)
    if order:
        ref = fd.kron_to_original(ref, [sA.out_qubit, sB.out_qubit])
        bound = fd.kron_to_original(bound, [sA.out_qubit, sB.out_qubit])
    att = [torch.from_numpy(a.astype(np.float32)).cuda() for a in A]
    total = torch.zeros(1, dtype=torch.float64, device="cuda")
    out, _ = cq.cutqc_reconstruct_fd([sA, sB], att, order, precision, sum_out=total)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    err = np.abs(got - ref)
    assert (err <= 2.0 ** -20 * bound + 1e-30).all(), (err / (bound + 1e-300)).max()
    assert abs(total.item() - got.sum()) <= 2.0 ** -20 * np.abs(got).sum()
    assert cq.cutqc_device_status() == 0


@pytest.mark.parametrize("precision", [0, 1], ids=["simt", "tc"])
def test_fd_last_step_over_few_terms_row_range(cq, precision):
    """The few-term last step over a row range (the outer-product kernel
    covers whole outputs only; a range takes the FP32 GEMM): rows [64, 320)
    of a 2^22-output, 4-term step against the FP64 oracle's rows."""
    import torch
    from types import SimpleNamespace
    from oracle import fd
    oA, oB, k = 9, 13, 1
    rng = np.random.default_rng(401)
    e = list(range(k))
    sA = SimpleNamespace(w=oA + k, in_local=[], in_edge=[], out_local=list(range(oA, oA + k)), out_edge=e,
                         out_qubit=list(range(oB, oB + oA)), edges=e, o=oA)
    sB = SimpleNamespace(w=oB, in_local=list(range(k)), in_edge=e, out_local=[], out_edge=[],
                         out_qubit=list(range(oB)), edges=e, o=oB)
    A = [rng.standard_normal((1 << s.o, 4 ** k)).astype(np.float32).astype(np.float64) for s in (sA, sB)]
    rows, cols = cq.cutqc_fd_shape([sA, sB])
    r0, r1 = 64, 320
    assert rows >= r1 and rows * cols == 1 << (oA + oB)
    ref = fd.reconstruct_kron(A, [e, e], k)[r0 * cols:r1 * cols]
    bound = fd.reconstruct_kron([np.abs(a) for a in A], [e, e], k)[r0 * cols:r1 * cols]
    att = [torch.from_numpy(a.astype(np.float32)).cuda() for a in A]
    out, _ = cq.cutqc_reconstruct_fd([sA, sB], att, 0, precision, row_begin=r0, row_end=r1)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    assert got.shape == ref.shape
    assert (np.abs(got - ref) <= 2.0 ** -20 * bound + 1e-30).all()
    assert cq.cutqc_device_status() == 0


@pytest.mark.parametrize("decades", [8, 10])
def test_fd_wide_dynamic_range(cq, decades):
    """Split-precision robustness: two subcircuits joined by 4 cuts (one
    256-term contraction) whose attributed rows span 8-10 decades, with
    zeros and sign flips, so that small entries fall into the FP16
    subnormal range of the lo plane.  Every output is checked against the
    bound of the FP16 hi/lo split with power-of-two scales (max |x| of a row,
    or of the whole operand, scaled into [2^14, 2^15)): per product
    3 * 2^-22 |a b| + 2^-39 (|a| max|B| + |b| max|A|), plus the FP32
    accumulation (<= 26 truncations of 2^-23 of the running sum); tested
    with a 4x margin on each term:
        |P - P_exact| <= 2^-16 sum_k |a_k b_k| + 2^-37 (|A_m|_1 max|B| + |B_n|_1 max|A|)  (times 2^-K)."""
    import torch
    from types import SimpleNamespace
    rng = np.random.default_rng(100 + decades)
    o0, o1, k = 8, 9, 4
    e = list(range(k))
    s0 = SimpleNamespace(w=o0 + k, in_local=[], in_edge=[], out_local=list(range(o0, o0 + k)), out_edge=e,
                         out_qubit=list(range(o1, o1 + o0)), edges=e, o=o0)
    s1 = SimpleNamespace(w=o1, in_local=list(range(k)), in_edge=e, out_local=[], out_edge=[],
                         out_qubit=list(range(o1)), edges=e, o=o1)
    A = _wide_range(rng, 1 << o0, 4 ** k, decades)
    B = _wide_range(rng, 1 << o1, 4 ** k, decades)
    scale = 2.0 ** -k
    exact = (A @ B.T) * scale                          # [x0][x1]: Kronecker order, s0 most significant
    absum = (np.abs(A) @ np.abs(B).T) * scale
    under = (np.abs(A).sum(1)[:, None] * np.abs(B).max() + np.abs(B).sum(1)[None, :] * np.abs(A).max()) * scale
    bound = 2.0 ** -16 * absum + 2.0 ** -37 * under
    att = [torch.from_numpy(a.astype(np.float32)).cuda() for a in (A, B)]
    for prec in (cq.PREC_FP16X3_TC, cq.PREC_FP32_SIMT):
        out, _ = cq.cutqc_reconstruct_fd([s0, s1], att, cq.ORDER_KRON, prec)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64).reshape(1 << o0, 1 << o1)
        err = np.abs(got - exact)
        assert (err <= bound).all(), (prec, float((err / bound).max()))
        # zero rows of either operand give exact zeros
        assert (got[np.abs(A).sum(1) == 0] == 0).all() and (got[:, np.abs(B).sum(1) == 0] == 0).all()
    assert cq.cutqc_device_status() == 0


def test_tuned_fd_work_items_match_oracle(cq):
    """The FD autotuner (work-item size of the SM-pair contraction): every
    candidate's output is bit-identical to the default's, and the tuned
    setting's reconstruction matches the FP64 oracle (TV <= 1e-6) on a
    synthetic two-subcircuit contraction of 256 terms and 2^24 outputs."""
    import torch
    from types import SimpleNamespace
    from paper_2205_05836_gb300.tune import FD_CANDIDATES, tune_fd
    rng = np.random.default_rng(77)
    o0, o1, k = 10, 14, 4
    e = list(range(k))
    s0 = SimpleNamespace(w=o0 + k, in_local=[], in_edge=[], out_local=list(range(o0, o0 + k)), out_edge=e,
                         out_qubit=list(range(o1, o1 + o0)), edges=e, o=o0)
    s1 = SimpleNamespace(w=o1, in_local=list(range(k)), in_edge=e, out_local=[], out_edge=[],
                         out_qubit=list(range(o1)), edges=e, o=o1)
    A = [rng.standard_normal((1 << s.o, 4 ** k)).astype(np.float32) for s in (s0, s1)]
    att = [torch.from_numpy(a).cuda() for a in A]
    try:
        best, trials = tune_fd([s0, s1], att, reps=2)
        assert best in FD_CANDIDATES and len(trials) == len(FD_CANDIDATES)
        assert all(same for _, _, same in trials)
        out, _ = cq.cutqc_reconstruct_fd([s0, s1], att, cq.ORDER_KRON, cq.PREC_FP16X3_TC)
        torch.cuda.synchronize()
    finally:
        cq.cutqc_fd_set_tiles_per_item(0)
    got = out.cpu().numpy().astype(np.float64).reshape(1 << o0, 1 << o1)
    ref = (A[0].astype(np.float64) @ A[1].astype(np.float64).T) * 2.0 ** -k
    bound = (np.abs(A[0]).astype(np.float64) @ np.abs(A[1]).astype(np.float64).T) * 2.0 ** -k
    assert np.all(np.abs(got - ref) <= 2.0 ** -16 * bound)
    assert 0.5 * float(np.abs(got - ref).sum()) <= 1e-6 * float(bound.sum())
    assert cq.cutqc_device_status() == 0


def test_fd_row_split_reassembles(cq):
    """Offset/stride sharding: row ranges written separately equal the whole."""
    import torch
    from workloads import circuits as C
    from workloads.cutting import search_cut
    from workloads.simulate import simulate_variants
    cut = search_cut(C.supremacy(3, 4, 8, 1), 8, 2, restarts=4)
    subs = cut.subcircuits
    att = _gpu_att(cq, subs, [simulate_variants(s) for s in subs])
    for prec in (0, 1):
        full, _ = cq.cutqc_reconstruct_fd(subs, att, 0, prec)
        rows, cols = cq.cutqc_fd_shape(subs)
        parts = []
        for r0, r1 in ((0, 3), (3, rows)):
            p, _ = cq.cutqc_reconstruct_fd(subs, att, 0, prec, row_begin=r0, row_end=r1)
            parts.append(p)
        torch.cuda.synchronize()
        assert torch.equal(torch.cat(parts), full)


def test_fd_two_subcircuit_30q_full_size(cq):
    """30-qubit supremacy-family circuit, K=4, 2^30 outputs, in the launch
    configuration the benchmark times: full TV against the FP64 oracle
    (row blocks of A^T B), sum p, and both precisions agree."""
    import torch
    from workloads.configs import fd_two_sub
    w = fd_two_sub()
    subs = w.subcircuits
    var = w.variants()
    A64, B64 = _oracle_att(subs, var)
    att = _gpu_att(cq, subs, var)
    total = torch.zeros(1, dtype=torch.float64, device="cuda")
    out, _ = cq.cutqc_reconstruct_fd(subs, att, 0, 1, sum_out=total)
    torch.cuda.synchronize()
    assert abs(total.item() - 1.0) <= 1e-6
    M, N = A64.shape[0], B64.shape[0]
    out2 = out.view(M, N)
    tv = 0.0
    step = 512
    for r0 in range(0, M, step):
        ref = (A64[r0:r0 + step] @ B64.T) * 0.5 ** w.K
        got = out2[r0:r0 + step].cpu().numpy().astype(np.float64)
        tv += 0.5 * np.abs(got - ref).sum()
    assert tv <= TV_GATE, tv
    simt, _ = cq.cutqc_reconstruct_fd(subs, att, 0, 0)
    torch.cuda.synchronize()
    diff = (simt - out).abs().sum().item() * 0.5
    assert diff <= 2 * TV_GATE
    assert cq.cutqc_device_status() == 0


def test_fd_chain_32q_full_size(cq):
    """32-qubit AQFT chain (4 subcircuits, K = 12, 2^32 outputs = 16 GiB) on
    the tensor-core path, with and without cut-term pruning, in both output
    orders: sum p against 1, and 2^20 seeded uniformly sampled outputs (the
    sample size the 32-qubit configuration states) against the FP64 oracle
    (max error, and the total variation they estimate).  The oracle sums the
    edges inside the pairs (C0, C1) and (C2, C3) for all their outputs first
    (fd.contract_pair), then Eq. 1 over the four edges between the pairs at
    each sampled output."""
    import torch
    from oracle import fd
    from workloads.configs import fd_chain
    w = fd_chain()
    subs = w.subcircuits
    var = w.variants()
    A64 = _oracle_att(subs, var)
    att = _gpu_att(cq, subs, var)
    L, eL = fd.contract_pair(A64[0], subs[0].edges, A64[1], subs[1].edges)
    R, eR = fd.contract_pair(A64[2], subs[2].edges, A64[3], subs[3].edges)
    rng = np.random.default_rng(2024)
    idx = np.unique(rng.integers(0, 1 << w.n, size=1 << 20))
    assert len(idx) > (1 << 20) - 1000
    for order, precision in ((0, 1), (1, 1), (0, 2), (1, 2)):
        total = torch.zeros(1, dtype=torch.float64, device="cuda")
        out, _ = cq.cutqc_reconstruct_fd(subs, att, order, precision, sum_out=total)
        torch.cuda.synchronize()
        assert out.numel() == 1 << 32
        assert abs(total.item() - 1.0) <= 1e-6
        got = out[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.float64)
        del out
        torch.cuda.empty_cache()
        parts = fd.split_kron_index(idx, [s.o for s in subs]) if order == 0 else \
            fd.split_original_index(idx, [s.out_qubit for s in subs])
        pairs = [(parts[0] << subs[1].o) | parts[1], (parts[2] << subs[3].o) | parts[3]]
        ref = fd.entries([L, R], [eL, eR], w.K, pairs)
        err = np.abs(got - ref)
        assert err.max() <= 1e-6, err.max()
        tv_est = 0.5 * (1 << w.n) * err.mean()
        assert tv_est <= TV_GATE, tv_est
    assert cq.cutqc_device_status() == 0


def _single_sub_cut():
    from workloads import circuits as C
    from workloads.cutting import Dag, build_cut
    c = C.brickwall(7, 4, 21)
    return build_cut(c, [0] * Dag(c).nv)


@pytest.mark.parametrize("precision", [0, 1], ids=["simt", "tc"])
@pytest.mark.parametrize("order", [0, 1], ids=["kron", "original"])
def test_fd_single_subcircuit_no_cuts(cq, precision, order):
    """Degenerate case K = 0: the reconstruction is the subcircuit's own
    distribution (in the requested order)."""
    import torch
    from oracle import metrics, statevector
    from workloads.simulate import simulate_variants
    cut = _single_sub_cut()
    assert cut.K == 0 and len(cut.subcircuits) == 1
    subs = cut.subcircuits
    att = _gpu_att(cq, subs, [simulate_variants(s) for s in subs])
    total = torch.zeros(1, dtype=torch.float64, device="cuda")
    out, _ = cq.cutqc_reconstruct_fd(subs, att, order, precision, sum_out=total)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    ref = statevector.probabilities(cut.circuit)
    # one subcircuit: the Kronecker order is its local output order, which
    # is ascending qubit order, so both orders give the uncut distribution
    assert list(subs[0].out_qubit) == list(range(cut.circuit.n))
    assert metrics.tv(got, ref) <= TV_GATE
    assert abs(total.item() - 1.0) <= 1e-6


@pytest.mark.parametrize("precision", [0, 1], ids=["simt", "tc"])
def test_fd_empty_row_range(cq, precision):
    """An empty row range writes nothing and adds nothing to the sum."""
    import torch
    from workloads import circuits as C
    from workloads.cutting import search_cut
    from workloads.simulate import simulate_variants
    cut = search_cut(C.supremacy(3, 4, 8, 1), 8, 2, restarts=4)
    subs = cut.subcircuits
    att = _gpu_att(cq, subs, [simulate_variants(s) for s in subs])
    rows, cols = cq.cutqc_fd_shape(subs)
    sentinel = torch.full((cols,), 7.0, device="cuda")
    total = torch.zeros(1, dtype=torch.float64, device="cuda")
    out, _ = cq.cutqc_reconstruct_fd(subs, att, 0, precision, row_begin=2, row_end=2, out=sentinel, sum_out=total)
    torch.cuda.synchronize()
    assert torch.all(sentinel == 7.0) and total.item() == 0.0
    with pytest.raises(cq.CutqcError) as e:
        cq.cutqc_reconstruct_fd(subs, att, 0, precision, row_begin=3, row_end=2, out=sentinel)
    assert e.value.code == cq.EINVAL
    assert cq.cutqc_device_status() == 0


@pytest.mark.parametrize("tiny", [1e-24, 1e-3], ids=["negligible", "significant"])
def test_fd_prune_drops_only_negligible_terms(cq, tiny):
    """Cut-term pruning on a two-subcircuit contraction whose column operand
    has most cut-term columns scaled by `tiny`: with 1e-24 those terms weigh
    far below 2^-30 and are skipped, with 1e-3 they are kept.  Either way
    every output matches the FP64 oracle of the full Eq. 1 sum within the
    split-precision bound plus the pruning bound, and the pruned result
    differs from the unpruned one by at most 2^-30 in L1."""
    import torch
    from oracle import fd
    from types import SimpleNamespace
    rng = np.random.default_rng(11)
    k, oa, ob = 4, 9, 12
    edges = list(range(k))
    s0 = SimpleNamespace(w=oa + k, in_local=[], in_edge=[], out_local=list(range(oa, oa + k)), out_edge=edges,
                         out_qubit=list(range(ob, ob + oa)), edges=edges, o=oa)
    s1 = SimpleNamespace(w=ob, in_local=list(range(k)), in_edge=edges, out_local=[], out_edge=[],
                         out_qubit=list(range(ob)), edges=edges, o=ob)
    A0 = np.abs(rng.standard_normal((1 << oa, 4 ** k))) / (1 << oa)
    A1 = rng.standard_normal((1 << ob, 4 ** k)) / (1 << ob)
    keep = rng.choice(4 ** k, size=40, replace=False)
    scale = np.full(4 ** k, tiny)
    scale[keep] = 1.0
    A1 = A1 * scale
    A = [a.astype(np.float32).astype(np.float64) for a in (A0, A1)]
    ref = fd.reconstruct_kron(A, [edges, edges], k)
    bound = fd.reconstruct_kron([np.abs(a) for a in A], [edges, edges], k)
    att = [torch.from_numpy(a.astype(np.float32)).cuda() for a in A]
    full, _ = cq.cutqc_reconstruct_fd([s0, s1], att, 0, cq.PREC_FP16X3_TC)
    pruned, _ = cq.cutqc_reconstruct_fd([s0, s1], att, 0, cq.PREC_FP16X3_TC_PRUNE)
    torch.cuda.synchronize()
    f = full.cpu().numpy().astype(np.float64)
    p = pruned.cpu().numpy().astype(np.float64)
    assert (np.abs(f - ref) <= 2.0 ** -16 * bound + 1e-30).all()
    assert (np.abs(p - ref) <= 2.0 ** -16 * bound + cq.PRUNE_TOL).all()
    assert np.abs(p - f).sum() <= cq.PRUNE_TOL + 2.0 ** -16 * bound.sum()
    if tiny > 1e-10:
        assert np.array_equal(p, f)      # nothing skipped: the same kernels on the same operands
    assert cq.cutqc_device_status() == 0


def _synthetic_pair(oa, ob, k, seed):
    """Two structural subcircuits joined by k cuts (s0 measures them, s1
    initialises them) with seeded random attributed tensors."""
    from types import SimpleNamespace
    rng = np.random.default_rng(seed)
    edges = list(range(k))
    s0 = SimpleNamespace(w=oa + k, in_local=[], in_edge=[], out_local=list(range(oa, oa + k)), out_edge=edges,
                         out_qubit=list(range(ob, ob + oa)), edges=edges, o=oa)
    s1 = SimpleNamespace(w=max(ob, k), in_local=list(range(k)), in_edge=edges, out_local=[], out_edge=[],
                         out_qubit=list(range(ob)), edges=edges, o=ob)
    A0 = rng.standard_normal((1 << oa, 4 ** k)) / (1 << oa)
    A1 = rng.standard_normal((1 << ob, 4 ** k)) / (1 << ob)
    return [s0, s1], [a.astype(np.float32).astype(np.float64) for a in (A0, A1)]


def test_fd_prune_everything_negligible(cq):
    """Every cut term below the bound: all are skipped and the output is
    exactly zero, within 2^-30 in L1 of the full sum."""
    import torch
    from oracle import fd
    subs, A = _synthetic_pair(8, 9, 3, 5)
    A[1] = A[1] * 1e-30
    A = [a.astype(np.float32).astype(np.float64) for a in A]
    ref = fd.reconstruct_kron(A, [s.edges for s in subs], 3)
    att = [torch.from_numpy(a.astype(np.float32)).cuda() for a in A]
    out, _ = cq.cutqc_reconstruct_fd(subs, att, 0, cq.PREC_FP16X3_TC_PRUNE)
    got = out.cpu().numpy().astype(np.float64)
    assert not got.any()
    assert np.abs(got - ref).sum() <= cq.PRUNE_TOL
    assert cq.cutqc_device_status() == 0


def test_fd_prune_not_applied_above_1024_terms(cq):
    """A last contraction of 4^6 = 4096 terms (the K > 256 tensor-core
    kernel) is not pruned: the pruned precision gives the same bits as the
    plain split precision, and both match the FP64 oracle."""
    import torch
    from oracle import fd
    subs, A = _synthetic_pair(7, 8, 6, 9)
    ref = fd.reconstruct_kron(A, [s.edges for s in subs], 6)
    bound = fd.reconstruct_kron([np.abs(a) for a in A], [s.edges for s in subs], 6)
    att = [torch.from_numpy(a.astype(np.float32)).cuda() for a in A]
    a, _ = cq.cutqc_reconstruct_fd(subs, att, 0, cq.PREC_FP16X3_TC)
    b, _ = cq.cutqc_reconstruct_fd(subs, att, 0, cq.PREC_FP16X3_TC_PRUNE)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    got = a.cpu().numpy().astype(np.float64)
    assert (np.abs(got - ref) <= 2.0 ** -16 * bound + 1e-30).all()
    assert cq.cutqc_device_status() == 0


@pytest.mark.parametrize("precision", [0, 1], ids=["simt", "tc"])
def test_fd_eight_cuts_long_term_chain(cq, precision):
    """A last contraction over 8 cuts (4^8 = 65,536 terms, 1,024 chunks of
    the tensor-core kernel, summed with compensation): every output against
    the FP64 oracle within 2^-16 of the sum of |terms|, and the float64 total
    against the oracle's."""
    import torch
    from oracle import fd
    if "eight" not in _SYN_CACHE:
        subs, A = _synthetic_pair(6, 8, 8, 17)
        edges = [s.edges for s in subs]
        _SYN_CACHE["eight"] = (subs, A, fd.reconstruct_kron(A, edges, 8),
                               fd.reconstruct_kron([np.abs(a) for a in A], edges, 8))
    subs, A, ref, bound = _SYN_CACHE["eight"]
    att = [torch.from_numpy(a.astype(np.float32)).cuda() for a in A]
    total = torch.zeros(1, dtype=torch.float64, device="cuda")
    out, _ = cq.cutqc_reconstruct_fd(subs, att, 0, precision, sum_out=total)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    assert (np.abs(got - ref) <= 2.0 ** -16 * bound + 1e-30).all(), (np.abs(got - ref) / bound).max()
    assert abs(total.item() - ref.sum()) <= 2.0 ** -16 * bound.sum()
    assert cq.cutqc_device_status() == 0


def test_fd_from_finite_shot_variants(cq):
    """Variants sampled with a finite number of shots (the paper's
    shot-based evaluation) reconstruct on the GPU exactly as in the FP64
    oracle (TV <= 1e-6 between the two, negative entries included), and
    Eq. 3 against the exact distribution matches the oracle's value."""
    import torch
    from oracle import fd, metrics, statevector
    from workloads import circuits as C
    from workloads.cutting import search_cut
    from workloads.simulate import sample_variants, simulate_variants
    c = C.brickwall(8, 6, 0)
    cut = search_cut(c, 7, 2, restarts=4)
    subs = cut.subcircuits
    truth = statevector.probabilities(c)
    var = [sample_variants(simulate_variants(s), 10 ** 4, 21 + i) for i, s in enumerate(subs)]
    A = _oracle_att(subs, var)
    ref = fd.kron_to_original(fd.reconstruct_kron(A, [s.edges for s in subs], cut.K), [s.out_qubit for s in subs])
    att = _gpu_att(cq, subs, var)
    for precision in (0, 1):
        out, _ = cq.cutqc_reconstruct_fd(subs, att, 1, precision)
        got = out.cpu().numpy().astype(np.float64)
        assert metrics.tv(got, ref) <= TV_GATE
        # Eq. 3 divides by a_i + b_i, which finite shots bring near 0 (1.8e-5 here): loose
        assert abs(metrics.chi2(got, truth) - metrics.chi2(ref, truth)) <= 1e-2 * metrics.chi2(ref, truth)
    assert (ref < 0).any()        # finite shots: the reconstruction is not a distribution


@pytest.mark.parametrize("precision", [1, 2], ids=["tc", "tc_prune"])
def test_fd_captured_in_cuda_graph(cq, precision):
    """The reconstruction enqueues without host synchronisation (pruning
    chooses its terms on the device): captured in a CUDA graph and replayed
    twice it gives the eager call's bits and FP64 total."""
    import torch
    from workloads import circuits as C
    from workloads.cutting import search_cut
    from workloads.simulate import simulate_variants
    cut = search_cut(C.aqft(12, 3, max_dist=3), 7, 3, restarts=4)
    subs = cut.subcircuits
    att = _gpu_att(cq, subs, [simulate_variants(s) for s in subs])
    ref_total = torch.zeros(1, dtype=torch.float64, device="cuda")
    ref, _ = cq.cutqc_reconstruct_fd(subs, att, 1, precision, sum_out=ref_total)
    out = torch.empty_like(ref)
    total = torch.zeros(1, dtype=torch.float64, device="cuda")
    ws = torch.empty(max(1, cq.cutqc_reconstruct_fd_workspace_size(subs, precision)), dtype=torch.uint8,
                     device="cuda")
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        total.zero_()
        cq.cutqc_reconstruct_fd(subs, att, 1, precision, out=out, sum_out=total, ws=ws)
    for _ in range(2):
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        assert abs(total.item() - ref_total.item()) <= 1e-12
    assert cq.cutqc_device_status() == 0


def test_bounded_wait_expires_with_status(cq):
    """Failure path without a GPU fault: a device wait that nothing satisfies
    gives up after its bound (about 2 s of clock cycles), the status word
    reads CUTQC_ETIMEOUT (-4) once and is then clear, and the context still
    runs a reconstruction correctly."""
    import torch
    from workloads import circuits as C
    from workloads.cutting import search_cut
    from workloads.simulate import simulate_variants
    from oracle import fd, metrics
    assert cq.cutqc_device_status() == 0
    waited = torch.zeros(1, dtype=torch.int32, device="cuda")
    cq.cutqc_selftest_wait_timeout(waited)
    assert cq.cutqc_device_status() == -4
    assert cq.cutqc_device_status() == 0
    assert waited.item() >= 1000          # >= ~1e9 cycles: the bound, not an early exit
    cut = search_cut(C.brickwall(8, 6, 0), 7, 2, restarts=4)
    subs = cut.subcircuits
    var = [simulate_variants(s) for s in subs]
    ref = fd.reconstruct_kron(_oracle_att(subs, var), [s.edges for s in subs], cut.K)
    out, _ = cq.cutqc_reconstruct_fd(subs, _gpu_att(cq, subs, var), 0, 1)
    assert metrics.tv(out.cpu().numpy().astype(np.float64), ref) <= TV_GATE
    assert cq.cutqc_device_status() == 0


@pytest.mark.parametrize("graph", [False, True], ids=["eager", "graph"])
@pytest.mark.parametrize("precision", [0, 1], ids=["simt", "tc"])
def test_fd_waits_for_input_events(cq, precision, graph):
    """Issued before its inputs are written: the subcircuits are attributed
    on two other streams (one held back ~1 ms by a sleep kernel) into
    NaN-filled tensors, each followed by an event; the reconstruction, on a
    stream that never waited for them, gets those events
    (cutqc_fd_input_events) and must give the bits of the reconstruction of
    the same tensors written beforehand, eagerly and as a replayed graph."""
    import torch
    from workloads import circuits as C
    from workloads.cutting import search_cut
    from workloads.simulate import simulate_variants
    cut = search_cut(C.brickwall(12, 3, 2), 5, 4, restarts=6)
    subs = cut.subcircuits
    assert len(subs) >= 3
    var = [torch.from_numpy(simulate_variants(s)).cuda() for s in subs]
    ref_att = [cq.cutqc_attribute(s, v) for s, v in zip(subs, var)]
    ref, _ = cq.cutqc_reconstruct_fd(subs, ref_att, 0, precision)
    torch.cuda.synchronize()
    att = [torch.full_like(a, float("nan")) for a in ref_att]
    out = torch.full_like(ref, float("nan"))
    ws = torch.empty(max(1, cq.cutqc_reconstruct_fd_workspace_size(subs, precision)), dtype=torch.uint8,
                     device="cuda")
    att_ws = [torch.empty(max(1, cq.cutqc_attribute_workspace_size(s)), dtype=torch.uint8, device="cuda")
              for s in subs]
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()

    def step():
        cur = torch.cuda.current_stream()
        fork = torch.cuda.Event()
        fork.record(cur)
        sa.wait_event(fork)
        sb.wait_event(fork)
        ev = [torch.cuda.Event() for _ in subs]
        for i, s in enumerate(subs):
            st = sa if i % 2 == 0 else sb
            with torch.cuda.stream(st):
                if i == 0:
                    torch.cuda._sleep(2_000_000)
                cq.cutqc_attribute(s, var[i], out=att[i], ws=att_ws[i])
            ev[i].record(st)
        cq.cutqc_reconstruct_fd(subs, att, 0, precision, out=out, ws=ws, input_events=ev)
        cur.wait_stream(sa)
        cur.wait_stream(sb)

    if not graph:
        step()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    else:
        stream = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            step()
        for _ in range(2):
            for a in att:
                a.fill_(float("nan"))
            out.fill_(float("nan"))
            torch.cuda.synchronize()
            g.replay()
            torch.cuda.synchronize()
            assert torch.equal(out, ref)
    assert cq.cutqc_device_status() == 0
