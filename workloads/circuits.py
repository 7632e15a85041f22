"""Seeded synthetic circuit generators (the benchmark families of the paper's
Methodology section: BV, Adder, AQFT, Supremacy, plus the brick-wall family).

A circuit is an ordered gate list on ``n`` qubits.  Each gate is a tuple
``(name, qubits, params)``.  The gate names and their matrices are fixed here;
the post-processing never sees gates, only subcircuit outputs.

Qubit ``q`` is bit ``q`` of a basis-state index (little-endian).

This module holds no reconstruction arithmetic: it only produces inputs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ONE_QUBIT = ("h", "x", "s", "sdg", "rx", "ry", "rz", "sx", "sy", "sw")
TWO_QUBIT = ("cz", "cx", "cp")


@dataclass
class Circuit:
    n: int
    gates: list = field(default_factory=list)
    name: str = ""
    meta: dict = field(default_factory=dict)

    def add(self, name, qubits, params=()):
        qubits = tuple(int(q) for q in qubits)
        assert all(0 <= q < self.n for q in qubits), (name, qubits)
        if name in TWO_QUBIT:
            assert len(qubits) == 2 and qubits[0] != qubits[1]
        else:
            assert name in ONE_QUBIT and len(qubits) == 1, name
        self.gates.append((name, qubits, tuple(float(p) for p in params)))

    def two_qubit_gates(self):
        return [g for g in self.gates if len(g[1]) == 2]


def gate_matrix(name, params=()):
    """Unitary of a gate.  Two-qubit matrices act on (first, second) qubit with
    the first qubit as the LOW bit of the 4-dim index."""
    c = complex
    if name == "h":
        return np.array([[1, 1], [1, -1]], dtype=complex) / math.sqrt(2)
    if name == "x":
        return np.array([[0, 1], [1, 0]], dtype=complex)
    if name == "s":
        return np.array([[1, 0], [0, 1j]], dtype=complex)
    if name == "sdg":
        return np.array([[1, 0], [0, -1j]], dtype=complex)
    if name in ("rx", "ry", "rz"):
        t = params[0] / 2
        co, si = math.cos(t), math.sin(t)
        if name == "rx":
            return np.array([[co, -1j * si], [-1j * si, co]], dtype=complex)
        if name == "ry":
            return np.array([[co, -si], [si, co]], dtype=complex)
        return np.array([[c(math.cos(-t), math.sin(-t)), 0], [0, c(math.cos(t), math.sin(t))]], dtype=complex)
    if name == "sx":  # sqrt(X)
        return 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]], dtype=complex)
    if name == "sy":  # sqrt(Y)
        return 0.5 * np.array([[1 + 1j, -1 - 1j], [1 + 1j, 1 + 1j]], dtype=complex)
    if name == "sw":  # sqrt(W), W = (X + Y)/sqrt(2)
        w = (np.array([[0, 1], [1, 0]]) + np.array([[0, -1j], [1j, 0]])) / math.sqrt(2)
        # sqrt of a Pauli-like involution P: (1+i)/2 * I + (1-i)/2 * P
        return (1 + 1j) / 2 * np.eye(2) + (1 - 1j) / 2 * w
    if name == "cz":
        return np.diag([1, 1, 1, -1]).astype(complex)
    if name == "cp":
        return np.diag([1, 1, 1, np.exp(1j * params[0])]).astype(complex)
    if name == "cx":  # control = first (low bit), target = second (high bit)
        m = np.zeros((4, 4), dtype=complex)
        for i in range(4):
            ctl, tgt = i & 1, (i >> 1) & 1
            j = ctl | ((tgt ^ ctl) << 1)
            m[j, i] = 1
        return m
    raise KeyError(name)


# --------------------------------------------------------------------------
# generators
# --------------------------------------------------------------------------

def brickwall(n, depth, seed, side=None):
    """Brick-wall circuit: each layer applies Rx, Ry, Rz with angles drawn from
    U[0, 2pi) on every qubit, then CZ on pairs (0,1),(2,3),... for even layers
    and (1,2),(3,4),... for odd layers.

    ``side(q, layer)``, if given, assigns each qubit to a block at each layer;
    a CZ is kept only when both qubits are in the same block at that layer
    (see ``blocked_sides``)."""
    rng = np.random.default_rng(seed)
    c = Circuit(n, name=f"brickwall_n{n}_d{depth}_s{seed}" + ("_blocked" if side else ""))
    for layer in range(depth):
        for q in range(n):
            for g in ("rx", "ry", "rz"):
                c.add(g, (q,), (rng.uniform(0, 2 * math.pi),))
        for a in range(layer % 2, n - 1, 2):
            if side is None or side(a, layer) == side(a + 1, layer):
                c.add("cz", (a, a + 1))
    c.meta.update(kind="brickwall", depth=depth, seed=seed, blocked=side is not None)
    return c


def blocked_sides(block_sizes, bridges, switch_layer):
    """Partition rule for a 1-D register split into contiguous blocks.  The
    first ``bridges[j]`` qubits of block j+1 are bridge qubits: they belong to
    block j before ``switch_layer`` and to block j+1 from then on.  Every other
    qubit stays in its own block.  Returns side(q, layer)."""
    starts = np.cumsum([0] + list(block_sizes))
    home = {}
    for j, (a, b) in enumerate(zip(starts[:-1], starts[1:])):
        for q in range(int(a), int(b)):
            home[q] = j
    bridge_of = {}
    for j, m in enumerate(bridges):
        for q in range(int(starts[j + 1]), int(starts[j + 1]) + m):
            bridge_of[q] = j
    def side(q, layer):
        if q in bridge_of and layer < switch_layer:
            return bridge_of[q]
        return home[q]
    return side


# Eight coupler patterns of a rows x cols grid.  Pattern p activates horizontal
# couplers (r,c)-(r,c+1) (p < 4) or vertical couplers (r,c)-(r+1,c) (p >= 4)
# whose (row parity, column parity) equals the pattern's offset.
SUPREMACY_PATTERN_ORDER = (
    ("h", 0, 0), ("h", 1, 1), ("v", 0, 0), ("v", 1, 1),
    ("h", 0, 1), ("h", 1, 0), ("v", 0, 1), ("v", 1, 0),
)


def supremacy_pattern(rows, cols, p):
    kind, rpar, cpar = SUPREMACY_PATTERN_ORDER[p % 8]
    pairs = []
    for r in range(rows):
        for col in range(cols):
            if r % 2 != rpar:
                continue
            if kind == "h":
                if col % 2 == cpar and col + 1 < cols:
                    pairs.append((r * cols + col, r * cols + col + 1))
            else:
                if col % 2 == cpar and r + 1 < rows:
                    pairs.append((r * cols + col, (r + 1) * cols + col))
    return pairs


def supremacy(rows, cols, depth, seed, side=None):
    """2-D random circuit of the supremacy family on a rows x cols grid
    (qubit r*cols + c).  An H layer first; then ``depth`` cycles.  Cycle t
    applies, on every qubit that took part in a CZ in cycle t-1, one gate drawn
    uniformly from {sqrt(X), sqrt(Y), sqrt(W)} minus the last one applied to it,
    then the CZs of coupler pattern t mod 8.

    ``side(q, cycle)``, if given, keeps a CZ only when both qubits are on the
    same side at that cycle (see ``bridged_grid_sides``)."""
    rng = np.random.default_rng(seed)
    n = rows * cols
    c = Circuit(n, name=f"supremacy_{rows}x{cols}_d{depth}_s{seed}" + ("_bridged" if side else ""))
    for q in range(n):
        c.add("h", (q,))
    last = [None] * n
    prev = set()
    choices = ("sx", "sy", "sw")
    for t in range(depth):
        for q in sorted(prev):
            opts = [g for g in choices if g != last[q]]
            g = opts[int(rng.integers(len(opts)))]
            c.add(g, (q,))
            last[q] = g
        pairs = supremacy_pattern(rows, cols, t)
        if side is not None:
            pairs = [(a, b) for a, b in pairs if side(a, t) == side(b, t)]
        cur = set()
        for a, b in pairs:
            c.add("cz", (a, b))
            cur.update((a, b))
        prev = cur
    c.meta.update(kind="supremacy", rows=rows, cols=cols, depth=depth, seed=seed,
                  bridged=side is not None)
    return c


def bridged_grid_sides(rows, cols, side_a, bridges, switch_cycle):
    """Two-sided partition rule for a grid: qubits in ``side_a`` are side 0,
    the others side 1, except the ``bridges`` qubits, which are side 0 before
    ``switch_cycle`` and side 1 from then on.  Returns side(q, cycle)."""
    side_a, bridges = set(side_a), set(bridges)
    def side(q, t):
        if q in bridges:
            return 0 if t < switch_cycle else 1
        return 0 if q in side_a else 1
    return side


def supremacy_5x6_bridged(seed, depth=10):
    """30-qubit supremacy-family circuit on a 5 x 6 grid whose couplers respect
    a 13 | 4 | 13 split.  Side A: columns 0-1 and (0,2),(2,2),(4,2); side B:
    columns 4-5 and (0,3),(1,3),(3,3); bridge qubits (1,2),(3,2),(2,3),(4,3)
    couple to side A in cycles 0-3 and to side B from cycle 4 on.  Cut on the
    four bridge wires it splits into two 17-qubit subcircuits (13 outputs + 4
    measured cuts, and 13 inputs + 4 initialised cuts).  The unrestricted 5 x 6
    depth-10 circuit has no such cut: every column boundary carries five
    active couplers."""
    rows, cols = 5, 6
    q = lambda r, c: r * cols + c
    a = [q(r, c) for r in range(rows) for c in (0, 1)] + [q(0, 2), q(2, 2), q(4, 2)]
    bridges = [q(1, 2), q(3, 2), q(2, 3), q(4, 3)]
    side = bridged_grid_sides(rows, cols, a, bridges, 4)
    return supremacy(rows, cols, depth, seed, side=side)


def aqft(n, seed, max_dist=4, input_scale=1.0):
    """Approximate QFT: an input layer of Ry(U[0, pi)) on every qubit (angles
    multiplied by ``input_scale``), then for j = 0..n-1: H on qubit j followed
    by controlled phases CP(pi / 2^d) between qubits j + d and j for
    1 <= d <= max_dist (smaller angles are dropped).  No final swaps (the
    output is in bit-reversed order)."""
    rng = np.random.default_rng(seed)
    c = Circuit(n, name=f"aqft_n{n}_s{seed}")
    for q in range(n):
        c.add("ry", (q,), (input_scale * rng.uniform(0, math.pi),))
    for j in range(n):
        c.add("h", (j,))
        for d in range(1, max_dist + 1):
            if j + d < n:
                c.add("cp", (j + d, j), (math.pi / 2 ** d,))
    c.meta.update(kind="aqft", seed=seed, max_dist=max_dist)
    return c


def bv(n, seed, hidden=None):
    """Bernstein-Vazirani circuit on n qubits: data qubits 0..n-2 and the
    ancilla n-1.  The hidden string (n-1 bits, seeded) decides which data
    qubits control a CNOT onto the ancilla.  A final H on the ancilla makes the
    output a single basis state: data qubits = hidden string, ancilla = 1."""
    rng = np.random.default_rng(seed)
    if hidden is None:
        hidden = rng.integers(0, 2, size=n - 1)
    hidden = [int(b) for b in hidden]
    anc = n - 1
    c = Circuit(n, name=f"bv_n{n}_s{seed}")
    for q in range(n - 1):
        c.add("h", (q,))
    c.add("x", (anc,))
    c.add("h", (anc,))
    for q in range(n - 1):
        if hidden[q]:
            c.add("cx", (q, anc))
    for q in range(n - 1):
        c.add("h", (q,))
    c.add("h", (anc,))
    c.meta.update(kind="bv", seed=seed, hidden=hidden)
    return c


def _toffoli(c, a, b, t):
    """Toffoli with controls a, b and target t, in the gate set here: the
    standard decomposition into 6 CNOTs, H and T / T^dagger (T = Rz(pi/4) up
    to a global phase, which no probability sees)."""
    T, Td = (math.pi / 4,), (-math.pi / 4,)
    c.add("h", (t,))
    c.add("cx", (b, t))
    c.add("rz", (t,), Td)
    c.add("cx", (a, t))
    c.add("rz", (t,), T)
    c.add("cx", (b, t))
    c.add("rz", (t,), Td)
    c.add("cx", (a, t))
    c.add("rz", (b,), T)
    c.add("rz", (t,), T)
    c.add("h", (t,))
    c.add("cx", (a, b))
    c.add("rz", (a,), T)
    c.add("rz", (b,), Td)
    c.add("cx", (a, b))


def adder(n, seed):
    """Ripple-carry adder (the paper's Adder benchmark: one ancilla, linear
    depth, two registers of the same width, so n is even): m = (n - 2) / 2
    bit registers a and b, the ancilla carry-in c0 (qubit 0) and the carry
    out z (qubit n - 1), laid out c0, b0, a0, b1, a1, ..., b_{m-1}, a_{m-1}, z.
    The carry ripples up through MAJ blocks stored in a, z takes the top
    carry, and UMA blocks ripple back down, leaving b = a + b mod 2^m and a
    restored (the majority / unmajority-and-add construction of a
    ripple-carry adder with one ancilla).  Inputs: a in uniform superposition
    (H on each a_i), b a seeded classical value, so the output is uniform
    over the 2^m values of a: (a, a + b mod 2^m, carry), c0 = 0."""
    if n < 4 or n % 2:
        raise ValueError("the adder needs an even n >= 4")
    m = (n - 2) // 2
    rng = np.random.default_rng(seed)
    bval = int(rng.integers(0, 1 << m))
    c0, z = 0, n - 1
    bq = [1 + 2 * i for i in range(m)]
    aq = [2 + 2 * i for i in range(m)]
    c = Circuit(n, name=f"adder_n{n}_s{seed}")
    for i in range(m):
        c.add("h", (aq[i],))
        if (bval >> i) & 1:
            c.add("x", (bq[i],))

    def maj(x, y, w):      # carry x, b bit y, a bit w -> w = majority
        c.add("cx", (w, y))
        c.add("cx", (w, x))
        _toffoli(c, x, y, w)

    def uma(x, y, w):      # undo maj and write the sum bit into y
        _toffoli(c, x, y, w)
        c.add("cx", (w, x))
        c.add("cx", (x, y))

    carry = [c0] + aq[:-1]
    for i in range(m):
        maj(carry[i], bq[i], aq[i])
    c.add("cx", (aq[m - 1], z))
    for i in reversed(range(m)):
        uma(carry[i], bq[i], aq[i])
    c.meta.update(kind="adder", seed=seed, m=m, b=bval, a_qubits=aq, b_qubits=bq, carry_qubit=z)
    return c


def random_family_circuit(rng, n):
    """One circuit of a random family, size n (used for the cut-scorer
    training set)."""
    kind = int(rng.integers(4))
    seed = int(rng.integers(1 << 31))
    if kind == 0:
        return brickwall(n, int(rng.integers(3, 9)), seed)
    if kind == 1:
        return aqft(n, seed, max_dist=int(rng.integers(1, 5)))
    if kind == 2:
        rows = max(2, int(round(math.sqrt(n))))
        cols = max(2, n // rows)
        return supremacy(rows, cols, int(rng.integers(4, 11)), seed)
    return bv(n, seed)
