"""Attribution: subcircuit variant outputs -> edge-basis tensors (FP64).

Circuit Cutting section: each cut runs over the Pauli bases {I, X, Y, Z}, and
the subcircuits are initialised and measured differently for each basis
(Eq. 1 sums the products of the resulting vectors).  The paper defers the
physics to its citation; the coefficients below follow from the one-qubit
identity

    rho = 1/2 * sum_{M in {I,X,Y,Z}} Tr(rho M) M,

with I = |0><0| + |1><1|, Z = |0><0| - |1><1|, X = 2|+><+| - I,
Y = 2|+i><+i| - I.

Upstream side of a cut (the measured qubit), outcome m in {0,1}:
    I: sum_m p_Z(m)            Z: sum_m (-1)^m p_Z(m)
    X: sum_m (-1)^m p_X(m)     Y: sum_m (-1)^m p_Y(m)
where p_B is the run measuring the cut qubit in basis B (computational basis
for I and Z, which share one run: three measurement variants per cut).

Downstream side (the initialised qubit), p_s the run starting in state s:
    I: p_0 + p_1               Z: p_0 - p_1
    X: 2 p_+ - p_0 - p_1       Y: 2 p_+i - p_0 - p_1
(four initialisation variants per cut).

The factor 1/2 per cut is applied in the reconstruction, not here.

Input layout (variants): [4^k_in][3^k_out][2^w], init digits s in
{0:|0>, 1:|1>, 2:|+>, 3:|+i>} over init cuts in ascending local order
(digit j has weight 4^j), measurement digits m in {0: computational, 1: X,
2: Y} over measured cuts in ascending local order (weight 3^j), local qubit q
= bit q of the last index.

Output layout (attributed): [2^o][4^k], k = k_in + k_out, row index = output
bits (output qubits in ascending local order, first = bit 0), column index
c = sum_j d_j 4^j over the subcircuit's cut edges in ascending edge id, with
d in {0:I, 1:X, 2:Y, 3:Z}.

Test infrastructure only.
"""
from __future__ import annotations

import numpy as np

# downstream side: rows I, X, Y, Z; columns the init runs |0>, |1>, |+>, |+i>
INIT_MAP = np.array([[1, 1, 0, 0],
                     [-1, -1, 2, 0],
                     [-1, -1, 0, 2],
                     [1, -1, 0, 0]], dtype=np.float64)
# upstream side: for I, X, Y, Z the measurement run used (0: computational,
# 1: X basis, 2: Y basis) and the weight of outcome 0 and outcome 1
MEAS_MAP = ((0, 1.0, 1.0),
            (1, 1.0, -1.0),
            (2, 1.0, -1.0),
            (0, 1.0, -1.0))


def attribute(variants, w, in_local, out_local, in_edge, out_edge):
    """Return the attributed tensor (float64, [2^o][4^k]) of one subcircuit."""
    v = np.asarray(variants, dtype=np.float64)
    kin, kout = len(in_local), len(out_local)
    assert v.shape == (4 ** kin, 3 ** kout, 2 ** w), v.shape
    # axes: init digits (s_{kin-1} .. s_0), meas digits (m_{kout-1} .. m_0),
    # local qubits (q_{w-1} .. q_0)
    t = v.reshape((4,) * kin + (3,) * kout + (2,) * w)
    names = [("s", j) for j in reversed(range(kin))] + \
            [("m", j) for j in reversed(range(kout))] + \
            [("q", q) for q in reversed(range(w))]

    # downstream (init) side: state axis -> basis axis
    for j in range(kin):
        ax = names.index(("s", j))
        runs = [np.take(t, i, axis=ax) for i in range(4)]     # |0>, |1>, |+>, |+i>
        basis = [sum(INIT_MAP[b, i] * runs[i] for i in range(4)) for b in range(4)]
        t = np.stack(basis, axis=ax)
        names[ax] = ("e", in_edge[j])

    # upstream (measured) side: (measurement-basis axis, outcome axis) -> basis axis
    for j in range(kout):
        q = out_local[j]
        axm = names.index(("m", j))
        axq = names.index(("q", q))
        def run(basis_idx, outcome):
            return np.take(np.take(t, outcome, axis=axq), basis_idx,
                           axis=axm if axm < axq else axm - 1)
        basis = [w0 * run(r, 0) + w1 * run(r, 1) for (r, w0, w1) in MEAS_MAP]
        # both axes removed; put the new basis axis where the meas axis was
        new_names = [nm for nm in names if nm not in (("m", j), ("q", q))]
        pos = min(axm, axq)
        t = np.stack(basis, axis=pos)
        new_names.insert(pos, ("e", out_edge[j]))
        names = new_names

    # final order: output qubits (descending local -> row index bits), then
    # edges descending id (-> column index with the smallest id as digit 0)
    outs = sorted((nm for nm in names if nm[0] == "q"), key=lambda x: -x[1])
    edges = sorted((nm for nm in names if nm[0] == "e"), key=lambda x: -x[1])
    perm = [names.index(nm) for nm in outs + edges]
    t = np.transpose(t, perm)
    o, k = len(outs), len(edges)
    return np.ascontiguousarray(t.reshape(2 ** o, 4 ** k))
