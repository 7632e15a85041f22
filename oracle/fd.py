"""Full-definition reconstruction, Eq. 1, in float64.

    P = 2^-K * sum_{e in {I,X,Y,Z}^K}  kron_i  A_i[:, c_i(e)]

A_i is subcircuit i's attributed tensor ([2^o_i][4^k_i], see attribution);
c_i(e) picks the digits of the cut edges that touch subcircuit i.  The factor
2^-K is the 1/2 of the one-qubit Pauli identity, once per cut (Eq. 1 as
printed leaves it implicit).

Output orders:
* "kron": numpy's Kronecker order, subcircuit 1's output bits most
  significant: index = (((x_1) 2^o_2 + x_2) 2^o_3 + x_3) ...
* "original": index = sum_q b_q 2^q over the uncut circuit's qubits.

Test infrastructure only.
"""
from __future__ import annotations

import itertools

import numpy as np


def _column(e_digits, edges):
    """Column index of a subcircuit whose (ascending) cut edges are ``edges``."""
    c = 0
    for j, ed in enumerate(edges):
        c += int(e_digits[ed]) * 4 ** j
    return c


def reconstruct_kron(attributed, edge_lists, K):
    """Eq. 1 term by term: 4^K Kronecker products, accumulated in float64.
    ``attributed[i]`` is [2^o_i][4^k_i]; ``edge_lists[i]`` its cut edges,
    ascending."""
    total = None
    for e in itertools.product(range(4), repeat=K):
        digits = e[::-1]            # digits[edge id]; order of the loop is irrelevant
        term = np.ones(1)
        for A, edges in zip(attributed, edge_lists):
            term = np.kron(term, A[:, _column(digits, edges)])
        total = term if total is None else total + term
    return total * 0.5 ** K


def kron_to_original(p_kron, out_qubits_per_sub):
    """Permute a Kronecker-ordered vector to original qubit order.
    ``out_qubits_per_sub[i]`` lists subcircuit i's output qubits, bit 0
    first."""
    n = sum(len(q) for q in out_qubits_per_sub)
    # bit position of each Kronecker bit: subcircuit 1's bits are the most
    # significant block
    kron_bit_to_qubit = []
    for qs in reversed(out_qubits_per_sub):
        kron_bit_to_qubit.extend(qs)
    idx = np.arange(2 ** n, dtype=np.int64)
    orig = np.zeros_like(idx)
    for b, q in enumerate(kron_bit_to_qubit):
        orig |= ((idx >> b) & 1) << q
    out = np.empty_like(p_kron)
    out[orig] = p_kron
    return out


def split_kron_index(idx, outs):
    """Kronecker-order output index -> per-subcircuit output indices."""
    idx = np.asarray(idx, dtype=np.int64)
    parts = []
    shift = sum(outs)
    for o in outs:
        shift -= o
        parts.append((idx >> shift) & ((1 << o) - 1))
    return parts


def split_original_index(idx, out_qubits_per_sub):
    idx = np.asarray(idx, dtype=np.int64)
    parts = []
    for qs in out_qubits_per_sub:
        x = np.zeros_like(idx)
        for b, q in enumerate(qs):
            x |= ((idx >> q) & 1) << b
        parts.append(x)
    return parts


def entries(attributed, edge_lists, K, parts, chunk=4096):
    """P at selected outputs.  ``parts[i]`` holds, per sample, subcircuit i's
    output index.  Eq. 1 restricted to one output is a sum over the 4^K edge
    assignments of a product of one scalar per subcircuit; the sum is taken
    one cut edge at a time (the distributive law, no other rewriting; the
    edge whose elimination leaves the smallest factor goes first), which keeps
    12-cut chains tractable.  Returns float64 values."""
    n_s = len(parts[0])
    out = np.empty(n_s)
    for s0 in range(0, n_s, chunk):
        s1 = min(n_s, s0 + chunk)
        # factors: (array [S, 4, 4, ...] over its edges, list of edge ids)
        factors = []
        for A, edges, x in zip(attributed, edge_lists, parts):
            rows = A[x[s0:s1]]                               # [S, 4^k]
            k = len(edges)
            # column index c = sum_j d_j 4^j -> axes (d_{k-1}, ..., d_0)
            t = rows.reshape((s1 - s0,) + (4,) * k)
            factors.append((t, list(reversed(edges))))
        remaining = set(range(K))
        while remaining:
            # eliminate the edge whose summed-out product is smallest
            def result_edges(ed):
                touching = [f for f in factors if ed in f[1]]
                return set(x for f in touching for x in f[1]) - {ed}
            ed = min(sorted(remaining), key=lambda e: len(result_edges(e)))
            remaining.discard(ed)
            touching = [f for f in factors if ed in f[1]]
            rest = [f for f in factors if ed not in f[1]]
            if not touching:
                continue
            # product of the touching factors, then sum over edge ed
            labels = sorted(set(x for f in touching for x in f[1]))
            letters = {e: chr(ord("a") + i) for i, e in enumerate(labels)}
            spec_in = ",".join("Z" + "".join(letters[e] for e in f[1]) for f in touching)
            keep = [e for e in labels if e != ed]
            spec_out = "Z" + "".join(letters[e] for e in keep)
            t = np.einsum(spec_in + "->" + spec_out, *[f[0] for f in touching])
            factors = rest + [(t, keep)]
        val = np.ones(s1 - s0)
        for t, eds in factors:
            assert not eds
            val = val * t
        out[s0:s1] = val
    return out * 0.5 ** K


def contract_pair(A_i, edges_i, A_j, edges_j):
    """Eq. 1's sum over the cut edges that subcircuits i and j share, taken
    for every pair of their outputs at once (the distributive law applied to
    those edges only; the 2^-K factor is left to the caller).  A_i, A_j are
    attributed tensors ([2^o][4^k], column = sum_t d_t 4^t over the edges in
    ascending order).  Returns (T, open_edges): T is [2^(o_i + o_j)][4^m] in
    the same layout, row = x_i * 2^o_j + x_j (Kronecker order, i first),
    columns over the m edges that touch exactly one of the two, ascending.
    A library einsum (a tensor contraction) is the step; nothing else is
    rewritten.  Treated as one subcircuit, T gives the same entries as the
    pair it replaces."""
    shared = set(edges_i) & set(edges_j)
    open_edges = sorted(set(edges_i) ^ set(edges_j))
    labels = sorted(set(edges_i) | set(edges_j))
    letter = {e: chr(ord("a") + t) for t, e in enumerate(labels)}
    ti = A_i.reshape((A_i.shape[0],) + (4,) * len(edges_i))
    tj = A_j.reshape((A_j.shape[0],) + (4,) * len(edges_j))
    # axes after the row axis: the highest digit first (edges descending)
    spec_i = "Y" + "".join(letter[e] for e in reversed(edges_i))
    spec_j = "Z" + "".join(letter[e] for e in reversed(edges_j))
    spec_o = "YZ" + "".join(letter[e] for e in reversed(open_edges))
    assert all(letter[e] not in "YZ" for e in labels) and len(shared) + len(open_edges) == len(labels)
    t = np.einsum(f"{spec_i},{spec_j}->{spec_o}", ti, tj, optimize=True)
    return t.reshape(A_i.shape[0] * A_j.shape[0], 4 ** len(open_edges)), open_edges


def total_probability(attributed, edge_lists, K):
    """sum_x P(x) = 2^-K sum_e prod_i (sum_x A_i[x, c_i(e)]) (each Kronecker
    term sums to the product of its factors' sums)."""
    sums = [A.sum(axis=0)[None, :] for A in attributed]      # [1, 4^k]
    parts = [np.zeros(1, dtype=np.int64) for _ in attributed]
    return float(entries(sums, edge_lists, K, parts)[0])
