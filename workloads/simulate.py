"""Exact statevector simulation of subcircuit variants (the stand-in for the
QPUs that evaluate the subcircuits).

For a subcircuit with ``k_in`` initialised cuts and ``k_out`` measured cuts the
variant tensor has layout ``[4^k_in][3^k_out][2^w]`` (float64):

* init index  = sum_j s_j 4^j over the init-cut qubits in ascending local
  order, s in {0: |0>, 1: |1>, 2: |+>, 3: |+i>};
* meas index  = sum_j m_j 3^j over the measured-cut qubits in ascending local
  order, m in {0: computational basis, 1: X basis, 2: Y basis}; the X basis is
  measured by applying H, the Y basis by S^dagger then H, before measuring;
* the last axis is the full 2^w local outcome distribution, local qubit q =
  bit q.

The paper's worked example (Circuit Cutting, example figure) has three
measurement variants and four initialisation variants per cut; this layout
is that product over cuts.  Only inputs are produced here.
"""
from __future__ import annotations

import math

import numpy as np

from .circuits import gate_matrix
from .cutting import Subcircuit

_INIT_STATES = np.array([
    [1, 0],
    [0, 1],
    [1 / math.sqrt(2), 1 / math.sqrt(2)],
    [1 / math.sqrt(2), 1j / math.sqrt(2)],
], dtype=complex)                     # rows: |0>, |1>, |+>, |+i>

_H = np.array([[1, 1], [1, -1]], dtype=complex) / math.sqrt(2)
_SDG = np.array([[1, 0], [0, -1j]], dtype=complex)
_MEAS_ROT = [np.eye(2, dtype=complex), _H, _H @ _SDG]


def _axis(w, q):
    return w - 1 - q   # C-order reshape puts the highest bit first


def apply_gate(psi, w, name, qubits, params):
    """psi: array of shape (..., 2, 2, ..., 2) with w trailing qubit axes."""
    lead = psi.ndim - w
    if len(qubits) == 1:
        U = gate_matrix(name, params)
        ax = lead + _axis(w, qubits[0])
        psi = np.moveaxis(np.tensordot(U, psi, axes=([1], [ax])), 0, ax)
        return psi
    a, b = qubits
    if name in ("cz", "cp"):
        phase = -1.0 if name == "cz" else np.exp(1j * params[0])
        idx = [slice(None)] * psi.ndim
        idx[lead + _axis(w, a)] = 1
        idx[lead + _axis(w, b)] = 1
        psi = psi.copy()
        psi[tuple(idx)] *= phase
        return psi
    U = gate_matrix(name, params).reshape(2, 2, 2, 2)  # [out_b, out_a, in_b, in_a]
    axa, axb = lead + _axis(w, a), lead + _axis(w, b)
    psi = np.tensordot(U, psi, axes=([2, 3], [axb, axa]))   # new axes 0:b 1:a
    psi = np.moveaxis(psi, [0, 1], [axb, axa])
    return psi


def simulate_variants(sub: Subcircuit, dtype=np.float64):
    w = sub.w
    kin, kout = sub.k_in, sub.k_out
    in_local, out_local = sub.in_local, sub.out_local
    # one simulation per computational-basis setting of the init-cut qubits
    psi = np.zeros((2 ** kin,) + (2,) * w, dtype=complex)
    for bsel in range(2 ** kin):
        idx = [0] * w
        for j, q in enumerate(in_local):
            idx[_axis(w, q)] = (bsel >> j) & 1
        psi[(bsel,) + tuple(idx)] = 1.0
    for name, qs, params in sub.gates:
        psi = apply_gate(psi, w, name, qs, params)
    # linear map from the 2^kin basis runs to the 4^kin init-state runs
    # psi index bsel = sum_j b_j 2^j  ->  axes (b_{kin-1}, ..., b_0)
    psi = psi.reshape((2,) * kin + (2,) * w) if kin else psi.reshape((2,) * w)
    for j in range(kin):
        ax = kin - 1 - j
        psi = np.moveaxis(np.tensordot(_INIT_STATES, psi, axes=([1], [ax])), 0, ax)
    # now leading axes (s_{kin-1}, ..., s_0), each of size 4
    # measurement rotations: add one size-3 axis per measured cut
    for j, q in enumerate(out_local):
        ax = kin + _axis(w, q) + j   # qubit axes shift right by the j meas axes added so far
        # new meas axis inserted right after the init axes, in front of earlier meas axes
        rot = np.stack(_MEAS_ROT)     # [m, out, in]
        psi = np.tensordot(rot, psi, axes=([2], [ax]))   # axes: m, out, rest...
        psi = np.moveaxis(psi, 1, ax + 1)                # put the qubit axis back
        psi = np.moveaxis(psi, 0, kin)                   # meas axis after init axes
    probs = (psi.real ** 2 + psi.imag ** 2).astype(dtype)
    return probs.reshape(4 ** kin, 3 ** kout, 2 ** w)


def sample_variants(variants, shots, seed):
    """Finite-shot stand-in for running the variants on a QPU: each variant's
    outcome distribution (the last axis, 2^w outcomes) is replaced by the
    frequencies of `shots` seeded draws from it (a multinomial sample, as a
    device's shots give: the paper's shot-based evaluation mode).  Same shape
    and dtype float64; every row sums to 1."""
    rng = np.random.default_rng(seed)
    v = np.asarray(variants, np.float64)
    flat = v.reshape(-1, v.shape[-1])
    out = np.empty_like(flat)
    for i, p in enumerate(flat):
        p = np.clip(p, 0.0, None)
        out[i] = rng.multinomial(int(shots), p / p.sum()) / float(shots)
    return out.reshape(v.shape)


def sample_distribution(p, shots, seed):
    """Frequencies of `shots` seeded draws from the distribution p (the uncut
    circuit run on a device with that many shots)."""
    rng = np.random.default_rng(seed)
    p = np.clip(np.asarray(p, np.float64), 0.0, None)
    return rng.multinomial(int(shots), p / p.sum()) / float(shots)
