"""Brute-force state-vector simulation of an uncut circuit (ground truth).

The paper's Background section describes state-vector simulation as the
error-free baseline used to verify the other evaluation modes; this is that
baseline.  Written independently of the input generator's simulator: its own
gate table and index-arithmetic updates (no tensor reshapes), so that a wrong
matrix or axis convention in either one shows up as a mismatch.

Qubit q is bit q of the basis index.  Test infrastructure only.
"""
from __future__ import annotations

import cmath
import math

import numpy as np

_R2 = 1 / math.sqrt(2)


def _one_qubit(name, params):
    if name == "h":
        return [[_R2, _R2], [_R2, -_R2]]
    if name == "x":
        return [[0, 1], [1, 0]]
    if name == "s":
        return [[1, 0], [0, 1j]]
    if name == "sdg":
        return [[1, 0], [0, -1j]]
    if name == "rx":
        t = params[0] / 2
        return [[math.cos(t), -1j * math.sin(t)], [-1j * math.sin(t), math.cos(t)]]
    if name == "ry":
        t = params[0] / 2
        return [[math.cos(t), -math.sin(t)], [math.sin(t), math.cos(t)]]
    if name == "rz":
        t = params[0] / 2
        return [[cmath.exp(-1j * t), 0], [0, cmath.exp(1j * t)]]
    # square roots of X, Y and W = (X+Y)/sqrt(2): exp(i pi/4) exp(-i pi/4 P)
    if name in ("sx", "sy", "sw"):
        px = np.array([[0, 1], [1, 0]], dtype=complex)
        py = np.array([[0, -1j], [1j, 0]], dtype=complex)
        p = {"sx": px, "sy": py, "sw": (px + py) * _R2}[name]
        m = cmath.exp(1j * math.pi / 4) * (math.cos(math.pi / 4) * np.eye(2) - 1j * math.sin(math.pi / 4) * p)
        return m.tolist()
    raise KeyError(name)


def apply_1q(psi, u, q):
    idx = np.arange(psi.size)
    lo = idx[(idx >> q) & 1 == 0]
    hi = lo | (1 << q)
    a, b = psi[lo].copy(), psi[hi].copy()
    psi[lo] = u[0][0] * a + u[0][1] * b
    psi[hi] = u[1][0] * a + u[1][1] * b


def apply_2q(psi, name, q0, q1, params):
    idx = np.arange(psi.size)
    both = idx[((idx >> q0) & 1 == 1) & ((idx >> q1) & 1 == 1)]
    if name == "cz":
        psi[both] *= -1
    elif name == "cp":
        psi[both] *= cmath.exp(1j * params[0])
    elif name == "cx":   # control q0, target q1
        ctl = idx[((idx >> q0) & 1 == 1) & ((idx >> q1) & 1 == 0)]
        flip = ctl | (1 << q1)
        a = psi[ctl].copy()
        psi[ctl] = psi[flip]
        psi[flip] = a
    else:
        raise KeyError(name)


def statevector(circuit):
    """Final state U|0...0> of the circuit, complex128, length 2^n."""
    psi = np.zeros(2 ** circuit.n, dtype=complex)
    psi[0] = 1
    for name, qs, params in circuit.gates:
        if len(qs) == 1:
            apply_1q(psi, _one_qubit(name, params), qs[0])
        else:
            apply_2q(psi, name, qs[0], qs[1], params)
    return psi


def probabilities(circuit):
    """P(x) = |<x|U|0^n>|^2 (original qubit order)."""
    psi = statevector(circuit)
    return (psi.conj() * psi).real
