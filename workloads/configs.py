"""The five benchmark workloads (seeded), built from the generators, the cut
search and the variant simulator.

Each stated cut shape is checked against what the search finds on the
generated circuit; where the stated shape cannot exist for the stated circuit
the generated workload records the real one in ``notes``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from functools import lru_cache

import numpy as np

from . import circuits as C
from .cutting import Cut, search_cut, grid_orders, build_cut
from .simulate import simulate_variants


@dataclass
class Workload:
    name: str
    cut: Cut
    notes: list = field(default_factory=list)
    _variants: list = None

    @property
    def circuit(self):
        return self.cut.circuit

    @property
    def n(self):
        return self.cut.circuit.n

    @property
    def subcircuits(self):
        return self.cut.subcircuits

    @property
    def K(self):
        return self.cut.K

    def variants(self):
        if self._variants is None:
            self._variants = [simulate_variants(s) for s in self.subcircuits]
        return self._variants


def fd_plain(seed=0):
    """8-qubit brick-wall, depth 6, two subcircuits.  Two subcircuits of width
    <= 5 do not exist for this circuit (the narrowest split is 7 + 6 wires with
    5 cuts), so the search runs with width <= 7."""
    c = C.brickwall(8, 6, seed)
    cut = search_cut(c, 7, 2, restarts=8, seed=seed)
    return Workload("fd_plain_brickwall8", cut,
                    notes=["stated: 2 cuts, two 5-qubit subcircuits (infeasible); "
                           f"built: K={cut.K}, widths {[s.w for s in cut.subcircuits]}"])


def fd_two_sub(seed=0):
    """30-qubit supremacy-family circuit (5 x 6 grid, depth 10, bridged
    couplers) cut by 4 wire cuts into two 17-qubit subcircuits."""
    c = C.supremacy_5x6_bridged(seed)
    cut = search_cut(c, 17, 2, orders=grid_orders(5, 6), restarts=8, seed=seed)
    # put the subcircuit with the measured cuts first (rows of the GEMM)
    subs = sorted(cut.subcircuits, key=lambda s: -s.k_out)
    cut.subcircuits[:] = subs
    return Workload("fd_two_sub_supremacy30", cut)


def fd_chain(seed=0):
    """32-qubit AQFT (controlled phases up to distance 4, input Ry(U[0,pi)))
    cut into 4 subcircuits of <= 11 qubits.  Distance-4 phases need 4 cuts per
    boundary, so K = 12, not the stated 6."""
    c = C.aqft(32, seed, max_dist=4)
    cut = search_cut(c, 11, 4, restarts=8, seed=seed)
    return Workload("fd_chain_aqft32", cut,
                    notes=[f"stated: 6 cuts; built: K={cut.K} (4 per boundary)"])


DD_CIRCUITS = ((40, (10, 10, 10, 10), (1, 2, 1), 1),
               (50, (13, 12, 13, 12), (2, 1, 2), 2),
               (60, (12, 12, 12, 12, 12), (1, 2, 1, 2), 3))


def dd_batched():
    """Three blocked brick-wall circuits (40, 50, 60 qubits, depth 8, seeds
    1/2/3); blocks talk through 1-2 bridge qubits that switch block halfway,
    giving 4-5 subcircuits of <= 15 qubits with 1-3 cuts each."""
    out = []
    for n, blocks, bridges, seed in DD_CIRCUITS:
        side = C.blocked_sides(blocks, bridges, 4)
        c = C.brickwall(n, 8, seed, side=side)
        cut = search_cut(c, 15, len(blocks), restarts=6, seed=seed)
        out.append(Workload(f"dd_brickwall{n}", cut))
    return out


def bv_large(n=100, seed=5, w_max=20):
    c = C.bv(n, seed)
    n_sub = -(-(n + 8) // w_max)
    cut = search_cut(c, w_max, n_sub, restarts=4, seed=seed)
    return Workload(f"bv{n}", cut)
