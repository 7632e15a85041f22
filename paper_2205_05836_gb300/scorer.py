"""Learned cut proposal: rank candidate wire cuts with the cut-scoring MLP.

The paper finds cuts with a MIP over the circuit DAG (Framework Overview,
"MIP Cut Searcher") minimising Eq. 2.  This module adds a learned front end
that the paper does not have: many seeded candidate clusterings of the DAG's
two-qubit gates are generated, the infeasible ones are dropped exactly, the
network predicts each remaining candidate's log2 reconstruction cost in one
batched launch, and only the best-ranked few are costed exactly.  A
candidate is feasible when every
subcircuit fits the width limit and its variant tensor (4^k_in * 3^k_out *
2^w entries) stays within a size budget, since every variant has to be
evaluated; among exactly costed candidates of equal cost the one with the
smallest total variant volume wins.  The local cut search stays as the
fallback: it runs when no candidate is feasible, and (``check_restarts`` >
0) beside the network's pick, whose cut is replaced by the search's when the
search's is cheaper in the same exact cost model.
"""
from __future__ import annotations

import time

import numpy as np

from workloads.cutting import Dag, build_cut, contraction_cost, search_cut
from workloads.features import LABEL_SCALE, MAX_SUB, CandidateSet, candidates


def propose_cut(circuit, w_max, net, n_candidates=4096, n_exact=8, seed=0, max_variant_log2=26, check_restarts=0):
    """Returns (Cut, info).  ``net`` is a trained ``cutqc.MLP``.  With
    ``check_restarts`` > 0 the local search (that many restarts) also runs
    and wins when its cut is cheaper (info: ``fallback`` = "search cheaper");
    info keeps the network's own pick and time beside it."""
    import torch
    t0 = time.perf_counter()
    dag = Dag(circuit)
    rng = np.random.default_rng(seed)
    assign = candidates(dag, w_max, n_candidates, rng)
    cs = CandidateSet(dag, assign, w_max)
    ok = np.nonzero(cs.feasible & (cs.variant_log2.max(1) <= max_variant_log2))[0]
    info = {"candidates": int(n_candidates), "feasible": int(len(ok))}
    if len(ok) == 0:
        lo = min(MAX_SUB - 1, max(2, -(-circuit.n // w_max)))
        cut = search_cut(circuit, w_max, lo, restarts=4, seed=seed)
        info.update(fallback=True, seconds=time.perf_counter() - t0)
        return cut, info
    feas = cs.subset(ok)
    x = torch.from_numpy(np.ascontiguousarray(feas.features())).to(net.device)
    pred = net.forward(x).cpu().numpy()
    order = np.argsort(pred, kind="stable")[:n_exact]
    top = ok[order]
    costs = [feas.exact_cost(int(j)) for j in order]
    volume = [float(np.exp2(feas.variant_log2[j][feas.used[j]]).sum()) for j in order]
    pick = min(range(len(top)), key=lambda j: (costs[j], volume[j]))
    best = int(top[pick])
    cut = build_cut(circuit, assign[best], w_max=w_max)
    info.update(fallback=False, seconds=time.perf_counter() - t0, mlp_seconds=time.perf_counter() - t0,
                predicted_log2_cost=float(pred[np.searchsorted(ok, best)] * LABEL_SCALE + circuit.n),
                exact_cost=int(costs[pick]), mlp_cost=int(costs[pick]), variant_entries=volume[pick])
    if check_restarts > 0:
        t1 = time.perf_counter()
        lo = min(MAX_SUB - 1, max(2, -(-circuit.n // w_max)))
        alt = search_cut(circuit, w_max, max(lo, len(cut.subcircuits)), restarts=check_restarts, seed=seed)
        info["search_seconds"] = time.perf_counter() - t1
        if alt is not None:
            alt_cost = contraction_cost(alt)
            info["search_cost"] = int(alt_cost)
            if alt_cost < costs[pick]:
                cut = alt
                info.update(fallback="search cheaper", exact_cost=int(alt_cost))
        info["seconds"] = time.perf_counter() - t0
    return cut, info
