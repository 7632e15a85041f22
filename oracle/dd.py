"""Dynamic-definition query, Algorithm 1, in float64.

Each recursion labels at most M qubits active, fixes ("zooms") the qubits
resolved by earlier recursions to the states of the bin being expanded, and
merges the rest.  The 2^#active bins are the reconstructed probabilities
summed over the merged qubits.  Because the attribution is linear and acts
only on cut qubits, the merge is applied to each subcircuit's attributed
tensor (summing rows over its merged output bits, keeping rows whose zoomed
bits match), and Eq. 1 is then evaluated on the merged tensors.

Readings where Algorithm 1 is silent or overloaded:
* active qubits: the M lowest-index qubits not yet resolved;
* Algorithm 1 uses R both for the recursion count and for the number of bins
  kept; here R = recursions and T = bins kept (appended per recursion and
  kept after truncation);
* a bin is appended only if it still has merged qubits;
* order: larger probability first, ties to the lower bin index; negative
  reconstructed values are kept as they are;
* strategy "dfs" is Algorithm 1 as written (pop the largest bin of L each
  recursion); strategy "bfs" expands, level by level, the T largest bins of
  the previous level (all jobs of a level are independent).

Bin index: bit j = state of the j-th active qubit in ascending qubit order.

Test infrastructure only.
"""
from __future__ import annotations

import numpy as np

from .fd import reconstruct_kron, kron_to_original, entries, split_original_index


def merge(A, out_qubits, active, zoom):
    """Merged tensor of one subcircuit: rows over its active output qubits
    (ascending), summed over its merged output qubits, restricted to rows
    whose zoomed qubits carry the zoomed bits."""
    o = len(out_qubits)
    act = [b for b, q in enumerate(out_qubits) if q in active]
    rows = np.arange(2 ** o)
    keep = np.ones(2 ** o, dtype=bool)
    for b, q in enumerate(out_qubits):
        if q in zoom:
            keep &= ((rows >> b) & 1) == zoom[q]
    a_idx = np.zeros(2 ** o, dtype=np.int64)
    for j, b in enumerate(act):
        a_idx |= ((rows >> b) & 1) << j
    out = np.zeros((2 ** len(act), A.shape[1]))
    np.add.at(out, a_idx[keep], A[keep])
    return out


def reconstruct_bins(attributed, out_qubits, edge_lists, K, active, zoom):
    """2^#active bins (index bit j = j-th active qubit ascending)."""
    active = sorted(active)
    merged = [merge(A, oq, set(active), zoom) for A, oq in zip(attributed, out_qubits)]
    act_per_sub = [[q for q in oq if q in active] for oq in out_qubits]
    if 4 ** K <= 4096:
        pk = reconstruct_kron(merged, edge_lists, K)
        # kron order -> active order: relabel qubits by their rank in `active`
        rank = {q: j for j, q in enumerate(active)}
        return kron_to_original(pk, [[rank[q] for q in a] for a in act_per_sub])
    rank = {q: j for j, q in enumerate(active)}
    idx = np.arange(2 ** len(active), dtype=np.int64)
    parts = split_original_index(idx, [[rank[q] for q in a] for a in act_per_sub])
    return entries(merged, edge_lists, K, parts)


def _top(bins, T, has_merged):
    if not has_merged:
        return []
    order = np.lexsort((np.arange(bins.size), -bins))
    return [int(i) for i in order[:T]]


def run(attributed, out_qubits, edge_lists, K, n, M, R, T, strategy="dfs"):
    """Algorithm 1.  Returns a list of jobs, each a dict with keys
    ``active`` (sorted qubits), ``zoom`` (qubit -> bit), ``bins``
    (float64 array) and ``top`` (bin indices appended to L)."""
    jobs = []

    def make_job(zoom):
        unresolved = [q for q in range(n) if q not in zoom]
        active = unresolved[:M]
        bins = reconstruct_bins(attributed, out_qubits, edge_lists, K, active, zoom)
        has_merged = len(unresolved) > len(active)
        job = dict(active=active, zoom=dict(zoom), bins=bins,
                   top=_top(bins, T, has_merged))
        jobs.append(job)
        return job

    def child_zoom(job, b):
        z = dict(job["zoom"])
        for j, q in enumerate(job["active"]):
            z[q] = (b >> j) & 1
        return z

    if strategy == "dfs":
        L = []
        zoom = {}
        for r in range(R):
            job = make_job(zoom)
            for b in job["top"]:
                L.append((float(job["bins"][b]), child_zoom(job, b)))
            # sort (largest first; ties keep insertion order) and truncate to T
            L.sort(key=lambda x: -x[0])
            L = L[:T]
            if not L:
                break
            _, zoom = L.pop(0)
        return jobs
    if strategy == "bfs":
        level = [make_job({})]
        for r in range(1, R):
            cands = []
            for jb in level:
                for b in jb["top"]:
                    cands.append((float(jb["bins"][b]), child_zoom(jb, b)))
            cands.sort(key=lambda x: -x[0])
            cands = cands[:T]
            if not cands:
                break
            level = [make_job(z) for _, z in cands]
        return jobs
    raise ValueError(strategy)
