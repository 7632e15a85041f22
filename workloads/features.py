"""Candidate wire cuts, their 64 structural features and their exact cost.

A candidate is a clustering of a circuit's two-qubit gates (the DAG vertices
of the paper's cut searcher) into at most ``MAX_SUB - 1`` clusters.  For a
batch of candidates of one circuit this module derives, with array
operations and without building subcircuits:

* per cluster: width w (wire segments), incoming and outgoing cut counts
  k_in / k_out, output count o = w - k_out;
* the cut edges and the clusters they join;
* the 64 features the cut-scoring network reads;
* the exact reconstruction cost (the greedy pairwise contraction cost of
  ``cutting.contraction_cost``), the network's training label.

Free qubits (no two-qubit gate) are placed exactly as ``cutting.build_cut``
places them: each, in qubit order, into the used cluster of smallest width
that still has spare width (lowest id on ties), else into a new cluster.

No reconstruction arithmetic lives here: this is input generation for the
cut scorer, shared by its tests and the benchmark.
"""
from __future__ import annotations

import math

import numpy as np

from .cutting import Dag, contraction_plan

N_FEATURES = 64
MAX_SUB = 8          # cluster slots per candidate (assignments use < MAX_SUB)
LABEL_SCALE = 16.0   # label = (log2 cost - n) / LABEL_SCALE


class CandidateSet:
    """Structure of a batch of candidate clusterings of one circuit."""

    def __init__(self, dag: Dag, assign, w_max):
        assign = np.asarray(assign, dtype=np.int64)
        if assign.ndim == 1:
            assign = assign[None]
        C, V = assign.shape
        assert V == dag.nv and assign.min(initial=0) >= 0 and assign.max(initial=0) < MAX_SUB - 1
        S = MAX_SUB
        self.dag, self.n, self.C, self.w_max = dag, dag.n, C, w_max
        wv = [v for q in range(dag.n) for v in dag.wire[q]]
        first = np.array([i == 0 for q in range(dag.n) for i in range(len(dag.wire[q]))], dtype=bool)
        last = np.array([i == len(dag.wire[q]) - 1 for q in range(dag.n) for i in range(len(dag.wire[q]))],
                        dtype=bool)
        cl = assign[:, np.asarray(wv, dtype=np.int64)] if wv else np.zeros((C, 0), np.int64)
        L = cl.shape[1]
        prev = np.concatenate([np.full((C, 1), -1), cl[:, :-1]], axis=1) if L else cl
        nxt = np.concatenate([cl[:, 1:], np.full((C, 1), -1)], axis=1) if L else cl
        start = first[None] | (cl != prev)
        end = last[None] | (cl != nxt)
        cut_at = start & ~first[None]          # a cut edge enters a run here
        # per (candidate, cluster) counts of run starts, cut entries and cut exits
        flat = np.arange(C, dtype=np.int64)[:, None] * S + cl
        count = lambda m: np.bincount(flat[m], minlength=C * S).reshape(C, S)
        w = count(start)
        k_in = count(cut_at)
        k_out = count(end & ~last[None])
        # free qubits, placed as build_cut places them
        overflow = np.zeros(C, dtype=bool)
        for _ in dag.free_qubits:
            used = w > 0
            spare = used & (w < w_max)
            key = np.where(spare, w, 1 << 30)
            best = key.argmin(1)
            none = ~spare.any(1)
            if none.any():
                # a new cluster: the lowest unused slot above every used id
                top = np.where(used, np.arange(S), -1).max(1) + 1
                overflow |= none & (top >= S)
                best = np.where(none, np.minimum(top, S - 1), best)
            w[np.arange(C), best] += 1
        self.w, self.k_in, self.k_out = w, k_in, k_out
        self.o = w - k_out
        self.used = w > 0
        self.K = cut_at.sum(1)
        # cut edges: (candidate, upstream cluster, downstream cluster)
        ci, pos = np.nonzero(cut_at)
        self._edge_c = ci
        self._edge_a = prev[ci, pos]
        self._edge_b = cl[ci, pos]
        pair = np.zeros((C, S, S), dtype=np.int64)
        np.add.at(pair, (ci, np.minimum(self._edge_a, self._edge_b), np.maximum(self._edge_a, self._edge_b)), 1)
        self.pair = pair + pair.transpose(0, 2, 1)     # symmetric cut counts
        self.feasible = (w.max(1) <= w_max) & (self.used.sum(1) >= 1) & ~overflow
        # variant tensor entries 4^k_in * 3^k_out * 2^w per subcircuit (log2)
        vlog = 2.0 * k_in + math.log2(3.0) * k_out + w
        self.variant_log2 = np.where(self.used, vlog, -np.inf)

    def subset(self, idx):
        """The candidates ``idx`` (in that order) as a CandidateSet of their
        own, without recomputing their structure."""
        idx = np.asarray(idx, dtype=np.int64)
        sub = object.__new__(CandidateSet)
        sub.dag, sub.n, sub.w_max, sub.C = self.dag, self.n, self.w_max, len(idx)
        for name in ("w", "k_in", "k_out", "o", "used", "K", "pair", "feasible", "variant_log2"):
            setattr(sub, name, getattr(self, name)[idx])
        pos = np.full(self.C, -1, dtype=np.int64)
        pos[idx] = np.arange(len(idx))
        keep = pos[self._edge_c] >= 0
        sub._edge_c = pos[self._edge_c[keep]]
        sub._edge_a = self._edge_a[keep]
        sub._edge_b = self._edge_b[keep]
        return sub

    # ------------------------------------------------------------------
    def features(self):
        """[C, 64] float32 features (see the module docstring)."""
        C, S = self.C, MAX_SUB
        f = np.zeros((C, N_FEATURES), dtype=np.float64)
        n = self.n
        nsub = self.used.sum(1)
        k_tot = self.k_in + self.k_out
        # per-slot contraction estimate with the cheapest partner:
        # log2(2 * 4^|Ea u Eb| * 2^(oa + ob))
        union = k_tot[:, :, None] + k_tot[:, None, :] - self.pair
        lc = 1.0 + 2.0 * union + self.o[:, :, None] + self.o[:, None, :]
        valid = self.used[:, :, None] & self.used[:, None, :] & ~np.eye(S, dtype=bool)[None]
        lc = np.where(valid, lc, np.inf).min(2)
        nbrs = (self.pair > 0).sum(2)
        # slots ordered by (o, w, k_in, k_out, neighbours, estimate), largest
        # first, unused last: the order does not depend on the cluster ids
        big = 1 << 20
        keys = [np.where(np.isfinite(lc), -lc, -big), nbrs, self.k_out, self.k_in, self.w,
                np.where(self.used, self.o, -big)]
        order = np.lexsort([-k for k in keys], axis=-1)
        take = lambda a: np.take_along_axis(a, order, axis=1)
        w, o, kin, kout, used = take(self.w), take(self.o), take(self.k_in), take(self.k_out), take(self.used)
        pair = np.take_along_axis(np.take_along_axis(self.pair, order[:, :, None], axis=1), order[:, None, :], axis=2)
        lc = take(lc)
        f[:, 0] = n / 64.0
        f[:, 1] = self.dag.nv / 512.0
        f[:, 2] = nsub / 8.0
        f[:, 3] = self.K / 16.0
        f[:, 4] = self.w.max(1) / 32.0
        f[:, 5] = self.w_max / 32.0
        f[:, 6] = eq2_log2(self.o, self.used, self.K) / 64.0 - n / 64.0
        f[:, 7] = (self.pair > 0).sum((1, 2)) / 2.0 / 16.0      # cluster pairs joined by cuts
        base = 8
        for s in range(S):
            f[:, base + 5 * s + 0] = w[:, s] / 32.0
            f[:, base + 5 * s + 1] = o[:, s] / 32.0
            f[:, base + 5 * s + 2] = kin[:, s] / 16.0
            f[:, base + 5 * s + 3] = kout[:, s] / 16.0
            f[:, base + 5 * s + 4] = (pair[:, s] > 0).sum(1) / 8.0
        base += 5 * S
        iu = np.triu_indices(S, 1)
        pc = np.sort(pair[:, iu[0], iu[1]], axis=1)[:, ::-1][:, :8]
        f[:, base:base + 8] = pc / 16.0
        base += 8
        # per slot: the cheapest-partner estimate, relative to n
        f[:, base:base + 8] = np.where(np.isfinite(lc), lc - n, 0.0) / 32.0
        assert base + 8 == N_FEATURES
        return f.astype(np.float32)

    def edge_sets(self, c):
        """Per used cluster of candidate c (ascending id): set of its cut-edge ids."""
        sel = np.nonzero(self._edge_c == c)[0]
        ids = {}
        for e in sel:
            ids.setdefault(int(self._edge_a[e]), set()).add(int(e))
            ids.setdefault(int(self._edge_b[e]), set()).add(int(e))
        return [ids.get(s, set()) for s in range(MAX_SUB) if self.used[c, s]]

    def exact_cost(self, c):
        """Greedy pairwise contraction flops + 4 bytes per output: the value
        ``cutting.contraction_cost`` gives for the built cut."""
        sizes = [int(self.o[c, s]) for s in range(MAX_SUB) if self.used[c, s]]
        _, flops = contraction_plan(sizes, self.edge_sets(c))
        return flops + 4 * 2 ** self.n

    def labels(self, idx=None):
        idx = range(self.C) if idx is None else idx
        return np.array([(math.log2(self.exact_cost(c)) - self.n) / LABEL_SCALE for c in idx], dtype=np.float32)


def eq2_log2(o, used, K):
    """log2 of Eq. 2 (subcircuits in ascending output count), per candidate:
    2 K + log2 sum_{c >= 2} 2^(o_(1) + ... + o_(c)) over the used slots in
    ascending order (array operations over the candidates)."""
    C, S = o.shape
    oo = np.sort(np.where(used, o, np.inf).astype(np.float64), axis=1)
    valid = np.isfinite(oo)
    prefix = np.cumsum(np.where(valid, oo, 0.0), axis=1)
    terms = np.where(valid & (np.arange(S)[None, :] >= 1), np.exp2(prefix), 0.0)
    tot = terms.sum(1)
    return 2.0 * np.asarray(K, dtype=np.float64) + np.where(tot > 0, np.log2(np.where(tot > 0, tot, 1.0)), 0.0)


# --------------------------------------------------------------------------
# candidate generator
# --------------------------------------------------------------------------

def _bfs_order(dag: Dag, start, rng):
    """Qubit order by breadth-first search over the interaction graph."""
    nb = [set() for _ in range(dag.n)]
    for a, b in dag.vq:
        nb[a].add(b)
        nb[b].add(a)
    seen, order, frontier = {start}, [start], [start]
    while frontier:
        nxt = []
        for q in frontier:
            for r in sorted(nb[q]):
                if r not in seen:
                    seen.add(r)
                    order.append(r)
                    nxt.append(r)
        frontier = nxt
    rest = [q for q in range(dag.n) if q not in seen]
    return order + rest


def candidates(dag: Dag, w_max, count, rng, n_sub_range=None):
    """``count`` seeded candidate clusterings [count, nv]: contiguous blocks of
    a qubit order (identity, reversed, or breadth-first from a random qubit)
    with jittered block sizes; a gate joins the block of one of its qubits
    (the lower block, the higher, or that of its lower-degree qubit); then a
    random fraction of gates moves to the block of the other qubit.  All
    candidates are drawn at once (array operations over the candidates)."""
    n = dag.n
    deg = np.array([len(dag.wire[q]) for q in range(n)])
    nv = dag.nv
    vq = np.asarray(dag.vq, dtype=np.int64).reshape(nv, 2)
    lo = min(MAX_SUB - 1, max(2, -(-n // max(w_max, 1))))
    if n_sub_range is None:
        n_sub_range = (lo, min(MAX_SUB - 1, lo + 2))
    S = rng.integers(n_sub_range[0], n_sub_range[1] + 1, size=count)
    kind = rng.integers(3, size=count)
    start = rng.integers(n, size=count)
    # rank of every qubit in each candidate's order
    ident = np.arange(n)
    bfs_rank = {}
    rank = np.empty((count, n), dtype=np.int64)
    rank[kind == 0] = ident
    rank[kind == 1] = ident[::-1]
    for i in np.nonzero(kind == 2)[0]:
        q = int(start[i])
        if q not in bfs_rank:
            r = np.empty(n, dtype=np.int64)
            r[np.asarray(_bfs_order(dag, q, rng))] = ident
            bfs_rank[q] = r
        rank[i] = bfs_rank[q]
    # block sizes: Dirichlet(8, ..., 8) over S blocks (gamma draws, masked)
    s_max = int(S.max())
    g = rng.gamma(8.0, size=(count, s_max)) * (np.arange(s_max)[None, :] < S[:, None])
    bounds = np.cumsum(g / g.sum(1, keepdims=True), axis=1) * n
    block = np.minimum((bounds[:, None, :] < rank[:, :, None] + 0.5).sum(-1), S[:, None] - 1)
    b0 = np.take_along_axis(block, np.broadcast_to(vq[:, 0], (count, nv)), 1)
    b1 = np.take_along_axis(block, np.broadcast_to(vq[:, 1], (count, nv)), 1)
    rule = rng.integers(3, size=count)[:, None]
    lower_deg = (deg[vq[:, 0]] <= deg[vq[:, 1]])[None, :]
    a = np.where(rule == 0, np.minimum(b0, b1),
                 np.where(rule == 1, np.maximum(b0, b1), np.where(lower_deg, b0, b1)))
    p = rng.choice(np.array([0.0, 0.0, 0.02, 0.05, 0.1]), size=count)[:, None]
    flip = rng.random((count, nv)) < p
    other = np.where(a == b0, b1, b0)
    return np.where(flip, other, a).astype(np.int64)


def training_set(n_circuits, per_circuit, seed, n_range=(20, 60)):
    """Seeded training data for the cut scorer: ``n_circuits`` random circuits
    of ``n_range`` qubits (brick-wall / AQFT / supremacy / BV mix), each with
    ``per_circuit`` feasible candidates under a random width limit; returns
    (x [N, 64] float32, t [N] float32 labels, circuit index [N])."""
    from .circuits import random_family_circuit
    rng = np.random.default_rng(seed)
    xs, ts, gs = [], [], []
    for g in range(n_circuits):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        c = random_family_circuit(rng, n)
        dag = Dag(c)
        w_max = int(rng.integers(max(4, n // 6), max(5, n // 2) + 1))
        cs = CandidateSet(dag, candidates(dag, w_max, 4 * per_circuit, rng), w_max)
        ok = np.nonzero(cs.feasible)[0][:per_circuit]
        if len(ok) == 0:
            continue
        sub = cs.subset(ok)
        xs.append(sub.features())
        ts.append(sub.labels())
        gs.append(np.full(len(ok), g))
    return np.concatenate(xs), np.concatenate(ts), np.concatenate(gs)


def _chunk(args):
    n, per, seed, n_range = args
    return training_set(n, per, seed, n_range)


def training_set_parallel(n_circuits, per_circuit, seed, workers=8, chunk=250, n_range=(20, 60)):
    """``training_set`` over chunks of ``chunk`` circuits (chunk i seeded
    ``seed * 1000003 + i``) in a pool of spawned processes; the result does not
    depend on ``workers``."""
    import multiprocessing as mp
    jobs = []
    for i, c0 in enumerate(range(0, n_circuits, chunk)):
        jobs.append((min(chunk, n_circuits - c0), per_circuit, seed * 1000003 + i, n_range))
    if workers <= 1:
        parts = [_chunk(j) for j in jobs]
    else:
        import os
        keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
        os.environ.update({k: "1" for k in keep})       # one BLAS thread per worker
        try:
            with mp.get_context("spawn").Pool(workers) as pool:
                parts = pool.map(_chunk, jobs)
        finally:
            for k, v in keep.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
    x = np.concatenate([p[0] for p in parts])
    t = np.concatenate([p[1] for p in parts])
    g = np.concatenate([p[2] + i * chunk for i, p in enumerate(parts)])
    return x, t, g
