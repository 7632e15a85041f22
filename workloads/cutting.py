"""Circuit DAG, wire cuts, subcircuit extraction and a simple cut search.

The paper's cut searcher (Framework Overview, "MIP Cut Searcher") models the
circuit as a DAG whose vertices are the multi-qubit gates and whose edges are
qubit-wire segments; single-qubit gates are ignored.  Cutting = clustering the
vertices; the cuts are the cross-cluster edges.  Its objective is Eq. 2.  The
MIP solver itself is a licensed comparison system and is not rebuilt; this
module searches the same space with a local search (gate moves between
clusters) under the same two user constraints: a maximum subcircuit width and
a maximum number of subcircuits.

Conventions fixed here (the paper is silent on them):
* a subcircuit's local qubits are its wire segments, sorted by (original
  qubit, time); an output segment is the last segment of its qubit, so output
  local order is ascending original-qubit order;
* a single-qubit gate between two multi-qubit gates of a wire belongs to the
  segment of the earlier one (the cut sits just before the later gate);
* cut-edge ids are numbered in program order of the downstream gate (ties by
  qubit);
* qubits that touch no multi-qubit gate are placed in a subcircuit with spare
  width, or in an extra cut-free subcircuit.

No reconstruction arithmetic lives here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .circuits import Circuit


@dataclass
class Subcircuit:
    """One subcircuit (its structure, not its outputs).

    ``w``          width (number of local qubits)
    ``seg``        per local qubit: (original qubit, run index on that qubit)
    ``init``       per local qubit: -1 for |0> (original input) else the id of
                   the incoming cut edge
    ``meas``       per local qubit: -1 for an output else the id of the outgoing
                   cut edge
    ``gates``      local gate list (name, local qubits, params)
    """
    w: int
    seg: list
    init: list
    meas: list
    gates: list = field(default_factory=list)

    @property
    def in_local(self):
        return [q for q in range(self.w) if self.init[q] >= 0]

    @property
    def out_local(self):
        return [q for q in range(self.w) if self.meas[q] >= 0]

    @property
    def in_edge(self):
        return [self.init[q] for q in self.in_local]

    @property
    def out_edge(self):
        return [self.meas[q] for q in self.out_local]

    @property
    def output_local(self):
        return [q for q in range(self.w) if self.meas[q] < 0]

    @property
    def out_qubit(self):
        return [self.seg[q][0] for q in self.output_local]

    @property
    def k_in(self):
        return len(self.in_local)

    @property
    def k_out(self):
        return len(self.out_local)

    @property
    def o(self):
        return self.w - self.k_out

    @property
    def edges(self):
        """Cut edges touching this subcircuit, ascending id."""
        return sorted(self.in_edge + self.out_edge)


@dataclass
class Cut:
    circuit: Circuit
    cluster: list           # cluster id per two-qubit gate (program order)
    free_cluster: dict      # qubit -> cluster for qubits without 2q gates
    subcircuits: list
    edges: list             # edge id -> (qubit, upstream cluster, downstream cluster)

    @property
    def K(self):
        return len(self.edges)

    @property
    def n_sub(self):
        return len(self.subcircuits)


class Dag:
    """Vertices: two-qubit gates; per qubit the ordered list of its vertices."""

    def __init__(self, circuit: Circuit):
        self.circuit = circuit
        self.n = circuit.n
        self.vpos = []        # program index of each vertex
        self.vq = []          # (q0, q1)
        self.wire = [[] for _ in range(circuit.n)]   # per qubit: vertex ids
        for p, (name, qs, _) in enumerate(circuit.gates):
            if len(qs) == 2:
                v = len(self.vpos)
                self.vpos.append(p)
                self.vq.append(qs)
                for q in qs:
                    self.wire[q].append(v)
        self.nv = len(self.vpos)
        # position of vertex v on each of its qubits
        self.slot = [dict() for _ in range(self.nv)]
        for q in range(self.n):
            for i, v in enumerate(self.wire[q]):
                self.slot[v][q] = i
        self.free_qubits = [q for q in range(self.n) if not self.wire[q]]


# --------------------------------------------------------------------------
# clustering -> subcircuits
# --------------------------------------------------------------------------

def build_cut(circuit: Circuit, cluster, free_cluster=None, w_max=None):
    dag = Dag(circuit)
    cluster = [int(c) for c in cluster]
    assert len(cluster) == dag.nv
    # runs per qubit
    runs = {}   # q -> list of (cluster, first slot, last slot)
    for q in range(dag.n):
        r = []
        for i, v in enumerate(dag.wire[q]):
            c = cluster[v]
            if r and r[-1][0] == c:
                r[-1][2] = i
            else:
                r.append([c, i, i])
        runs[q] = r
    used = sorted(set(cluster))
    width = {c: 0 for c in used}
    for q in range(dag.n):
        for c, _, _ in runs[q]:
            width[c] += 1
    # free qubits
    if free_cluster is None:
        free_cluster = {}
        for q in dag.free_qubits:
            best = None
            for c in used:
                if w_max is None or width[c] < w_max:
                    if best is None or width[c] < width[best]:
                        best = c
            if best is None:
                best = max(list(width.keys()) + [-1]) + 1
                width[best] = 0
                used.append(best)
            free_cluster[q] = best
            width[best] += 1
    else:
        for q, c in free_cluster.items():
            width.setdefault(c, 0)
            width[c] += 1
            if c not in used:
                used.append(c)
    used = sorted(set(used))
    for q in dag.free_qubits:
        runs[q] = [[free_cluster[q], -1, -1]]
    # cut edges: between consecutive runs, numbered by downstream gate position
    raw_edges = []
    for q in range(dag.n):
        r = runs[q]
        for j in range(len(r) - 1):
            v_down = dag.wire[q][r[j + 1][1]]
            raw_edges.append((dag.vpos[v_down], q, j, r[j][0], r[j + 1][0]))
    raw_edges.sort()
    edge_id = {}
    edges = []
    for e, (_, q, j, cu, cd) in enumerate(raw_edges):
        edge_id[(q, j)] = e
        edges.append((q, cu, cd))
    # subcircuits
    remap = {c: i for i, c in enumerate(used)}
    segs = {i: [] for i in range(len(used))}
    for q in range(dag.n):
        for j, (c, _, _) in enumerate(runs[q]):
            segs[remap[c]].append((q, j))
    subs = []
    local_of = {}
    for i in range(len(used)):
        sl = sorted(segs[i])
        init, meas = [], []
        for lq, (q, j) in enumerate(sl):
            local_of[(q, j)] = (i, lq)
            init.append(edge_id[(q, j - 1)] if j > 0 else -1)
            meas.append(edge_id[(q, j)] if j < len(runs[q]) - 1 else -1)
        subs.append(Subcircuit(w=len(sl), seg=sl, init=init, meas=meas))
    # assign gates to segments
    v_of_pos = {p: v for v, p in enumerate(dag.vpos)}
    for p, (name, qs, params) in enumerate(circuit.gates):
        if len(qs) == 2:
            v = v_of_pos[p]
            locs = []
            for q in qs:
                j = _run_index(runs[q], dag.slot[v][q])
                locs.append(local_of[(q, j)])
            i = locs[0][0]
            assert locs[1][0] == i
            subs[i].gates.append((name, (locs[0][1], locs[1][1]), params))
        else:
            q = qs[0]
            if not dag.wire[q]:
                j = 0
            else:
                # latest 2q gate on q before p (upstream segment), else first run
                slot = -1
                for i2, v in enumerate(dag.wire[q]):
                    if dag.vpos[v] < p:
                        slot = i2
                    else:
                        break
                j = _run_index(runs[q], max(slot, 0))
            i, lq = local_of[(q, j)]
            subs[i].gates.append((name, (lq,), params))
    cl = [remap[c] for c in cluster]
    fc = {q: remap[c] for q, c in free_cluster.items()}
    edges = [(q, remap[cu], remap[cd]) for (q, cu, cd) in edges]
    return Cut(circuit=circuit, cluster=cl, free_cluster=fc, subcircuits=subs, edges=edges)


def _run_index(runs_q, slot):
    for j, (_, a, b) in enumerate(runs_q):
        if a <= slot <= b:
            return j
    raise ValueError(slot)


# --------------------------------------------------------------------------
# cost models
# --------------------------------------------------------------------------

def eq2_cost(cut: Cut):
    """Eq. 2: L = 4^K * sum_{c=2}^{n_C} prod_{i=1}^{c} 2^{n_i}, with n_i the
    output-qubit count of subcircuit i and subcircuits taken in ascending n_i
    (the paper does not fix either)."""
    o = sorted(s.o for s in cut.subcircuits)
    total = 0
    for c in range(2, len(o) + 1):
        total += 2 ** sum(o[:c])
    return (4 ** cut.K) * total


def contraction_plan(sizes, edge_sets):
    """Greedy pairwise contraction order.  ``sizes[i]`` = number of output bits
    of tensor i, ``edge_sets[i]`` = set of its open cut edges.  Repeatedly
    contracts the pair (sharing at least one edge if any pair does) whose
    contraction is cheapest, where contracting (a, b) costs
    2 * 4^|Ea u Eb| * 2^(oa + ob) flops.  Returns (steps, total_flops), steps a
    list of (i, j) over a growing tensor list (new tensors appended)."""
    sizes = list(sizes)
    es = [frozenset(e) for e in edge_sets]
    alive = list(range(len(sizes)))
    steps, total = [], 0
    while len(alive) > 1:
        best = None
        for ia in range(len(alive)):
            for ib in range(ia + 1, len(alive)):
                a, b = alive[ia], alive[ib]
                share = bool(es[a] & es[b])
                cost = 2 * 4 ** len(es[a] | es[b]) * 2 ** (sizes[a] + sizes[b])
                key = (0 if share else 1, cost, a, b)
                if best is None or key < best[0]:
                    best = (key, a, b, cost)
        _, a, b, cost = best
        total += cost
        steps.append((a, b))
        sizes.append(sizes[a] + sizes[b])
        es.append(es[a] ^ es[b])
        alive = [x for x in alive if x not in (a, b)] + [len(sizes) - 1]
    return steps, total


def contraction_cost(cut: Cut):
    """Flops of the greedy pairwise contraction of the FD reconstruction
    (2 per multiply-add) plus 4 bytes per output written; the exact
    reconstruction cost the cut scorer learns."""
    _, flops = contraction_plan([s.o for s in cut.subcircuits],
                                [set(s.edges) for s in cut.subcircuits])
    return flops + 4 * 2 ** cut.circuit.n


# --------------------------------------------------------------------------
# local search
# --------------------------------------------------------------------------

class _State:
    """Incremental bookkeeping for gate moves: per-cluster width and cut count."""

    def __init__(self, dag: Dag, cluster, n_clusters):
        self.dag = dag
        self.c = list(cluster)
        self.k = n_clusters
        self.width = [0] * n_clusters
        self.cuts = 0
        for q in range(dag.n):
            seq = [self.c[v] for v in dag.wire[q]]
            for i, x in enumerate(seq):
                if i == 0 or seq[i - 1] != x:
                    self.width[x] += 1
                if i > 0 and seq[i - 1] != x:
                    self.cuts += 1

    def delta(self, v, b):
        """(d_cuts, d_width per cluster as dict) of moving vertex v to b."""
        a = self.c[v]
        if a == b:
            return 0, {}
        dcut = 0
        dw = {}
        for q in self.dag.vq[v]:
            seq = self.dag.wire[q]
            i = self.dag.slot[v][q]
            prev = self.c[seq[i - 1]] if i > 0 else None
            nxt = self.c[seq[i + 1]] if i + 1 < len(seq) else None
            # starts of runs among positions i and i+1 before/after
            def starts(cur):
                s = []
                if prev is None or prev != cur:
                    s.append(cur)
                if nxt is not None and nxt != cur:
                    s.append(nxt)
                return s
            def ncut(cur):
                return (prev is not None and prev != cur) + (nxt is not None and nxt != cur)
            for x in starts(a):
                dw[x] = dw.get(x, 0) - 1
            for x in starts(b):
                dw[x] = dw.get(x, 0) + 1
            dcut += ncut(b) - ncut(a)
        return dcut, dw

    def apply(self, v, b):
        dcut, dw = self.delta(v, b)
        self.cuts += dcut
        for x, d in dw.items():
            self.width[x] += d
        self.c[v] = b


def _objective(cuts, width, w_max):
    excess = sum(max(0, w - w_max) for w in width)
    return excess * 1000 + cuts


def _initial_blocks(dag: Dag, order, k):
    """Contiguous blocks of the given qubit order; a gate goes to the block of
    its first qubit in that order."""
    n = dag.n
    rank = {q: i for i, q in enumerate(order)}
    block = {q: min(k - 1, rank[q] * k // n) for q in range(n)}
    return [min(block[a], block[b]) for (a, b) in dag.vq]


def search_cut(circuit: Circuit, w_max, n_sub, orders=None, restarts=4, seed=0,
               max_passes=50, anneal_steps=None):
    """Local search for a clustering of the two-qubit gates into ``n_sub``
    clusters with every width <= w_max, minimising the number of cuts, then
    the contraction cost.  Each restart starts from contiguous qubit blocks of
    one of ``orders`` (randomly perturbed after the first round), runs
    simulated annealing over single-gate moves to a neighbouring cluster, then
    a greedy descent.  Returns the best Cut found, or None if no restart
    reached a feasible clustering."""
    dag = Dag(circuit)
    rng = np.random.default_rng(seed)
    if orders is None:
        orders = [list(range(circuit.n))]
    if anneal_steps is None:
        anneal_steps = 200 * max(dag.nv, 1)
    best = None
    n_free = len(dag.free_qubits)
    for r in range(restarts):
        order = orders[r % len(orders)]
        init = _initial_blocks(dag, order, n_sub)
        if r >= len(orders):
            init = list(init)
            for v in range(dag.nv):
                if rng.random() < 0.1:
                    nb = _neighbour_clusters(dag, init, v)
                    if nb:
                        init[v] = int(rng.choice(sorted(nb)))
        st = _State(dag, init, n_sub)
        _anneal(st, w_max, rng, anneal_steps)
        _descend(st, w_max, rng, max_passes)
        cand = _finish(circuit, st, w_max, n_free)
        if cand is None:
            continue
        key = _rank(cand, w_max)
        if best is None or key < best[0]:
            best = (key, cand)
    return None if best is None else best[1]


def _anneal(st: _State, w_max, rng, steps, t0=2.0, t1=0.05, penalty=3.0):
    """Simulated annealing on cuts + penalty * width excess; leaves ``st`` at
    the best feasible state seen (or the best state if none was feasible)."""
    dag = st.dag
    if dag.nv == 0 or steps <= 0:
        return

    def obj(cuts, width):
        return cuts + penalty * sum(max(0, w - w_max) for w in width)

    cur = obj(st.cuts, st.width)
    best_c, best_val = list(st.c), (cur if max(st.width) <= w_max else None)
    best_any, best_any_val = list(st.c), cur
    verts = rng.integers(0, dag.nv, size=steps)
    us = rng.random(steps)
    for i in range(steps):
        t = t0 * (t1 / t0) ** (i / steps)
        v = int(verts[i])
        nb = _neighbour_clusters(dag, st.c, v)
        if not nb:
            continue
        nb = sorted(nb)
        b = nb[int(us[i] * len(nb)) % len(nb)]
        dcut, dw = st.delta(v, b)
        w2 = list(st.width)
        for x, d in dw.items():
            w2[x] += d
        if w2[st.c[v]] <= 0 and st.width[st.c[v]] > 0 and sum(1 for w in w2 if w > 0) < sum(1 for w in st.width if w > 0):
            continue    # never empty a cluster
        val = obj(st.cuts + dcut, w2)
        d = val - cur
        if d <= 0 or rng.random() < math.exp(-d / t):
            st.apply(v, b)
            cur = val
            if max(st.width) <= w_max and (best_val is None or cur < best_val):
                best_c, best_val = list(st.c), cur
            if cur < best_any_val:
                best_any, best_any_val = list(st.c), cur
    target = best_c if best_val is not None else best_any
    for v in range(dag.nv):
        if st.c[v] != target[v]:
            st.apply(v, target[v])


def _neighbour_clusters(dag, cl, v):
    s = set()
    for q in dag.vq[v]:
        seq = dag.wire[q]
        i = dag.slot[v][q]
        if i > 0:
            s.add(cl[seq[i - 1]])
        if i + 1 < len(seq):
            s.add(cl[seq[i + 1]])
    s.discard(cl[v])
    return s


def _descend(st: _State, w_max, rng, max_passes):
    dag = st.dag
    cur = _objective(st.cuts, st.width, w_max)
    for _ in range(max_passes):
        improved = False
        order = rng.permutation(dag.nv)
        for v in order:
            v = int(v)
            for b in sorted(_neighbour_clusters(dag, st.c, v)):
                dcut, dw = st.delta(v, b)
                w2 = list(st.width)
                for x, d in dw.items():
                    w2[x] += d
                val = _objective(st.cuts + dcut, w2, w_max)
                if val < cur:
                    st.apply(v, b)
                    cur = val
                    improved = True
                    break
        if not improved:
            break
    return cur


def _finish(circuit, st: _State, w_max, n_free):
    if any(w > w_max for w in st.width):
        return None
    cut = build_cut(circuit, st.c, w_max=w_max)
    if any(s.w > w_max for s in cut.subcircuits):
        return None
    return cut


def _rank(cut: Cut, w_max):
    return (cut.K, contraction_cost(cut))


def grid_orders(rows, cols):
    """Row-major and column-major qubit orders of a rows x cols grid."""
    rm = list(range(rows * cols))
    cm = [r * cols + c for c in range(cols) for r in range(rows)]
    return [rm, cm]


# --------------------------------------------------------------------------
# exact search (branch and bound) for small circuits
# --------------------------------------------------------------------------

def _eq2_from_outputs(K, outs):
    """Eq. 2 for K cuts and the subcircuits' output counts (ascending order)."""
    o = sorted(outs)
    return (4 ** K) * sum(2 ** sum(o[:c]) for c in range(2, len(o) + 1))


def exact_cut(circuit: Circuit, w_max, n_sub, max_nodes=2_000_000, incumbent=None, max_ties=64, lookahead=True):
    """Branch and bound for the cut the paper's MIP cut searcher finds: a
    clustering of the two-qubit gates into at most ``n_sub`` clusters, every
    width <= w_max (its two constraints), minimising Eq. 2, L = 4^K sum_c
    prod_{i<=c} 2^{n_i} (``eq2_cost``); among equal L the cheaper contraction
    (``contraction_cost``) wins.  Gates are assigned in program order, so each
    qubit's wire grows one gate at a time: a gate placed in a cluster other
    than its qubit's previous one cuts the wire there and opens a new wire
    segment in that cluster (width + 1); a qubit's first gate opens its
    original input.  Clusters are introduced in order (symmetry).  Bound: L >=
    4^(K_now + k_ahead) 2^n for n_C >= 2, where k_ahead counts the unassigned
    gates that are the next gate on both of their qubits while those qubits'
    latest gates sit in different clusters (each must cut one of its two
    wires, and no two share a wire).  ``incumbent`` (a Cut, e.g. from the
    local search) seeds the best L so that worse branches are cut from the
    start (``lookahead=False`` drops k_ahead from the bound).  Returns
    (Cut, exhaustive) -- exhaustive False when the node
    budget ran out first (the Cut is then the best found, never worse than
    the incumbent) -- or (None, exhaustive) when nothing fits."""
    dag = Dag(circuit)
    nv, n = dag.nv, dag.n
    free = list(dag.free_qubits)
    nxt_of = [[-1, -1] for _ in range(nv)]       # next gate on each of v's two qubits
    for v in range(nv):
        for t, q in enumerate(dag.vq[v]):
            i = dag.slot[v][q]
            nxt_of[v][t] = dag.wire[q][i + 1] if i + 1 < len(dag.wire[q]) else -1
    pos_on = [[dag.slot[v][q] for q in dag.vq[v]] for v in range(nv)]
    best = {"L": None, "leaves": []}
    if incumbent is not None and all(sb.w <= w_max for sb in incumbent.subcircuits) \
            and len(incumbent.subcircuits) <= n_sub + len(free):
        best["L"] = eq2_cost(incumbent)
    assign = [0] * nv
    last = [-1] * n              # cluster of each qubit's latest assigned gate
    done_on = [0] * n            # gates assigned on each qubit
    width = [0] * n_sub
    nodes = [0]
    two_n = 2 ** n

    def ready_conflict(u):
        if u < 0:
            return 0
        a, b = dag.vq[u]
        if done_on[a] != pos_on[u][0] or done_on[b] != pos_on[u][1]:
            return 0
        return 1 if (last[a] >= 0 and last[b] >= 0 and last[a] != last[b]) else 0

    def leaf_L(cuts, used):
        outs = [0] * used
        for q in range(n):
            if last[q] >= 0:
                outs[last[q]] += 1
        w = list(width[:used])
        for _ in free:          # as build_cut: the narrowest cluster with room, else a new one
            c = min((c for c in range(len(w)) if w[c] < w_max), key=lambda c: (w[c], c), default=None)
            if c is None:
                w.append(0)
                outs.append(0)
                c = len(w) - 1
            w[c] += 1
            outs[c] += 1
        return _eq2_from_outputs(cuts, outs)

    def rec(v, used, cuts, ahead):
        nodes[0] += 1
        if nodes[0] > max_nodes:
            return False
        if best["L"] is not None and cuts + ahead > 0 and (4 ** (cuts + ahead)) * two_n > best["L"]:
            return True
        if v == nv:
            L = leaf_L(cuts, used)
            if L is None:
                return True
            if best["L"] is None or L < best["L"]:
                best["L"], best["leaves"] = L, []
            if L == best["L"] and len(best["leaves"]) < max_ties:
                best["leaves"].append(list(assign))
            return True
        q0, q1 = dag.vq[v]
        before = ready_conflict(v)
        for c in range(min(used + 1, n_sub)):
            dc = 0
            opened = 0
            for q in (q0, q1):
                if last[q] != c:
                    if last[q] >= 0:
                        dc += 1
                    opened += 1
            if width[c] + opened > w_max:
                continue
            saved = (last[q0], last[q1])
            width[c] += opened
            last[q0] = last[q1] = c
            done_on[q0] += 1
            done_on[q1] += 1
            assign[v] = c
            u0, u1 = nxt_of[v]
            after = ready_conflict(u0) + (ready_conflict(u1) if u1 != u0 else 0)
            ok = rec(v + 1, max(used, c + 1), cuts + dc, (ahead - before + after) if lookahead else 0)
            done_on[q0] -= 1
            done_on[q1] -= 1
            last[q0], last[q1] = saved
            width[c] -= opened
            if not ok:
                return False
        return True

    exhaustive = rec(0, 0, 0, 0) if nv else True
    cands = []
    for cl in best["leaves"]:
        cut = build_cut(circuit, cl, w_max=w_max)
        if all(sb.w <= w_max for sb in cut.subcircuits) and len(cut.subcircuits) <= n_sub + len(free):
            cands.append(((eq2_cost(cut), contraction_cost(cut)), cut))
    if incumbent is not None and best["L"] is not None and eq2_cost(incumbent) <= best["L"]:
        cands.append(((eq2_cost(incumbent), contraction_cost(incumbent)), incumbent))
    if not cands:
        return None, exhaustive
    return min(cands, key=lambda x: x[0])[1], exhaustive
