"""Seeded star and chain basic graph patterns drawn from witnesses in the data.

Each BGP is made from a witness: a random star (k edges at one node) or chain
(a k-edge path, edges taken in either direction) of the graph.  The witness's
nodes become variables except one or two that are kept as constants, so every
generated BGP has at least one solution (the witness itself).  Class and rank
terms and label terms are hubs or dead ends and may only be a leaf of a witness.

A candidate is kept only if an upper bound on its result size stays at or below
``max_rows``: starting from the constants, each variable is reached by one edge
of a spanning tree and can take at most the largest fan-out of that predicate in
that direction (a statistic of the data, not a join).  The bound replaces a
result-size filter that would need the query evaluated.

A pattern is ``(s, p, o, var_mask)``: bit 0 set means ``s`` holds a variable id,
bit 2 set means ``o`` holds a variable id; the predicate is always a constant.
"""
from __future__ import annotations

import numpy as np

from .rng import Rng
from .university import FIRST_ENTITY, P

VAR_S, VAR_P, VAR_O = 1, 2, 4


class GraphIndex:
    """Incidence lists of a triple set, for drawing witnesses."""

    def __init__(self, s, p, o):
        self.s = np.asarray(s, dtype=np.int64)
        self.p = np.asarray(p, dtype=np.int64)
        self.o = np.asarray(o, dtype=np.int64)
        n_ids = int(max(self.s.max(), self.o.max())) + 1
        self.out_order = np.argsort(self.s, kind="stable")
        self.out_first = np.searchsorted(self.s[self.out_order], np.arange(n_ids + 1))
        self.in_order = np.argsort(self.o, kind="stable")
        self.in_first = np.searchsorted(self.o[self.in_order], np.arange(n_ids + 1))
        self.is_label = np.zeros(n_ids, dtype=bool)
        self.is_label[self.o[self.p == P["label"]]] = True
        self.n_ids = n_ids
        n_pred = int(self.p.max()) + 1
        self.max_out = np.zeros(n_pred, dtype=np.int64)
        self.max_in = np.zeros(n_pred, dtype=np.int64)
        for side, dst in ((self.s, self.max_out), (self.o, self.max_in)):
            keys, cnt = np.unique(self.p * (1 << 32) + side, return_counts=True)
            np.maximum.at(dst, keys >> 32, cnt)

    def is_inner(self, node: int) -> bool:
        """May a witness pass through this node (entity, not a hub or label)?"""
        return node >= FIRST_ENTITY and not self.is_label[node]

    def incident(self, node: int):
        """Edges at ``node`` as (triple index, other endpoint, node is subject)."""
        a, b = self.out_first[node], self.out_first[node + 1]
        out_t = self.out_order[a:b]
        c, d = self.in_first[node], self.in_first[node + 1]
        in_t = self.in_order[c:d]
        tri = np.concatenate((out_t, in_t))
        other = np.concatenate((self.o[out_t], self.s[in_t]))
        is_subj = np.concatenate((np.ones(out_t.shape[0], bool), np.zeros(in_t.shape[0], bool)))
        return tri, other, is_subj


def _draw_star(g: GraphIndex, r: Rng, k: int):
    for _ in range(64):
        c = int(FIRST_ENTITY + r.below(1, g.n_ids - FIRST_ENTITY)[0])
        if not g.is_inner(c):
            continue
        tri, _, _ = g.incident(c)
        if tri.shape[0] < k:
            continue
        pick = np.argsort(r.u64(tri.shape[0]), kind="stable")[:k]
        return [int(t) for t in tri[pick]]
    return None


def _draw_chain(g: GraphIndex, r: Rng, k: int):
    for _ in range(64):
        cur = int(FIRST_ENTITY + r.below(1, g.n_ids - FIRST_ENTITY)[0])
        if not g.is_inner(cur):
            continue
        visited = {cur}
        edges = []
        ok = True
        for step in range(k):
            if not g.is_inner(cur):
                ok = False
                break
            tri, other, _ = g.incident(cur)
            fresh = np.array([int(x) not in visited for x in other], dtype=bool)
            if not fresh.any():
                ok = False
                break
            tri, other = tri[fresh], other[fresh]
            j = int(r.below(1, tri.shape[0])[0])
            edges.append(int(tri[j]))
            cur = int(other[j])
            visited.add(cur)
        if ok:
            return edges
    return None


def _bound(g: GraphIndex, pats, const_nodes, nodes):
    """Spanning-tree fan-out bound on the number of solutions."""
    reached = set(const_nodes)
    bound = 1
    changed = True
    while changed:
        changed = False
        for (s, p, o) in pats:
            if s in reached and o not in reached:
                bound *= int(g.max_out[p])
                reached.add(o)
                changed = True
            elif o in reached and s not in reached:
                bound *= int(g.max_in[p])
                reached.add(s)
                changed = True
    assert reached == set(nodes)
    return bound


def generate_bgps(g: GraphIndex, n: int, seed: int, k_range=(3, 6), var_range=(2, 5),
                  max_rows: int = 1 << 26):
    """``n`` BGPs, alternating star and chain.  Each entry is a dict with
    ``patterns`` (list of (s, p, o, var_mask)), ``shape``, ``witness`` (variable id
    -> term id) and ``bound``."""
    out = []
    attempt = 0
    while len(out) < n:
        r = Rng(seed, 1 << 20 | attempt)
        attempt += 1
        shape = "star" if len(out) % 2 == 0 else "chain"
        k = int(r.between(1, k_range[0], k_range[1])[0])
        edges = _draw_star(g, r, k) if shape == "star" else _draw_chain(g, r, k)
        if edges is None:
            continue
        trip = [(int(g.s[t]), int(g.p[t]), int(g.o[t])) for t in edges]
        nodes = []
        for (s, _, o) in trip:
            for x in (s, o):
                if x not in nodes:
                    nodes.append(x)
        choices = [1, 2] if r.below(1, 2)[0] == 0 else [2, 1]
        n_const = None
        for c in choices:
            nv = len(nodes) - c
            if var_range is None or var_range[0] <= nv <= var_range[1]:
                n_const = c
                break
        if n_const is None or n_const >= len(nodes):
            continue
        perm = np.argsort(r.u64(len(nodes)), kind="stable")
        consts = [nodes[int(i)] for i in perm[:n_const]]
        variables = [x for x in nodes if x not in consts]
        var_id = {x: i for i, x in enumerate(variables)}
        bound = _bound(g, trip, consts, nodes)
        if bound > max_rows:
            continue
        pats = []
        for (s, p, o) in trip:
            mask = 0
            fs, fo = s, o
            if s in var_id:
                mask |= VAR_S
                fs = var_id[s]
            if o in var_id:
                mask |= VAR_O
                fo = var_id[o]
            pats.append((fs, p, fo, mask))
        out.append({"patterns": pats, "shape": shape,
                    "witness": {v: x for x, v in var_id.items()}, "bound": bound})
    return out
