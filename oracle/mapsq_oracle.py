"""CPU oracle for MapSQ's join of partial-match tables (test infrastructure).

This module is test infrastructure.  Only the test suite, the package smoke
check and the benchmark's CPU-baseline leg may import or run it; the library
never does.  It is plain, slow and written to be checked against the paper by
eye: numpy arrays, no index structures, no blocking.

What it computes (MapSQ, arXiv 1702.03484):

* ``join_mapreduce``: Algorithm 1 (MapReduce-based Join) in the paper's order:
  Map splits every row of Tp1 and Tp2 into (key = shared variables, label =
  LEFT/RIGHT, value = the other columns); Sort orders the intermediates by key;
  ReduceDuplicate pairs, within each key, every LEFT value with every RIGHT
  value and puts (key, value1, value2) into RS.  Table 1(c) fixes the column
  layout: key, then Tp1's value, then Tp2's value.
* ``join_nested_loop``: the plain definition of the same result,
  { (l[K], l[V_L - K], r[V_R - K]) : l in L, r in R, l[K] = r[K] }, with
  multiplicities multiplied (bag semantics), by looping over every pair.
* ``scan_pattern``: a triple pattern's partial matches (Section 1, Section 2
  "partial matching"), a linear filter over the triple set.
* ``evaluate_bgp``: pattern-at-a-time evaluation, joining the partial results
  after each pattern is matched (Section 2).
* ``split_by_predicate``: the triple set grouped by predicate, so that a
  pattern with a constant predicate is filtered against that predicate's
  triples only (the same partial matches, a shorter linear filter).
* ``join_star``: the join of k tables that share one variable and no other
  (a star of patterns around it), in one step: for every value of that
  variable, every combination of one row from each table holding it -- the
  key/value framing of Section 1 and Algorithm 1 with k inputs instead of two.
* ``project``: the SELECT clause of a query (Section 1, query Q selects
  ?person): the solutions restricted to the selected variables, duplicates
  kept (SPARQL's default bag semantics).
* ``distinct``: SELECT DISTINCT, each distinct row once.
* ``decode``: dictionary decoding of term ids back to their strings.
* ``brute_force_bgp``: every assignment of the variables over the graph's terms,
  kept when each substituted pattern is a triple of the graph (the SPARQL
  definition of a BGP's solutions).

Readings where the paper is silent: the label test of Algorithm 1 emits each
LEFT x RIGHT pair of a key once and never a same-side pair; ReduceDuplicate is
not a DISTINCT (bag semantics); with two shared variables the key is the pair;
with none the join is the cross product (one key group); the graph is a set of
triples (duplicates dropped before matching); row order is unspecified, so
results are compared as canonically sorted multisets.

A table here is ``(vars, rows)``: a list of variable ids and a uint32 array of
shape (nrows, len(vars)), one row per binding.
"""
from __future__ import annotations

import itertools

import numpy as np

LEFT, RIGHT = 0, 1
VAR_S, VAR_P, VAR_O = 1, 2, 4


def as_rows(t):
    """(vars, rows) from a structure-of-arrays table with ``.vars``/``.cols``/``.nrows``."""
    if isinstance(t, tuple):
        rows = np.asarray(t[1], dtype=np.uint32)
        return list(t[0]), rows.reshape(rows.shape[0], len(t[0]))
    if len(t.vars) == 0:
        return [], np.zeros((t.nrows, 0), dtype=np.uint32)
    return list(t.vars), np.stack([np.asarray(c, dtype=np.uint32) for c in t.cols], axis=1)


def _layout(lvars, rvars):
    """Column layout of the join result: key variables (ascending id), then the
    left table's other variables, then the right table's (Table 1(c))."""
    key = sorted(set(lvars) & set(rvars))
    lk = [lvars.index(v) for v in key]
    rk = [rvars.index(v) for v in key]
    lrest = [c for c, v in enumerate(lvars) if v not in key]
    rrest = [c for c, v in enumerate(rvars) if v not in key]
    out_vars = key + [lvars[c] for c in lrest] + [rvars[c] for c in rrest]
    return key, lk, rk, lrest, rrest, out_vars


def join_nested_loop(L, R):
    """Definition of the join, every pair of rows tested (small inputs only)."""
    lvars, lrows = as_rows(L)
    rvars, rrows = as_rows(R)
    _, lk, rk, lrest, rrest, out_vars = _layout(lvars, rvars)
    out = []
    for l in lrows.tolist():
        for r in rrows.tolist():
            if all(l[a] == r[b] for a, b in zip(lk, rk)):
                out.append([l[a] for a in lk] + [l[c] for c in lrest] + [r[c] for c in rrest])
    return out_vars, np.asarray(out, dtype=np.uint32).reshape(len(out), len(out_vars))


def join_mapreduce(L, R):
    """Algorithm 1: Map, Sort, ReduceDuplicate."""
    lvars, lrows = as_rows(L)
    rvars, rrows = as_rows(R)
    _, lk, rk, lrest, rrest, out_vars = _layout(lvars, rvars)
    nl, nr = lrows.shape[0], rrows.shape[0]

    # Map: every row of Tp1 and Tp2 is split into an intermediate
    # (key, label, value); the value is carried as the row's index in its table.
    key = np.concatenate((lrows[:, lk], rrows[:, rk]), axis=0).astype(np.uint64)
    label = np.concatenate((np.full(nl, LEFT), np.full(nr, RIGHT)))
    value = np.concatenate((np.arange(nl), np.arange(nr)))

    # Sort the intermediates by key (labels kept LEFT before RIGHT inside a key).
    order = np.lexsort([label] + [key[:, c] for c in reversed(range(key.shape[1]))])
    key, label, value = key[order], label[order], value[order]

    # ReduceDuplicate: within each key, every (LEFT value, RIGHT value) pair once.
    n = key.shape[0]
    if n == 0:
        return out_vars, np.zeros((0, len(out_vars)), dtype=np.uint32)
    new_key = np.ones(n, dtype=bool)
    if key.shape[1] > 0:
        new_key[1:] = np.any(key[1:] != key[:-1], axis=1)
    else:
        new_key[1:] = False
    group = np.cumsum(new_key) - 1
    n_groups = int(group[-1]) + 1
    n_left = np.bincount(group, weights=(label == LEFT), minlength=n_groups).astype(np.int64)
    n_right = np.bincount(group, weights=(label == RIGHT), minlength=n_groups).astype(np.int64)
    group_start = np.flatnonzero(new_key)
    # In a group the LEFT intermediates come first, then the RIGHT ones.
    left_pos = np.flatnonzero(label == LEFT)
    pairs_per_left = n_right[group[left_pos]]
    rs_left = np.repeat(left_pos, pairs_per_left)
    first_right = group_start[group[rs_left]] + n_left[group[rs_left]]
    # j-th pair of a LEFT intermediate takes the j-th RIGHT intermediate of its key.
    run_start = np.repeat(np.cumsum(pairs_per_left) - pairs_per_left, pairs_per_left)
    j = np.arange(rs_left.shape[0]) - run_start
    rs_right = first_right + j
    lsel = lrows[value[rs_left]]
    rsel = rrows[value[rs_right]]
    rs = np.concatenate((lsel[:, lk], lsel[:, lrest], rsel[:, rrest]), axis=1)
    return out_vars, rs.astype(np.uint32).reshape(rs_left.shape[0], len(out_vars))


def canonical(t):
    """Columns in ascending variable id, rows sorted lexicographically."""
    vars_, rows = as_rows(t)
    perm = np.argsort(np.asarray(vars_, dtype=np.int64), kind="stable")
    cols = [rows[:, c] for c in perm]
    if rows.shape[0] and cols:
        order = np.lexsort(list(reversed(cols)))
        rows = rows[order][:, perm]
    else:
        rows = rows[:, perm]
    return [vars_[c] for c in perm], np.ascontiguousarray(rows)


def distinct_triples(s, p, o):
    """The graph as a set: triples sorted by (s, p, o), duplicates dropped."""
    s, p, o = (np.asarray(x, dtype=np.uint32) for x in (s, p, o))
    order = np.lexsort((o, p, s))
    s, p, o = s[order], p[order], o[order]
    keep = np.ones(s.shape[0], dtype=bool)
    keep[1:] = (s[1:] != s[:-1]) | (p[1:] != p[:-1]) | (o[1:] != o[:-1])
    return s[keep], p[keep], o[keep]


def scan_pattern(graph, pattern):
    """Partial matches of one triple pattern: a linear filter over the triples.

    ``pattern = (s, p, o, var_mask)``; a field whose var_mask bit is set holds a
    variable id, otherwise a constant term.  Variables appear as columns in the
    order s, p, o; a variable used twice must bind the same term in both places.
    """
    s, p, o = graph
    fields = (s, p, o)
    bits = (VAR_S, VAR_P, VAR_O)
    mask = np.ones(s.shape[0], dtype=bool)
    first_pos = {}
    for f, b, val in zip(fields, bits, pattern[:3]):
        if pattern[3] & b:
            if val in first_pos:
                mask &= f == first_pos[val]
            else:
                first_pos[val] = f
        else:
            mask &= f == np.uint32(val)
    vars_ = list(first_pos.keys())
    n = int(mask.sum())
    if not vars_:
        return [], np.zeros((n, 0), dtype=np.uint32)
    return vars_, np.stack([first_pos[v][mask] for v in vars_], axis=1).astype(np.uint32)


def split_by_predicate(graph):
    """The triple set cut into one triple set per predicate id: ``{p: (s, p, o)}``.

    The same triples, grouped by their predicate, so that a pattern whose
    predicate is a constant can be matched (still by a linear filter) against
    the triples of that predicate only; the partial matches are unchanged."""
    s, p, o = (np.asarray(x, dtype=np.uint32) for x in graph)
    order = np.argsort(p, kind="stable")
    ps = p[order]
    cuts = np.flatnonzero(ps[1:] != ps[:-1]) + 1
    starts = np.concatenate(([0], cuts)).astype(np.int64)
    ends = np.concatenate((cuts, [ps.shape[0]])).astype(np.int64)
    if ps.shape[0] == 0:
        return {}
    return {int(ps[a]): (s[order[a:b]], ps[a:b], o[order[a:b]]) for a, b in zip(starts, ends)}


def _pattern_source(graph, pattern):
    """The triples a pattern is matched against: the whole set, or, for a graph
    split by predicate, the constant predicate's triples (all of them when the
    predicate is a variable)."""
    if not isinstance(graph, dict):
        return graph
    if pattern[3] & VAR_P:
        parts = list(graph.values())
        if not parts:
            return tuple(np.zeros(0, np.uint32) for _ in range(3))
        return tuple(np.concatenate([g[i] for g in parts]) for i in range(3))
    empty = np.zeros(0, np.uint32)
    return graph.get(int(pattern[1]), (empty, empty, empty))


def pattern_vars(pattern):
    return {val for b, val in zip((VAR_S, VAR_P, VAR_O), pattern[:3]) if pattern[3] & b}


def smallest_first_order(bgp, sizes):
    """Start with the pattern with the fewest matches, then repeatedly take the
    pattern with the fewest matches among those sharing a variable with the ones
    already taken (any pattern when none does).  Any order gives the same result;
    this one keeps the partial results small."""
    rest = sorted(range(len(bgp)), key=lambda i: (sizes[i], i))
    order = [rest.pop(0)]
    seen = set(pattern_vars(bgp[order[0]]))
    while rest:
        nxt = next((i for i in rest if pattern_vars(bgp[i]) & seen), rest[0])
        rest.remove(nxt)
        order.append(nxt)
        seen |= pattern_vars(bgp[nxt])
    return order


def evaluate_bgp(graph, bgp, order=None, join=join_mapreduce, is_set=False):
    """Pattern at a time: match each pattern, join the partial results in ``order``.

    ``is_set=True`` states that ``graph`` has no duplicate triples (for instance the
    output of ``distinct_triples``), so the set step is skipped.  ``graph`` may also
    be the output of ``split_by_predicate`` applied to such a set."""
    if isinstance(graph, dict):
        g = graph
    else:
        g = graph if is_set else distinct_triples(*graph)
    partial = [scan_pattern(_pattern_source(g, pat), pat) for pat in bgp]
    if order is None:
        order = smallest_first_order(bgp, [rows.shape[0] for _, rows in partial])
    acc = partial[order[0]]
    for i in order[1:]:
        acc = join(acc, partial[i])
    return acc


def brute_force_bgp(graph, bgp):
    """Every assignment of the BGP's variables over the graph's terms (tiny graphs)."""
    g = distinct_triples(*graph)
    triples = set(zip(*(x.tolist() for x in g)))
    terms = sorted(set(g[0].tolist()) | set(g[1].tolist()) | set(g[2].tolist()))
    vars_ = []
    for pat in bgp:
        for b, val in zip((VAR_S, VAR_P, VAR_O), pat[:3]):
            if pat[3] & b and val not in vars_:
                vars_.append(val)
    rows = []
    for values in itertools.product(terms, repeat=len(vars_)):
        mu = dict(zip(vars_, values))
        ok = True
        for pat in bgp:
            t = tuple(mu[val] if pat[3] & b else val for b, val in zip((VAR_S, VAR_P, VAR_O), pat[:3]))
            if t not in triples:
                ok = False
                break
        if ok:
            rows.append(list(values))
    return vars_, np.asarray(rows, dtype=np.uint32).reshape(len(rows), len(vars_))


def join_batch(pairs, join=join_mapreduce):
    """Independent joins, one after another."""
    return [join(L, R) for (L, R) in pairs]


def project(t, vars_):
    """SELECT ``vars_``: every solution restricted to those variables, in that
    order; the number of rows is unchanged (no duplicate is removed)."""
    tv, rows = as_rows(t)
    cols = [tv.index(v) for v in vars_]
    return list(vars_), np.ascontiguousarray(rows[:, cols]).reshape(rows.shape[0], len(cols))


def distinct(t):
    """SELECT DISTINCT: the table's distinct rows, each once (sorted)."""
    tv, rows = as_rows(t)
    if rows.shape[0] == 0 or rows.shape[1] == 0:
        return tv, rows[: min(rows.shape[0], 1)]
    return tv, np.unique(rows, axis=0)


def decode(ids, terms):
    """The string of each term id: ``terms[i]`` is the term with id i."""
    return [terms[int(i)] for i in ids]


def join_star(tables, key_var):
    """k tables (each with the column ``key_var``; no other variable in two of
    them): for every key value x, every combination (x, rest of a row of table
    1 with key x, ..., rest of a row of table k with key x).  Columns: the key,
    then each table's other columns in table order.  Plain nested products per
    key (small inputs)."""
    tabs = [as_rows(t) for t in tables]
    rest = [[c for c, v in enumerate(tv) if v != key_var] for tv, _ in tabs]
    others = [v for (tv, _), rc in zip(tabs, rest) for v in (tv[c] for c in rc)]
    assert len(others) == len(set(others)) and key_var not in others, "tables share more than the key"
    out_vars = [key_var] + others
    groups = []
    for (tv, rows), rc in zip(tabs, rest):
        kc = tv.index(key_var)
        g = {}
        for r in rows.tolist():
            g.setdefault(r[kc], []).append([r[c] for c in rc])
        groups.append(g)
    out = []
    for x in sorted(set.intersection(*[set(g) for g in groups])) if groups else []:
        for combo in itertools.product(*[g[x] for g in groups]):
            out.append([x] + [v for part in combo for v in part])
    return out_vars, np.asarray(out, dtype=np.uint32).reshape(len(out), len(out_vars))
