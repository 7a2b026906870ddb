"""Pins of the CPU oracle to facts that do not come from the oracle itself:
the paper's worked example (Table 1), brute-force enumeration, the cardinality
identity, closed forms of the synthetic workloads and special cases.  The last
test plants mistakes in copies of the oracle and checks that the pins catch them."""
import itertools
from collections import Counter

import numpy as np
import pytest

import gen
import oracle
from gen.bgp import GraphIndex, generate_bgps
from oracle import mapsq_oracle as om
from golden_example import Dictionary, load

JOINS = [oracle.join_mapreduce, oracle.join_nested_loop]


def multiset(t):
    vars_, rows = oracle.canonical(t)
    return vars_, [tuple(r) for r in rows.tolist()]


# ---------------------------------------------------------------- worked example

def table1_tables():
    g = load()
    d = Dictionary()
    tp1 = gen.Table([0, 1], [np.array([d.id(r[0]) for r in g["Tp1"]], np.uint32),
                             np.array([d.id(r[1]) for r in g["Tp1"]], np.uint32)])
    tp2 = gen.Table([0, 2], [np.array([d.id(r[0]) for r in g["Tp2"]], np.uint32),
                             np.array([d.id(r[1]) for r in g["Tp2"]], np.uint32)])
    return g, d, tp1, tp2


def check_table1(join):
    g, d, tp1, tp2 = table1_tables()
    vars_, rows = join(tp1, tp2)
    got = sorted(tuple(d.term(x) for x in r) for r in rows.tolist())
    return vars_ == [0, 1, 2] and got == sorted(tuple(r) for r in g["RS"])


@pytest.mark.parametrize("join", JOINS)
def test_table1_rs_exact(join):
    """Tp1 joined with Tp2 on ?job gives exactly RS, columns Key, Value1, Value2."""
    assert check_table1(join)


def table1_query():
    g = load()
    d = Dictionary()
    s, p, o = (np.array([d.id(t[i]) for t in g["GRAPH"]], np.uint32) for i in range(3))
    var_ids = {}
    bgp = []
    for pat in g["BGP"]:
        f, mask = [], 0
        for bit, term in zip((1, 2, 4), pat):
            if term.startswith("?"):
                f.append(var_ids.setdefault(term, len(var_ids)))
                mask |= bit
            else:
                f.append(d.id(term))
        bgp.append((f[0], f[1], f[2], mask))
    header = [k for k in g if k.startswith("SOLUTIONS")][0].split()[1:]
    expected = sorted(tuple(r) for r in g[[k for k in g if k.startswith("SOLUTIONS")][0]])
    return (s, p, o), bgp, d, var_ids, header, expected


def test_table1_as_query():
    graph, bgp, d, var_ids, header, expected = table1_query()
    for order in itertools.permutations(range(len(bgp))):
        vars_, rows = oracle.evaluate_bgp(graph, bgp, order=order)
        pos = [vars_.index(var_ids[h]) for h in header]
        got = sorted(tuple(d.term(r[c]) for c in pos) for r in rows.tolist())
        assert got == expected
    vars_, rows = oracle.brute_force_bgp(graph, bgp)
    pos = [vars_.index(var_ids[h]) for h in header]
    assert sorted(tuple(d.term(r[c]) for c in pos) for r in rows.tolist()) == expected


def test_query_q_select_person():
    """Query Q of Section 1 selects ?person: the answer is exactly Jim and Susan
    (the golden [SELECT ?person] section), with or without DISTINCT, decoded
    through the dictionary."""
    graph, bgp, d, var_ids, header, expected = table1_query()
    g = load()
    want = sorted(r[0] for r in g["SELECT ?person"])
    assert want == ["Jim", "Susan"]
    sol = oracle.evaluate_bgp(graph, bgp)
    for t in (oracle.project(sol, [var_ids["?person"]]), oracle.distinct(oracle.project(sol, [var_ids["?person"]]))):
        vars_, rows = t
        assert vars_ == [var_ids["?person"]]
        assert sorted(oracle.decode(rows[:, 0], d.terms)) == want


def test_project_and_distinct_match_brute_force():
    """Projection keeps every solution (multiplicities counted independently with
    Counter over brute-force assignments); DISTINCT keeps each projected row once
    (a Python set); on tiny graphs, including projections that create duplicates."""
    for seed in range(40):
        graph = tiny_graph(seed + 500, n_terms=7, n_triples=30)
        bgp = tiny_bgp(seed + 500, n_terms=7)
        bv, brows = oracle.brute_force_bgp(graph, bgp)
        if not bv:
            continue
        r = gen.Rng(seed, 21)
        k = int(r.between(1, 1, len(bv))[0])
        sel = [bv[int(i)] for i in r.permutation(len(bv))[:k]]
        want = Counter(tuple(row[bv.index(v)] for v in sel) for row in brows.tolist())
        pv, prow = oracle.project(oracle.evaluate_bgp(graph, bgp), sel)
        assert pv == sel and Counter(map(tuple, prow.tolist())) == want, (seed, bgp, sel)
        dv, drow = oracle.distinct((pv, prow))
        assert dv == sel and sorted(map(tuple, drow.tolist())) == sorted(want), (seed, bgp, sel)
    # a projection with duplicates: ?x has three ?y
    rows = np.array([[1, 10], [1, 11], [1, 12], [2, 10]], np.uint32)
    assert Counter(map(tuple, oracle.project(([0, 1], rows), [0])[1].tolist())) == Counter({(1,): 3, (2,): 1})
    assert oracle.distinct(oracle.project(([0, 1], rows), [0]))[1].tolist() == [[1], [2]]


def star_tables(seed, k, n_max=30, dom=6):
    """k random tables sharing variable 0 and nothing else."""
    r = gen.Rng(seed, 31)
    tabs, nxt = [], 1
    for _ in range(k):
        extra = int(r.between(1, 0, 2)[0])
        vars_ = [0] + list(range(nxt, nxt + extra))
        nxt += extra
        perm = r.permutation(len(vars_))
        vars_ = [vars_[i] for i in perm]
        tabs.append(gen.random_table(r, int(r.between(1, 0, n_max)[0]), vars_, dom))
    return tabs


def test_star_join_matches_pairwise_joins_and_histograms():
    """The k-way star join equals k - 1 pairwise joins (Algorithm 1) in order,
    and its row count is the sum over keys of the product of the tables' key
    counts, from independent Counter histograms."""
    for seed in range(60):
        k = 2 + seed % 5
        tabs = star_tables(seed, k)
        got = oracle.join_star(tabs, 0)
        acc = tabs[0]
        for t in tabs[1:]:
            acc = oracle.join_nested_loop(acc, t)
        assert multiset(got) == multiset(acc), seed
        hist = [Counter(t.cols[t.vars.index(0)].tolist()) for t in tabs]
        keys = set(hist[0]).intersection(*hist[1:])
        assert got[1].shape[0] == sum(int(np.prod([h[x] for h in hist])) for x in keys)


def test_star_bgp_equals_brute_force():
    """A star BGP (every pattern on one centre variable, no other variable
    shared) evaluated by one star join of its partial matches equals brute
    force."""
    done = 0
    for seed in range(200):
        graph = tiny_graph(seed + 900, n_terms=6, n_triples=30, n_pred=3)
        r = gen.Rng(seed, 41)
        k = int(r.between(1, 2, 4)[0])
        bgp, nxt = [], 1
        for _ in range(k):
            if r.below(1, 2)[0]:
                bgp.append((0, int(r.below(1, 3)[0]), nxt, 5)); nxt += 1   # ?x p ?y
            else:
                bgp.append((nxt, int(r.below(1, 3)[0]), 0, 5)); nxt += 1   # ?y p ?x
        g = oracle.distinct_triples(*graph)
        parts = [oracle.scan_pattern(g, pat) for pat in bgp]
        got = oracle.join_star(parts, 0)
        want = oracle.brute_force_bgp(graph, bgp)
        assert multiset(got) == multiset(want), (seed, bgp)
        done += got[1].shape[0] > 0
    assert done > 20


# ---------------------------------------------------------------- pairwise join

def key_histogram_count(L, R):
    """|L join R| = sum over keys of |L_k| * |R_k|, from independent histograms."""
    shared = sorted(set(L.vars) & set(R.vars))
    lk = list(zip(*[L.cols[L.vars.index(v)].tolist() for v in shared])) if shared else [()] * L.nrows
    rk = list(zip(*[R.cols[R.vars.index(v)].tolist() for v in shared])) if shared else [()] * R.nrows
    cl, cr = Counter(lk), Counter(rk)
    return sum(n * cr[k] for k, n in cl.items())


def random_pair(seed, n_shared):
    r = gen.Rng(seed, 7)
    nl, nr = (int(x) for x in r.between(2, 0, 60))
    dom = int(r.between(1, 1, 12)[0])
    lv = list(range(n_shared)) + [10 + i for i in range(int(r.between(1, 0, 2)[0]))]
    rv = list(range(n_shared)) + [20 + i for i in range(int(r.between(1, 0, 2)[0]))]
    if not lv:
        lv = [10]
    if not rv:
        rv = [20]
    # shuffle column order so keys are not always in front
    lv = [lv[i] for i in r.permutation(len(lv))]
    rv = [rv[i] for i in r.permutation(len(rv))]
    return gen.random_table(r, nl, lv, dom), gen.random_table(r, nr, rv, dom)


@pytest.mark.parametrize("n_shared", [0, 1, 2, 3])
def test_join_matches_definition(n_shared):
    for seed in range(40):
        L, R = random_pair(seed * 4 + n_shared, n_shared)
        a = multiset(oracle.join_mapreduce(L, R))
        b = multiset(oracle.join_nested_loop(L, R))
        assert a == b
        assert len(a[1]) == key_histogram_count(L, R)


def test_join_layout_key_left_right():
    L = gen.Table([5, 3], [np.array([7, 8], np.uint32), np.array([1, 2], np.uint32)])
    R = gen.Table([9, 5], [np.array([100, 200, 300], np.uint32), np.array([8, 7, 8], np.uint32)])
    for join in JOINS:
        vars_, rows = join(L, R)
        assert vars_ == [5, 3, 9]
        assert sorted(map(tuple, rows.tolist())) == [(7, 1, 200), (8, 2, 100), (8, 2, 300)]


@pytest.mark.parametrize("join", JOINS)
def test_join_special_cases(join):
    r = gen.Rng(11)
    # one key: the full cross product of the value columns
    L = gen.Table([0, 1], [np.full(7, 4, np.uint32), r.u32(7)])
    R = gen.Table([0, 2], [np.full(5, 4, np.uint32), r.u32(5)])
    _, rows = join(L, R)
    want = sorted((4, a, b) for a, b in itertools.product(L.cols[1].tolist(), R.cols[1].tolist()))
    assert sorted(map(tuple, rows.tolist())) == want
    # disjoint keys: empty
    R2 = gen.Table([0, 2], [np.full(5, 5, np.uint32), r.u32(5)])
    assert join(L, R2)[1].shape == (0, 3)
    # right side holds each key once: a lookup, one row per matching left row
    keys = r.below(50, 20).astype(np.uint32)
    L3 = gen.Table([0, 1], [keys, np.arange(50, dtype=np.uint32)])
    R3 = gen.Table([0, 2], [np.arange(10, dtype=np.uint32), np.arange(10, dtype=np.uint32) * 3])
    _, rows = join(L3, R3)
    assert sorted(map(tuple, rows.tolist())) == sorted(
        (int(k), i, int(k) * 3) for i, k in enumerate(keys.tolist()) if k < 10)
    # extreme ids 0 and 0xFFFFFFFF are ordinary data
    big = np.uint32(0xFFFFFFFF)
    L4 = gen.Table([0, 1], [np.array([0, big, big], np.uint32), np.array([1, 2, 3], np.uint32)])
    R4 = gen.Table([0, 2], [np.array([big, 0], np.uint32), np.array([9, 8], np.uint32)])
    assert sorted(map(tuple, join(L4, R4)[1].tolist())) == [(0, 1, 8), (0xFFFFFFFF, 2, 9), (0xFFFFFFFF, 3, 9)]
    # bag semantics: duplicate rows multiply
    L5 = gen.Table([0, 1], [np.array([1, 1], np.uint32), np.array([6, 6], np.uint32)])
    R5 = gen.Table([0, 2], [np.array([1, 1, 1], np.uint32), np.array([2, 2, 2], np.uint32)])
    assert join(L5, R5)[1].tolist() == [[1, 6, 2]] * 6
    # empty side
    L6 = gen.Table([0, 1], [np.zeros(0, np.uint32), np.zeros(0, np.uint32)])
    assert join(L6, R5)[1].shape == (0, 3)
    assert join(R5, L6)[1].shape == (0, 3)
    # no shared variable: cross product
    R7 = gen.Table([3], [np.array([5, 6, 7], np.uint32)])
    assert join(L5, R7)[1].shape == (6, 3)
    # zero-column unit table is the identity of the join
    unit = gen.Table.unit(1)
    assert sorted(map(tuple, join(L3, unit)[1].tolist())) == sorted(map(tuple, oracle.as_rows(L3)[1].tolist()))
    assert join(L3, gen.Table.unit(0))[1].shape == (0, 2)
    assert join(unit, unit)[1].shape == (1, 0)
    assert join(unit, gen.Table.unit(0))[1].shape == (0, 0)


def test_skewed_two_key_closed_form():
    """Every A row meets exactly ``reps`` B rows, so the join has reps * |A| rows."""
    A, B = gen.skewed_two_key(seed=3, log_a=13, log_b=11, log_keys=9, reps=4)
    vars_, rows = oracle.join_mapreduce(A, B)
    assert rows.shape == (4 << 13, 6)
    assert vars_ == [0, 1, 2, 3, 4, 5]
    assert rows.shape[0] == key_histogram_count(A, B)
    # the two key columns are a bijective image of the key id
    ids = np.unique(np.stack(A.cols[:2], 1), axis=0)
    assert ids.shape[0] <= 1 << 9


def test_uneven_batch_counts():
    batch = gen.uneven_batch(seed=4, n_joins=6, log_lo=6.0, log_hi=10.0)
    for L, R, s in batch:
        assert s in (0.0, 0.8, 1.2)
        vars_, rows = oracle.join_mapreduce(L, R)
        assert rows.shape[0] == key_histogram_count(L, R)
        assert multiset(oracle.join_mapreduce(L, R)) == multiset((vars_, rows))


def test_pairwise_uniform_expected_size():
    L, R = gen.pairwise_uniform(seed=1)
    n = oracle.join_mapreduce(L, R)[1].shape[0]
    assert n == key_histogram_count(L, R)
    # E[T] = 16384 * 8192 / 4096 = 32768; the seeded draw lies within a few sigma
    assert abs(n - 32768) < 2000


# ---------------------------------------------------------------- BGPs

def tiny_graph(seed, n_terms=10, n_triples=24, n_pred=3):
    r = gen.Rng(seed, 9)
    s = r.below(n_triples, n_terms).astype(np.uint32)
    p = r.below(n_triples, n_pred).astype(np.uint32)
    o = r.below(n_triples, n_terms).astype(np.uint32)
    return s, p, o


def tiny_bgp(seed, n_terms=10, n_pred=3, max_vars=4):
    r = gen.Rng(seed, 13)
    k = int(r.between(1, 1, 4)[0])
    bgp = []
    for _ in range(k):
        f = []
        mask = 0
        for bit in (1, 4):
            if r.below(1, 4)[0] > 0:
                f.append(int(r.below(1, max_vars)[0]))
                mask |= bit
            else:
                f.append(int(r.below(1, n_terms)[0]))
        bgp.append((f[0], int(r.below(1, n_pred)[0]), f[1], mask))
    return bgp


def test_patterns_without_variables_brute_force():
    """A pattern with no variable holds under every assignment or under none:
    present, the BGP's solutions are those of the other patterns; absent,
    there are none (with every variable of the BGP); alone, one row without
    columns or none.  Checked against brute-force enumeration."""
    for seed in range(40):
        graph = tiny_graph(seed)
        s, p, o = graph
        here = (int(s[0]), int(p[0]), int(o[0]), 0)
        triples = set(zip(s.tolist(), p.tolist(), o.tolist()))
        gone = next((a, int(p[0]), b, 0) for a in range(12) for b in range(12) if (a, int(p[0]), b) not in triples)
        rest = [tp for tp in tiny_bgp(seed) if tp[3]] or [(0, int(p[1]), 1, 5)]
        base = multiset(oracle.brute_force_bgp(graph, rest))
        assert multiset(oracle.brute_force_bgp(graph, rest + [here])) == base
        none = multiset(oracle.brute_force_bgp(graph, [gone] + rest))
        assert none == (base[0], [])
        assert multiset(oracle.brute_force_bgp(graph, [here])) == ([], [()])
        assert multiset(oracle.brute_force_bgp(graph, [here, gone])) == ([], [])
        for bgp in (rest + [here], [gone] + rest, [here], [here, gone]):
            want = multiset(oracle.brute_force_bgp(graph, bgp))
            for join in JOINS:
                assert multiset(oracle.evaluate_bgp(graph, bgp, join=join)) == want, (seed, bgp)


def test_bgp_matches_brute_force():
    for seed in range(60):
        graph = tiny_graph(seed)
        bgp = tiny_bgp(seed)
        want = multiset(oracle.brute_force_bgp(graph, bgp))
        for join in JOINS:
            assert multiset(oracle.evaluate_bgp(graph, bgp, join=join)) == want, (seed, bgp)


def test_bgp_join_order_invariance_and_no_duplicates():
    for seed in range(30):
        graph = tiny_graph(seed + 100, n_terms=8, n_triples=30)
        bgp = tiny_bgp(seed + 100, n_terms=8)
        ref = multiset(oracle.evaluate_bgp(graph, bgp))
        assert len(set(ref[1])) == len(ref[1])
        for order in itertools.permutations(range(len(bgp))):
            assert multiset(oracle.evaluate_bgp(graph, bgp, order=order)) == ref


def test_bgp_on_graph_split_by_predicate():
    """Matching each pattern against its predicate's triples only (the graph
    split by predicate) gives the same solutions as the whole triple set and as
    brute force, variable predicates included."""
    for seed in range(40):
        graph = tiny_graph(seed + 300, n_terms=9, n_triples=28, n_pred=4)
        g = oracle.distinct_triples(*graph)
        split = oracle.split_by_predicate(g)
        assert sum(v[0].shape[0] for v in split.values()) == g[0].shape[0]
        assert all(np.all(v[1] == k) for k, v in split.items())
        bgp = tiny_bgp(seed + 300, n_terms=9, n_pred=5)  # predicate 4 has no triples
        if seed % 5 == 0:
            s, p, o, m = bgp[0]
            bgp[0] = (s, 3, o, m | 2)  # a variable predicate (id 3)
        want = multiset(oracle.brute_force_bgp(graph, bgp))
        assert multiset(oracle.evaluate_bgp(split, bgp)) == want, (seed, bgp)
        assert multiset(oracle.evaluate_bgp(g, bgp, is_set=True)) == want


def test_bgp_variable_repeated_in_pattern():
    s = np.array([1, 2, 3, 3], np.uint32)
    p = np.array([0, 0, 0, 1], np.uint32)
    o = np.array([1, 5, 3, 3], np.uint32)
    bgp = [(0, 0, 0, 5)]  # ?x p0 ?x
    assert multiset(oracle.evaluate_bgp((s, p, o), bgp)) == ([0], [(1,), (3,)])
    assert multiset(oracle.brute_force_bgp((s, p, o), bgp)) == ([0], [(1,), (3,)])


def test_bgp_duplicate_triples_are_one():
    s = np.array([1, 1, 1], np.uint32)
    p = np.array([0, 0, 0], np.uint32)
    o = np.array([2, 2, 3], np.uint32)
    assert multiset(oracle.evaluate_bgp((s, p, o), [(0, 0, 1, 5)])) == ([0, 1], [(1, 2), (1, 3)])


def test_generated_bgps_contain_their_witness():
    s, p, o = gen.university_graph(200_000, seed=2)
    g = GraphIndex(s, p, o)
    G = oracle.distinct_triples(s, p, o)
    assert G[0].shape[0] == 200_000  # the generator makes a set
    for b in generate_bgps(g, 12, seed=5):
        vars_, rows = oracle.evaluate_bgp(G, b["patterns"], is_set=True)
        assert 2 <= len(vars_) <= 5
        w = np.array([b["witness"][v] for v in vars_], np.uint32)
        assert (rows == w).all(axis=1).any()
        assert rows.shape[0] <= b["bound"]
        assert len({tuple(r) for r in rows.tolist()}) == rows.shape[0]


# ---------------------------------------------------------------- planted mistakes

def _mutants():
    def swapped_values(L, R):
        vars_, rows = oracle.join_mapreduce(L, R)
        return vars_, rows[:, [0, 2, 1]] if rows.shape[1] == 3 else rows

    def drops_last_pair(L, R):
        vars_, rows = oracle.join_mapreduce(L, R)
        return vars_, rows[:-1]

    def same_side_pairs(L, R):
        # also pairs LEFT with LEFT, as a label test that was left out would
        vars_, rows = oracle.join_mapreduce(L, R)
        extra = oracle.join_mapreduce(L, gen.Table(R.vars, [L.cols[L.vars.index(v)] if v in L.vars
                                                               else L.cols[-1] for v in R.vars])
                                      if hasattr(R, "cols") else R)[1]
        return vars_, np.concatenate((rows, extra)) if extra.shape[1] == rows.shape[1] else rows

    def first_key_only(L, R):
        # joins on one shared variable when there are two
        lvars, lrows = oracle.as_rows(L)
        rvars, rrows = oracle.as_rows(R)
        shared = sorted(set(lvars) & set(rvars))
        if len(shared) < 2:
            return oracle.join_mapreduce(L, R)
        drop = shared[1]
        R2 = (["d"] + [v for v in rvars if v != drop],
              np.concatenate((rrows[:, [rvars.index(drop)]], rrows[:, [c for c, v in enumerate(rvars) if v != drop]]), 1))
        vars_, rows = oracle.join_mapreduce((lvars, lrows), R2)
        keep = [i for i, v in enumerate(vars_) if v != "d"]
        return [vars_[i] for i in keep], rows[:, keep]

    return [swapped_values, drops_last_pair, same_side_pairs, first_key_only]


def _pins_pass(join):
    if not check_table1(join):
        return False
    for n_shared in (1, 2):
        for seed in range(20):
            L, R = random_pair(seed * 4 + n_shared, n_shared)
            try:
                got = multiset(join(L, R))
            except Exception:
                return False
            if len(got[1]) != key_histogram_count(L, R):
                return False
            if got != multiset(oracle.join_nested_loop(L, R)):
                return False
    return True


def test_pins_reject_planted_mistakes():
    assert _pins_pass(oracle.join_mapreduce)
    for m in _mutants():
        assert not _pins_pass(m), m.__name__


def test_generators_are_deterministic():
    a = gen.university_graph(50_000, seed=2)
    b = gen.university_graph(50_000, seed=2)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    A1, B1 = gen.skewed_two_key(seed=3, log_a=10, log_b=8, log_keys=6)
    A2, B2 = gen.skewed_two_key(seed=3, log_a=10, log_b=8, log_keys=6)
    assert all(np.array_equal(x, y) for x, y in zip(A1.cols + B1.cols, A2.cols + B2.cols))
    assert om.LEFT != om.RIGHT
