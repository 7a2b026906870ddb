"""SELECT on the GPU through the C ABI: projection (bag), DISTINCT and
dictionary decode against the oracle's project / distinct / decode."""
import numpy as np
import pytest

import gen
import oracle
from golden_example import Dictionary, load
from gpu_helpers import assert_same_multiset, device_table

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1702_03484_gb300 import Context
    with Context(device=0) as c:
        yield c


def test_query_q_selects_jim_and_susan(ctx):
    """Query Q of Section 1 on the graph of Table 1: SELECT ?person gives
    exactly Jim and Susan, decoded through the device dictionary."""
    g = load()
    d = Dictionary()
    s, p, o = (np.array([d.id(t[i]) for t in g["GRAPH"]], np.uint32) for i in range(3))
    var = {}
    bgp = []
    for pat in g["BGP"]:
        f, mask = [], 0
        for bit, term in zip((1, 2, 4), pat):
            if term.startswith("?"):
                f.append(var.setdefault(term, len(var)))
                mask |= bit
            else:
                f.append(d.id(term))
        bgp.append((f[0], f[1], f[2], mask))
    ctx.load_triples(s, p, o)
    ctx.dict_load(d.terms)
    want = sorted(r[0] for r in g["SELECT ?person"])
    for distinct in (False, True):
        res = ctx.query(bgp, select=[var["?person"]], distinct=distinct)
        assert res.vars == [var["?person"]]
        assert sorted(res.decode(0)) == want
        res.free()


def test_project_and_distinct_on_generated_bgps(ctx):
    """Random selections of the variables of generated BGPs over a small
    university graph, with and without DISTINCT, against the oracle."""
    from gen.bgp import GraphIndex, generate_bgps
    s, p, o = gen.university_graph(30_000, seed=2)
    ctx.load_triples(s, p, o)
    G = oracle.distinct_triples(s, p, o)
    r = gen.Rng(33)
    for b in generate_bgps(GraphIndex(s, p, o), 10, seed=7):
        bgp = b["patterns"]
        full = oracle.evaluate_bgp(G, bgp, is_set=True)
        vars_ = full[0]
        k = int(r.between(1, 1, len(vars_))[0])
        sel = [vars_[int(i)] for i in r.permutation(len(vars_))[:k]]
        for distinct in (False, True):
            want = oracle.project(full, sel)
            if distinct:
                want = oracle.distinct(want)
            res = ctx.query(bgp, select=sel, distinct=distinct)
            assert res.vars == sel
            assert_same_multiset(res, want, f"{bgp} select {sel} distinct={distinct}")
            res.free()


def test_distinct_large_with_duplicates(ctx):
    """DISTINCT over 2^20 rows of three columns drawn from small domains (many
    duplicates), one column and all three, and the same table projected
    without DISTINCT keeps every row."""
    r = gen.Rng(34)
    n = 1 << 20
    T = gen.Table([3, 5, 7], [r.below(n, 50).astype(np.uint32), r.below(n, 40).astype(np.uint32),
                              r.below(n, 3).astype(np.uint32)])
    t = device_table(ctx, T)
    for sel in ([5], [7, 3], [3, 5, 7]):
        res = ctx.project(t, sel, distinct=True)
        assert_same_multiset(res, oracle.distinct(oracle.project(T, sel)), f"distinct {sel}")
        res.free()
    res = ctx.project(t, [7, 3])
    assert res.nrows == n
    assert_same_multiset(res, oracle.project(T, [7, 3]), "bag projection")
    res.free()
    t.free()


def test_select_edge_cases(ctx):
    from paper_1702_03484_gb300.mapsq import MapsqError
    r = gen.Rng(35)
    E = gen.Table([0, 1], [np.zeros(0, np.uint32), np.zeros(0, np.uint32)])
    te = device_table(ctx, E)
    for distinct in (False, True):
        res = ctx.project(te, [1], distinct=distinct)
        assert res.nrows == 0 and res.vars == [1]
        res.free()
    one = device_table(ctx, gen.Table([0, 1], [np.array([7], np.uint32), np.array([9], np.uint32)]))
    res = ctx.project(one, [1, 0], distinct=True)
    assert_same_multiset(res, ([1, 0], np.array([[9, 7]], np.uint32)), "one row")
    res.free()
    for bad in ([], [2], [0, 0]):
        with pytest.raises(MapsqError) as e:
            ctx.project(one, bad)
        assert e.value.name == "INVALID"
    # decode: an id without a term
    ctx.dict_load(["a", "bb", ""])
    ok = device_table(ctx, gen.Table([0], [np.array([1, 0, 2, 1], np.uint32)]))
    assert ok.decode(0) == ["bb", "a", "", "bb"]
    with pytest.raises(MapsqError) as e:
        one.decode(0)
    assert e.value.name == "INVALID"
    for x in (te, one, ok):
        x.free()
