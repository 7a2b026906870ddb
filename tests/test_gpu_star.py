"""The multi-way star join on the GPU through the C ABI (mapsq_join_star, and
mapsq_query on star BGPs) against the oracle's join_star and evaluate_bgp."""
import numpy as np
import pytest

import gen
import oracle
from gpu_helpers import assert_same_multiset

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1702_03484_gb300 import Context
    with Context(device=0) as c:
        yield c


def _view(t, sort_key):
    """A caller-described device table (columns kept alive on the view),
    sorted on variable 0 and marked so when ``sort_key``."""
    import torch
    from paper_1702_03484_gb300 import mapsq
    cols = [np.ascontiguousarray(c) for c in t.cols]
    kc = t.vars.index(0)
    if sort_key:
        order = np.argsort(cols[kc], kind="stable")
        cols = [c[order] for c in cols]
    dev = [torch.from_numpy(c).cuda() for c in cols]
    v = mapsq.table_view(t.vars, dev, t.nrows, sorted_cols=(kc,) if sort_key else ())
    v._keep = dev
    return v, gen.Table(list(t.vars), cols)


def _check(ctx, tabs, unsorted=(), what=""):
    from paper_1702_03484_gb300 import TableRef, mapsq
    views, host = zip(*[_view(t, i not in unsorted) for i, t in enumerate(tabs)])
    res = TableRef(ctx, mapsq.mapsq_join_star(ctx.handle, list(views), 0))
    try:
        assert_same_multiset(res, oracle.join_star(list(host), 0), what)
        return res.nrows
    finally:
        res.free()


def _star(seed, k, n, dom, extra=(0, 2)):
    r = gen.Rng(seed, 51)
    tabs, nxt = [], 1
    for _ in range(k):
        e = int(r.between(1, *extra)[0])
        vars_ = [0] + list(range(nxt, nxt + e))
        nxt += e
        vars_ = [vars_[i] for i in r.permutation(len(vars_))]
        tabs.append(gen.random_table(r, int(r.between(1, 1, n)[0]), vars_, dom))
    return tabs


def test_random_stars(ctx):
    for seed in range(24):
        k = 2 + seed % 7
        tabs = _star(seed, k, n=3000, dom=600)
        _check(ctx, tabs, what=f"seed {seed} k {k}")
        _check(ctx, tabs, unsorted=(seed % k,), what=f"seed {seed} k {k}, one table unsorted (it drives)")


def test_unsorted_tables_fall_back_to_pairwise(ctx):
    tabs = _star(99, 4, n=2000, dom=300)
    assert _check(ctx, tabs, unsorted=(0, 2), what="two unsorted tables") > 0


def test_hot_key_large_product_and_key_only_tables(ctx):
    """One key with 100 x 100 x 100 rows (a million output rows for it), and
    tables holding only the key column (their multiplicity multiplies)."""
    r = gen.Rng(52)
    def table(vars_, n, hot):
        key = np.concatenate((np.full(hot, 7, np.uint32), r.below(n, 5000).astype(np.uint32)))
        return gen.Table(vars_, [key] + [r.u32(key.shape[0]) for _ in vars_[1:]])
    tabs = [table([0, 1], 4000, 100), table([0, 2], 3000, 100), table([0, 3, 4], 5000, 100)]
    assert _check(ctx, tabs, what="hot key") >= 100 ** 3
    only = [table([0], 300, 3), table([0, 5], 2000, 2), table([0], 400, 4)]
    _check(ctx, only, what="key-only tables")


def test_large_stars_search_by_bisection(ctx):
    """Driving tables of more than 152 CTAs' rows (the count and write bisect
    instead of searching K-ary) give the oracle's rows."""
    r = gen.Rng(54)
    for k in (2, 4):
        tabs = [gen.Table([0, j + 1], [r.below(60_000 + 7000 * j, 50_000).astype(np.uint32),
                                       r.u32(60_000 + 7000 * j)]) for j in range(k)]
        tabs[1].cols[0][:3] = [0, 0xFFFFFFFF, 0xFFFFFFFF]
        assert _check(ctx, tabs, what=f"large star k {k}") > 0


def test_empty_table_and_errors(ctx):
    from paper_1702_03484_gb300 import mapsq
    from paper_1702_03484_gb300.mapsq import MapsqError
    tabs = _star(7, 3, n=500, dom=100)
    tabs[1] = gen.Table(tabs[1].vars, [c[:0] for c in tabs[1].cols])
    assert _check(ctx, tabs, what="an empty table") == 0
    r = gen.Rng(53)
    a = gen.Table([0, 1], [r.below(50, 10).astype(np.uint32), r.u32(50)])
    b = gen.Table([0, 1], [r.below(50, 10).astype(np.uint32), r.u32(50)])  # shares variable 1 too
    views = [_view(a, True)[0], _view(b, True)[0]]
    with pytest.raises(MapsqError) as e:
        mapsq.mapsq_join_star(ctx.handle, views, 0)
    assert e.value.name == "INVALID"
    with pytest.raises(MapsqError) as e:
        mapsq.mapsq_join_star(ctx.handle, views, 3)  # no table holds variable 3
    assert e.value.name == "INVALID"


def test_star_bgps_through_query(ctx):
    """Generated star BGPs over a small university graph go through the star
    path of mapsq_query and equal the oracle's pattern-at-a-time evaluation."""
    from gen.bgp import GraphIndex, generate_bgps
    s, p, o = gen.university_graph(40_000, seed=2)
    ctx.load_triples(s, p, o)
    G = oracle.distinct_triples(s, p, o)
    n = 0
    for b in generate_bgps(GraphIndex(s, p, o), 24, seed=9):
        if b.get("shape") not in (None, "star"):
            continue
        res = ctx.query(b["patterns"])
        assert_same_multiset(res, oracle.evaluate_bgp(G, b["patterns"], is_set=True), str(b["patterns"]))
        n += res.nrows > 0
        res.free()
    assert n > 0
