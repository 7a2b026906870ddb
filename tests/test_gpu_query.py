"""GPU parity of the triple store, mapsq_scan_pattern and mapsq_query against
the CPU oracle (bit-exact multisets)."""
import itertools

import numpy as np
import pytest

import gen
import oracle
from gen.bgp import GraphIndex, generate_bgps
from gpu_helpers import assert_same_multiset, host_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_1702_03484_gb300 import Context
    assert torch.cuda.is_available()
    c = Context(device=0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def small_graph():
    return gen.university_graph(150_000, seed=2)


def test_load_dedups_and_counts(ctx):
    r = gen.Rng(3)
    s = r.below(5000, 50).astype(np.uint32)
    p = r.below(5000, 4).astype(np.uint32)
    o = r.below(5000, 50).astype(np.uint32)
    s = np.concatenate((s, s[:700]))
    p = np.concatenate((p, p[:700]))
    o = np.concatenate((o, o[:700]))
    ctx.load_triples(s, p, o)
    n, k = ctx.store_info()
    g = oracle.distinct_triples(s, p, o)
    assert n == g[0].shape[0]
    assert k == np.unique(p).shape[0]


def test_load_from_device_pointers(ctx, small_graph):
    import torch
    s, p, o = small_graph
    ctx.load_triples(*(torch.from_numpy(x).cuda() for x in (s, p, o)))
    assert ctx.store_info()[0] == oracle.distinct_triples(s, p, o)[0].shape[0]


def test_scan_every_pattern_kind(ctx, small_graph):
    s, p, o = small_graph
    ctx.load_triples(s, p, o)
    G = oracle.distinct_triples(s, p, o)
    r = gen.Rng(17)
    idx = r.below(40, s.shape[0])
    pats = []
    for i in idx.tolist():
        ss, pp, oo = int(s[i]), int(p[i]), int(o[i])
        pats += [(ss, pp, 0, 4), (0, pp, oo, 1), (0, pp, 1, 5), (ss, pp, oo, 0), (ss + 1, pp, oo, 0)]
    pats += [(0, 99, 1, 5), (5, 99, 1, 4), (0, 3, 0, 5), (0, 6, 0, 5)]
    for tp in pats:
        t = ctx.scan_pattern(tp)
        assert_same_multiset(t, oracle.scan_pattern(G, tp), f"scan {tp}")
        t.free()


def test_scan_results_outlive_a_store_reload(ctx, small_graph):
    """Scan results may alias the store; replacing the store must not change them."""
    s, p, o = small_graph
    ctx.load_triples(s, p, o)
    G = oracle.distinct_triples(s, p, o)
    pats = [(0, 6, 1, 5), (0, 0, 3, 1), (int(s[7]), int(p[7]), 0, 4)]
    held = [(tp, ctx.scan_pattern(tp)) for tp in pats]
    r = gen.Rng(4)
    ctx.load_triples(r.below(1000, 30).astype(np.uint32), r.below(1000, 3).astype(np.uint32),
                     r.below(1000, 30).astype(np.uint32))
    for tp, t in held:
        assert_same_multiset(t, oracle.scan_pattern(G, tp), f"held scan {tp}")
        t.free()
    ctx.load_triples(s, p, o)


def test_scan_same_variable_filter(ctx):
    s = np.array([1, 2, 3, 3, 4, 4], np.uint32)
    p = np.array([0, 0, 0, 1, 0, 0], np.uint32)
    o = np.array([1, 5, 3, 3, 4, 9], np.uint32)
    ctx.load_triples(s, p, o)
    t = ctx.scan_pattern((0, 0, 0, 5))
    assert_same_multiset(t, ([0], np.array([[1], [3], [4]], np.uint32)), "?x p ?x")


def test_worked_example_as_query(ctx):
    from golden_example import Dictionary, load
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
        bgp.append(tuple(f) + (mask,))
    ctx.load_triples(s, p, o)
    res = ctx.query(bgp)
    vars_, cols = res.to_host()
    header = [k for k in g if k.startswith("SOLUTIONS")][0]
    names = header.split()[1:]
    pos = [vars_.index(var_ids[n]) for n in names]
    rows = sorted(tuple(d.term(cols[c][i]) for c in pos) for i in range(res.nrows))
    assert rows == sorted(tuple(r) for r in g[header])


def test_query_tiny_graphs_brute_force(ctx):
    from test_oracle import tiny_bgp, tiny_graph
    for seed in range(40):
        graph = tiny_graph(seed)
        bgp = tiny_bgp(seed)
        ctx.load_triples(*graph)
        res = ctx.query(bgp)
        assert_same_multiset(res, oracle.brute_force_bgp(graph, bgp), f"seed {seed} {bgp}")
        res.free()


def test_query_generated_bgps(ctx, small_graph):
    s, p, o = small_graph
    ctx.load_triples(s, p, o)
    G = oracle.distinct_triples(s, p, o)
    bgps = generate_bgps(GraphIndex(s, p, o), 24, seed=7)
    for b in bgps:
        res = ctx.query(b["patterns"])
        want = oracle.evaluate_bgp(G, b["patterns"], is_set=True)
        assert_same_multiset(res, want, str(b["patterns"]))
        res.free()


def test_query_batch_matches_oracle(ctx, small_graph):
    """Batched BGP evaluation: every query of the batch equals the oracle."""
    s, p, o = small_graph
    ctx.load_triples(s, p, o)
    G = oracle.distinct_triples(s, p, o)
    bgps = [b["patterns"] for b in generate_bgps(GraphIndex(s, p, o), 24, seed=19)]
    bgps.append([(0, 6, 0, 5)])                       # one pattern, repeated variable
    bgps.append([(5, 99, 1, 4), (1, 6, 2, 5)])        # a pattern with no match
    res = ctx.query_batch(bgps)
    assert len(res) == len(bgps)
    for b, r in zip(bgps, res):
        assert_same_multiset(r, oracle.evaluate_bgp(G, b, is_set=True), str(b))
        r.free()
    assert ctx.query_batch([]) == []


def test_query_patterns_without_variables(ctx, small_graph):
    """A pattern without variables tests one triple's presence: a present one
    changes nothing, an absent one empties the BGP; BGPs of such patterns
    alone give one row without columns, or none.  Plain and batched, stars
    and chains, against the oracle."""
    s, p, o = small_graph
    ctx.load_triples(s, p, o)
    G = oracle.distinct_triples(s, p, o)
    here = (int(s[7]), int(p[7]), int(o[7]), 0)
    absent = (int(s[7]), int(p[7]), 0xFFFFFFF0, 0)
    bgps = generate_bgps(GraphIndex(s, p, o), 6, seed=23)
    cases = []
    for b in bgps:
        pats = list(b["patterns"])
        cases += [pats + [here], [here] + pats, pats + [absent], [here, absent] + pats]
    cases += [[here], [here, here], [absent], [here, absent], [absent, here]]
    for bgp in cases:
        res = ctx.query(bgp)
        assert_same_multiset(res, oracle.evaluate_bgp(G, bgp, is_set=True), str(bgp))
        res.free()
    for bgp, r in zip(cases, ctx.query_batch(cases)):
        assert_same_multiset(r, oracle.evaluate_bgp(G, bgp, is_set=True), "batched " + str(bgp))
        r.free()


def test_query_order_invariance(ctx, small_graph):
    s, p, o = small_graph
    ctx.load_triples(s, p, o)
    b = generate_bgps(GraphIndex(s, p, o), 2, seed=11)[1]["patterns"]
    ref = oracle.canonical(host_rows(ctx.query(b)))
    for perm in itertools.islice(itertools.permutations(b), 6):
        got = oracle.canonical(host_rows(ctx.query(list(perm))))
        assert got[0] == ref[0] and np.array_equal(got[1], ref[1])


def test_query_errors(ctx, small_graph):
    from paper_1702_03484_gb300 import MapsqError
    s, p, o = small_graph
    ctx.load_triples(s, p, o)
    with pytest.raises(MapsqError) as e:
        ctx.query([(0, 1, 2, 7)])
    assert e.value.name == "UNSUPPORTED"
    with pytest.raises(MapsqError) as e:
        ctx.query([(16, 1, 2, 5)])
    assert e.value.name == "INVALID"


def test_university_bgps_full_size(ctx):
    """The plain-BGP workload at full size: 32 star/chain BGPs over 1e7 triples."""
    s, p, o = gen.university_graph(10_000_000, seed=2)
    ctx.load_triples(s, p, o)
    assert ctx.store_info() == (10_000_000, 18)
    G = oracle.distinct_triples(s, p, o)
    bgps = generate_bgps(GraphIndex(s, p, o), 32, seed=2)
    total = 0
    batched = ctx.query_batch([b["patterns"] for b in bgps])
    for b, rb in zip(bgps, batched):
        res = ctx.query(b["patterns"])
        want = oracle.evaluate_bgp(G, b["patterns"], is_set=True)
        assert_same_multiset(res, want, str(b["patterns"]))
        assert_same_multiset(rb, want, "batched " + str(b["patterns"]))
        total += res.nrows
        res.free()
        rb.free()
    assert total > 0
