"""The serving loop (continuous batching of BGP queries with memory admission):
every query served in a mix of concurrent queries must return exactly the
oracle's result and exactly what the same query returns alone through
mapsq_query, with or without a memory budget tight enough to defer and put
back queries."""
import threading
import time

import numpy as np
import pytest

import gen
import oracle
from gen.bgp import GraphIndex, generate_bgps
from gpu_helpers import assert_same_multiset, host_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def graph():
    return gen.university_graph(150_000, seed=2)


@pytest.fixture(scope="module")
def ctx(graph):
    import torch
    from paper_1702_03484_gb300 import Context
    assert torch.cuda.is_available()
    c = Context(device=0)
    c.load_triples(*graph)
    yield c
    c.close()


@pytest.fixture(scope="module")
def bgps(graph):
    s, p, o = graph
    out = [b["patterns"] for b in generate_bgps(GraphIndex(s, p, o), 40, seed=23, k_range=(3, 8),
                                                var_range=None)]
    out.append([(0, 6, 0, 5)])                    # one pattern, repeated variable
    out.append([(5, 99, 1, 4), (1, 6, 2, 5)])     # a pattern with no match
    return out


def _serve_all(ctx, bgps, waves=4, **opts):
    """Submit ``bgps`` in waves from a second thread while this one polls; returns
    {index: rows or error name} and the serving counters."""
    from paper_1702_03484_gb300 import MapsqError
    ctx.serve_start(**opts)
    tickets = {}

    def producer():
        for w in range(waves):
            for i in range(w, len(bgps), waves):
                tickets[i] = ctx.submit(bgps[i])
            time.sleep(0.002)

    th = threading.Thread(target=producer)
    th.start()
    results = {}
    deadline = time.time() + 120
    while len(results) < len(bgps) and time.time() < deadline:
        for i, t in list(tickets.items()):
            if i in results:
                continue
            try:
                r = ctx.poll(t)
            except MapsqError as e:
                results[i] = e.name
                continue
            if r is not None:
                results[i] = host_rows(r)
                r.free()
        time.sleep(0.001)
    th.join()
    stats = ctx.serve_stats()
    ctx.serve_stop()
    assert len(results) == len(bgps), "serving loop did not finish in time"
    return results, stats


def _alone(ctx, bgps):
    out = []
    for b in bgps:
        r = ctx.query(b)
        out.append(oracle.canonical(host_rows(r)))
        r.free()
    return out


def _same(a, want_canon):
    got = oracle.canonical(a)
    return got[0] == want_canon[0] and np.array_equal(got[1], want_canon[1])


def test_served_results_equal_oracle_and_alone(ctx, graph, bgps):
    results, stats = _serve_all(ctx, bgps)
    alone = _alone(ctx, bgps)
    G = oracle.distinct_triples(*graph)
    for i, b in enumerate(bgps):
        assert not isinstance(results[i], str), (b, results[i])
        assert _same(results[i], alone[i]), b
        want = oracle.evaluate_bgp(G, b, is_set=True)
        got = results[i]

        class Rows:
            nrows = got[1].shape[0]

            @staticmethod
            def to_host():
                return got[0], [np.ascontiguousarray(got[1][:, c]) for c in range(got[1].shape[1])]

        assert_same_multiset(Rows, want, str(b))
    assert stats["submitted"] == len(bgps) and stats["completed"] == len(bgps) and stats["failed"] == 0
    assert stats["batched_joins"] == sum(len(b) - 1 for b in bgps)
    assert stats["rounds"] < stats["batched_joins"]            # joins of many queries shared rounds
    assert 0 < stats["p50_ms"] <= stats["p99_ms"]


def test_served_under_tight_budget(ctx, bgps):
    """A budget a little above the largest single step defers and puts back
    queries; results are unchanged."""
    alone = _alone(ctx, bgps)
    largest = max(a[1].nbytes for a in alone)
    budget = 3 * largest + (4 << 20)
    results, stats = _serve_all(ctx, bgps, waves=1, mem_budget_bytes=budget)
    for i, b in enumerate(bgps):
        if isinstance(results[i], str):
            assert results[i] == "BUDGET", (b, results[i])
        else:
            assert _same(results[i], alone[i]), b
    assert stats["completed"] + stats["failed"] == len(bgps)
    assert stats["completed"] >= len(bgps) // 2


def test_query_over_budget_fails_alone(ctx, bgps):
    alone = _alone(ctx, bgps)
    big = int(np.argmax([a[1].shape[0] for a in alone]))
    results, stats = _serve_all(ctx, [bgps[big], [(0, 6, 0, 5)]], waves=1, mem_budget_bytes=1 << 10)
    assert results[0] == "BUDGET"
    assert stats["failed"] >= 1


def test_serving_state_errors(ctx, bgps):
    from paper_1702_03484_gb300 import MapsqError
    with pytest.raises(MapsqError) as e:
        ctx.submit(bgps[0])
    assert e.value.name == "BUSY"                              # not serving
    ctx.serve_start(max_active=4)
    try:
        with pytest.raises(MapsqError) as e:
            ctx.serve_start()
        assert e.value.name == "BUSY"
        with pytest.raises(MapsqError) as e:
            ctx.query(bgps[0])
        assert e.value.name == "BUSY"                          # other calls wait for the stop
        with pytest.raises(MapsqError) as e:
            ctx.poll(10 ** 9)
        assert e.value.name == "NOT_FOUND"
        with pytest.raises(MapsqError) as e:
            ctx.submit([(0, 1, 2, 7)])
        assert e.value.name == "UNSUPPORTED"
        t = ctx.submit(bgps[1])
        while (r := ctx.poll(t)) is None:
            time.sleep(0.001)
        assert r.nrows >= 0
        r.free()
    finally:
        ctx.serve_stop()
    with pytest.raises(MapsqError) as e:
        ctx.serve_stop()
    assert e.value.name == "BUSY"


def test_concurrent_submitters(ctx, bgps):
    """Four threads submit at once (mapsq_submit is thread-safe) while the main
    thread polls; every result equals the query alone."""
    alone = _alone(ctx, bgps)
    ctx.serve_start()
    tickets = {}
    lock = threading.Lock()

    def submitter(offset):
        for i in range(offset, len(bgps), 4):
            t = ctx.submit(bgps[i])
            with lock:
                tickets[i] = t

    threads = [threading.Thread(target=submitter, args=(o,)) for o in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    results = {}
    deadline = time.time() + 120
    while len(results) < len(bgps) and time.time() < deadline:
        for i, t in tickets.items():
            if i not in results:
                r = ctx.poll(t)
                if r is not None:
                    results[i] = host_rows(r)
                    r.free()
        time.sleep(0.001)
    stats = ctx.serve_stats()
    ctx.serve_stop()
    assert len(set(tickets.values())) == len(bgps)  # distinct tickets
    assert len(results) == len(bgps)
    for i, b in enumerate(bgps):
        assert _same(results[i], alone[i]), b
    assert stats["submitted"] == len(bgps) and stats["failed"] == 0
