"""Parity at full size, every output row against the oracle.

* Skewed large join: A = 2^26 rows, B = 2^24 rows, two shared variables packed
  in a 64-bit key, Zipf(1.1) key frequencies on A, exactly 2^28 output rows.
  The key space is cut into 16 buckets (top four bits of x); per bucket the
  oracle joins the bucket's rows of A and B (Algorithm 1 restricted to those
  keys, so the buckets' results add up to the whole join) and the GPU rows of
  that bucket are compared with it as canonically sorted multisets.
* Uneven batch: all 256 joins of the batch, each compared in full.
* Serving: every distinct query of a served stream over the 1e8-triple graph
  equals the oracle's evaluation of it, and every served result equals the
  same query evaluated alone.

The oracle runs in spawned host processes meanwhile; the canonical sort of
large results runs on the device through torch.sort (a permutation of the
rows, which cannot make different multisets equal)."""
import numpy as np
import pytest

import gen
import oracle
import oracle_jobs
from gpu_helpers import assert_rows_equal_device, oracle_pool

pytestmark = pytest.mark.gpu


def _as_u64(col):
    import torch
    return col.view(torch.int32).to(torch.int64) & 0xFFFFFFFF


def _rows(cols, sel=None):
    import torch
    parts = [c.view(torch.int32) if sel is None else c.view(torch.int32)[sel] for c in cols]
    return torch.stack(parts, dim=1)


def test_skewed_join_full_size():
    import torch
    from paper_1702_03484_gb300 import Context
    A, B = gen.skewed_two_key(seed=3)
    buckets, shift = 16, np.uint32(28)
    ab, bb = A.cols[0] >> shift, B.cols[0] >> shift
    jobs = [((A.vars, [c[ab == b] for c in A.cols]), (B.vars, [c[bb == b] for c in B.cols])) for b in range(buckets)]
    with oracle_pool(8) as pool, Context(device=0) as ctx:
        wants = pool.imap(oracle_jobs.join_job, jobs)
        tA = ctx.table(A.vars, [torch.from_numpy(c).cuda() for c in A.cols])
        tB = ctx.table(B.vars, [torch.from_numpy(c).cuda() for c in B.cols])
        out = ctx.join(tA, tB)
        assert out.nrows == 1 << 28
        assert out.vars == [0, 1, 2, 3, 4, 5]
        cols = out.device_columns()
        xb = _as_u64(cols[0]) >> 28
        checked = 0
        for b, (wv, wr) in enumerate(wants):
            assert wv == out.vars
            got = _rows(cols, xb == b)
            assert_rows_equal_device(got, wr, f"key bucket {b}")
            checked += got.shape[0]
            del got
        assert checked == 1 << 28
        out.free()


def test_uneven_batch_full_size():
    """The 256-join batch at full size through mapsq_join_batch: every join
    compared in full with the oracle."""
    import torch
    from paper_1702_03484_gb300 import Context
    joins = gen.uneven_batch(seed=4)
    jobs = [((L.vars, L.cols), (R.vars, R.cols)) for L, R, _ in joins]
    with oracle_pool() as pool, Context(device=0) as ctx:
        wants = pool.imap(oracle_jobs.join_job, jobs)
        dev = [(ctx.table(L.vars, [torch.from_numpy(c).cuda() for c in L.cols]),
                ctx.table(R.vars, [torch.from_numpy(c).cuda() for c in R.cols])) for L, R, _ in joins]
        outs = ctx.join_batch([a for a, _ in dev], [b for _, b in dev])
        assert len(outs) == len(joins)
        total = 0
        for j, ((L, R, s), out, (wv, wr)) in enumerate(zip(joins, outs, wants)):
            assert out.vars == wv, f"join {j}"
            assert out.nrows == wr.shape[0], f"join {j} (s={s})"
            if out.nrows:
                assert_rows_equal_device(_rows(out.device_columns()), wr, f"join {j} (s={s})")
            total += out.nrows
            out.free()
        assert total > 1 << 27


def test_served_stream_full_size(tmp_path):
    """Serving over the 1e8-triple graph: 400 arrivals at about 2000 queries/s
    drawn from 128 witness BGPs are served concurrently; every served result
    equals the same query evaluated alone through mapsq_query, and every
    distinct query's result equals the oracle's."""
    import time
    from paper_1702_03484_gb300 import Context
    from gen.bgp import GraphIndex, generate_bgps
    from gpu_helpers import host_rows
    s, p, o = gen.university_graph(100_000_000, seed=2)
    bgps = [b["patterns"] for b in generate_bgps(GraphIndex(s, p, o), 128, seed=5, k_range=(3, 8),
                                                 var_range=None)]
    r = gen.Rng(5, 7)
    stream = [int(i) for i in r.below(400, len(bgps))]
    distinct = sorted(set(stream))
    G = oracle.distinct_triples(s, p, o)
    oracle_jobs.save_split_graph(oracle.split_by_predicate(G), str(tmp_path / "graph"))
    del G
    with oracle_pool(initializer=oracle_jobs.load_split_graph, initargs=(str(tmp_path / "graph"),)) as pool:
        pending = pool.map_async(oracle_jobs.bgp_job, [bgps[i] for i in distinct])
        with Context(device=0) as ctx:
            ctx.load_triples(s, p, o)
            ctx.serve_start(max_active=256, mem_budget_bytes=40 << 30)
            tickets = []
            for i in stream:
                tickets.append(ctx.submit(bgps[i]))
                time.sleep(0.0005)  # 2000 queries/s
            served = [None] * len(stream)
            deadline = time.time() + 300
            while any(x is None for x in served) and time.time() < deadline:
                for k, t in enumerate(tickets):
                    if served[k] is None:
                        res = ctx.poll(t)
                        if res is not None:
                            served[k] = oracle.canonical(host_rows(res))
                            res.free()
                time.sleep(0.001)
            stats = ctx.serve_stats()
            ctx.serve_stop()
            assert all(x is not None for x in served)
            assert stats["completed"] == len(stream) and stats["failed"] == 0
            alone = {}
            for i in distinct:
                res = ctx.query(bgps[i])
                alone[i] = oracle.canonical(host_rows(res))
                res.free()
        for k, i in enumerate(stream):
            assert served[k][0] == alone[i][0] and np.array_equal(served[k][1], alone[i][1]), bgps[i]
        wants = pending.get(timeout=1200)
    assert sum(w[1].shape[0] for w in wants) > 0
    for i, want in zip(distinct, wants):
        got = alone[i]
        assert got[0] == want[0] and np.array_equal(got[1], want[1]), bgps[i]
