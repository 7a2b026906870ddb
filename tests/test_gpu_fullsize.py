"""Parity at the full size of the skewed large join: A = 2^26 rows, B = 2^24 rows,
two shared variables packed in a 64-bit key, Zipf(1.1) key frequencies on A,
exactly 2^28 output rows.  The oracle cannot materialise 2^28 rows in seconds,
so the test checks (1) the exact row count, (2) the count of output rows of
every key against |A_k| * |B_k| from independent histograms, and (3) every
output row of a seeded sample of keys (the hottest included) against the
oracle's join restricted to those keys."""
import numpy as np
import pytest

import gen
import oracle
from gpu_helpers import assert_same_multiset

pytestmark = pytest.mark.gpu


def _u64(col):
    import torch
    return col.view(torch.int32).to(torch.int64) & 0xFFFFFFFF


def _packed(x, y):
    return (x.astype(np.uint64) << np.uint64(32)) | y.astype(np.uint64)


def test_skewed_join_full_size():
    import torch
    from paper_1702_03484_gb300 import Context
    A, B = gen.skewed_two_key(seed=3)
    with Context(device=0) as ctx:
        tA = ctx.table(A.vars, [torch.from_numpy(c).cuda() for c in A.cols])
        tB = ctx.table(B.vars, [torch.from_numpy(c).cuda() for c in B.cols])
        out = ctx.join(tA, tB)
        assert out.nrows == 1 << 28
        assert out.vars == [0, 1, 2, 3, 4, 5]
        cols = out.device_columns()
        key = (_u64(cols[0]) << 32) | _u64(cols[1])
        uk, cnt = torch.unique(key, return_counts=True)
        uk, cnt = uk.cpu().numpy().view(np.uint64), cnt.cpu().numpy()
        order = np.argsort(uk, kind="stable")  # torch orders the keys as signed int64
        uk, cnt = uk[order], cnt[order]

        ka, ca = np.unique(_packed(A.cols[0], A.cols[1]), return_counts=True)
        kb, cb = np.unique(_packed(B.cols[0], B.cols[1]), return_counts=True)
        common, ia, ib = np.intersect1d(ka, kb, assume_unique=True, return_indices=True)
        keep = ca[ia] * cb[ib] > 0
        assert np.array_equal(uk, common[keep])
        assert np.array_equal(cnt, (ca[ia] * cb[ib])[keep])

        # every row of a sample of keys, the hottest key included
        r = gen.Rng(31)
        sample = np.unique(np.concatenate((ka[np.argsort(-ca)[:1]], ka[r.below(24, ka.shape[0])])))
        sel = torch.isin(key, torch.from_numpy(sample.astype(np.int64)).cuda())
        got_rows = torch.stack([c.view(torch.int32)[sel] for c in cols], dim=1).cpu().numpy().view(np.uint32)
        ma = np.isin(_packed(A.cols[0], A.cols[1]), sample)
        mb = np.isin(_packed(B.cols[0], B.cols[1]), sample)
        As = gen.Table(A.vars, [c[ma] for c in A.cols])
        Bs = gen.Table(B.vars, [c[mb] for c in B.cols])

        class Rows:
            nrows = got_rows.shape[0]

            @staticmethod
            def to_host():
                return out.vars, [np.ascontiguousarray(got_rows[:, c]) for c in range(6)]

        assert_same_multiset(Rows, oracle.join_mapreduce(As, Bs), "sampled keys")


def test_uneven_batch_full_size():
    """The 256-join batch at full size through mapsq_join_batch: every join's row
    count against the cardinality identity from independent histograms; joins of
    up to 2^18 rows in full against the oracle, larger ones on a sample of keys
    (the hottest key of the left side included)."""
    import torch
    from paper_1702_03484_gb300 import Context
    joins = gen.uneven_batch(seed=4)
    r = gen.Rng(41)
    with Context(device=0) as ctx:
        dev = [(ctx.table(L.vars, [torch.from_numpy(c).cuda() for c in L.cols]),
                ctx.table(R.vars, [torch.from_numpy(c).cuda() for c in R.cols])) for L, R, _ in joins]
        outs = ctx.join_batch([a for a, _ in dev], [b for _, b in dev])
        assert len(outs) == len(joins)
        for j, ((L, R, s), out) in enumerate(zip(joins, outs)):
            kl, cl = np.unique(L.cols[0], return_counts=True)
            kr, cr = np.unique(R.cols[0], return_counts=True)
            _, il, ir = np.intersect1d(kl, kr, assume_unique=True, return_indices=True)
            assert out.nrows == int((cl[il].astype(np.int64) * cr[ir]).sum()), f"join {j} (s={s})"
            if out.nrows <= 1 << 18:
                assert_same_multiset(out, oracle.join_mapreduce(L, R), f"join {j}")
            else:
                common = kl[il]
                sample = np.unique(np.concatenate((kl[np.argsort(-cl)[:1]], common[r.below(6, common.shape[0])])))
                key_col = out.device_columns()[out.vars.index(0)]
                sel = torch.isin(key_col.view(torch.int32), torch.from_numpy(sample.view(np.int32)).cuda())
                got = torch.stack([c.view(torch.int32)[sel] for c in out.device_columns()], dim=1)
                got = got.cpu().numpy().view(np.uint32)
                Ls = gen.Table(L.vars, [c[np.isin(L.cols[0], sample)] for c in L.cols])
                Rs = gen.Table(R.vars, [c[np.isin(R.cols[0], sample)] for c in R.cols])

                class Rows:
                    nrows = got.shape[0]

                    @staticmethod
                    def to_host():
                        return out.vars, [np.ascontiguousarray(got[:, c]) for c in range(got.shape[1])]

                assert_same_multiset(Rows, oracle.join_mapreduce(Ls, Rs), f"join {j}, sampled keys")
            out.free()


def test_served_stream_full_size():
    """Serving over the 1e8-triple graph: a burst of the Poisson stream's queries
    is served concurrently; every result equals the same query evaluated alone
    through mapsq_query, and a sample of the smaller ones equals the oracle."""
    import time
    from paper_1702_03484_gb300 import Context
    from gen.bgp import GraphIndex, generate_bgps
    from gpu_helpers import host_rows
    s, p, o = gen.university_graph(100_000_000, seed=2)
    bgps = [b["patterns"] for b in generate_bgps(GraphIndex(s, p, o), 256, seed=5, k_range=(3, 8),
                                                 var_range=None)]
    r = gen.Rng(5, 7)
    stream = [bgps[int(i)] for i in r.below(400, len(bgps))]
    with Context(device=0) as ctx:
        ctx.load_triples(s, p, o)
        ctx.serve_start(max_active=256, mem_budget_bytes=40 << 30)
        tickets = []
        for b in stream:
            tickets.append(ctx.submit(b))
            time.sleep(0.0005)  # 2000 queries/s
        served = [None] * len(stream)
        deadline = time.time() + 300
        while any(x is None for x in served) and time.time() < deadline:
            for i, t in enumerate(tickets):
                if served[i] is None:
                    res = ctx.poll(t)
                    if res is not None:
                        served[i] = oracle.canonical(host_rows(res))
                        res.free()
            time.sleep(0.001)
        stats = ctx.serve_stats()
        ctx.serve_stop()
        assert all(x is not None for x in served)
        assert stats["completed"] == len(stream) and stats["failed"] == 0
        alone = {}
        for i, b in enumerate(stream):
            key = str(b)
            if key not in alone:
                res = ctx.query(b)
                alone[key] = (oracle.canonical(host_rows(res)), res.nrows)
                res.free()
            want = alone[key][0]
            assert served[i][0] == want[0] and np.array_equal(served[i][1], want[1]), b
    G = oracle.distinct_triples(s, p, o)
    small = sorted((k for k in alone if alone[k][1] > 0), key=lambda k: alone[k][1])[:4]
    assert small
    for key in small:
        b = next(x for x in stream if str(x) == key)
        want = oracle.canonical(oracle.evaluate_bgp(G, b, is_set=True))
        got = alone[key][0]
        assert got[0] == want[0] and np.array_equal(got[1], want[1]), b
