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
