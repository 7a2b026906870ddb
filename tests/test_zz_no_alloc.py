"""mapsq_join_noalloc, the join for callers that cannot allocate device memory
(a host that lends only fixed buffers, or a path where an allocation could
block or fail): called through the C ABI, its output must equal mapsq_join's
exactly (as canonically sorted multisets), on calls made one after another so
that leftovers of an earlier call in the shared scratch array would show.

This file is named to be collected last."""
import numpy as np
import pytest

import gen
import oracle
from gpu_helpers import device_table, host_rows

pytestmark = pytest.mark.gpu


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream or 1  # legacy default stream


def _noalloc_join(L, R, capacity, left_sorted=(), right_sorted=()):
    """Run the allocation-free join on device copies of L and R; returns
    (status, (vars, rows) or None, row count).  ``left_sorted`` and
    ``right_sorted`` list columns to mark as sorted (sorted_mask)."""
    import torch
    from paper_1702_03484_gb300 import mapsq
    lcols = [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in L.cols]
    rcols = [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in R.cols]
    lv = mapsq.table_view(L.vars, lcols, L.nrows, sorted_cols=left_sorted)
    rv = mapsq.table_view(R.vars, rcols, R.nrows, sorted_cols=right_sorted)
    n_out = len(set(L.vars) | set(R.vars))
    bufs = [torch.full((max(capacity, 1),), -1, dtype=torch.int32, device="cuda") for _ in range(n_out)]
    rc, out, rows = mapsq.mapsq_join_noalloc(lv, rv, [b.data_ptr() for b in bufs], capacity, _stream())
    torch.cuda.synchronize()
    if rc != 0:
        return rc, None, rows
    vars_ = list(out.var[: out.ncols])
    host = np.stack([b[:rows].cpu().numpy().view(np.uint32) for b in bufs], axis=1) if n_out else \
        np.zeros((rows, 0), np.uint32)
    return rc, (vars_, host), rows


def _reference(ctx, L, R):
    return host_rows(ctx.join(device_table(ctx, L), device_table(ctx, R)))


def _same(a, b):
    av, ar = oracle.canonical(a)
    bv, br = oracle.canonical(b)
    return av == bv and ar.shape == br.shape and np.array_equal(ar, br)


def test_noalloc_join_equals_mapsq_join_on_consecutive_calls():
    from paper_1702_03484_gb300 import Context
    big = gen.skewed_two_key(seed=3, log_a=18, log_b=16, log_keys=14)      # 2^18 x 2^16, two-variable key
    small = gen.pairwise_uniform(seed=1)                                    # 16384 x 8192, one-variable key
    r = gen.Rng(12)
    cross = (gen.Table([0, 1], [r.u32(300), r.u32(300)]), gen.Table([2], [r.u32(200)]))
    with Context(device=0) as ctx:
        for L, R in (big, small, small, cross, big):
            want = _reference(ctx, L, R)
            rc, got, rows = _noalloc_join(L, R, capacity=want[1].shape[0] + 7)
            assert rc == 0, rc
            assert rows == want[1].shape[0]
            assert _same(got, want)


def test_noalloc_join_reports_capacity_and_limits():
    from paper_1702_03484_gb300 import Context
    L, R = gen.pairwise_uniform(seed=1)
    with Context(device=0) as ctx:
        want = _reference(ctx, L, R)
    n = want[1].shape[0]
    rc, got, rows = _noalloc_join(L, R, capacity=n - 1)
    assert rc == -4 and rows == n          # MAPSQ_ERR_BUDGET, with the size needed
    rc, got, rows = _noalloc_join(L, R, capacity=n)
    assert rc == 0 and _same(got, want)
    too_big = gen.Table([0, 1], [np.zeros((1 << 18) + 1, np.uint32)] * 2)
    too_big2 = gen.Table([0, 2], [np.zeros((1 << 18) + 1, np.uint32)] * 2)
    rc, _, _ = _noalloc_join(too_big, too_big2, capacity=16)
    assert rc == -1                          # MAPSQ_ERR_INVALID: beyond the scratch array


def test_noalloc_join_sorted_larger_side_within_limits():
    """A key-sorted input (sorted_mask set) several times larger than the other
    must still be accepted: the limits bind the smaller and the larger input,
    whichever side each is on."""
    r = gen.Rng(77)
    nl, nr, dom = 1 << 19, 1 << 16, 1 << 17
    lk = np.sort(r.below(nl, dom).astype(np.uint32))
    L = gen.Table([0, 1], [lk, r.u32(nl)])
    R = gen.Table([0, 2], [r.below(nr, dom).astype(np.uint32), r.u32(nr)])
    want = oracle.join_mapreduce(L, R)
    for a, b, ls, rs in ((L, R, (0,), ()), (R, L, (), (0,))):
        w = oracle.join_mapreduce(a, b)
        rc, got, rows = _noalloc_join(a, b, capacity=w[1].shape[0] + 3, left_sorted=ls, right_sorted=rs)
        assert rc == 0, rc
        assert rows == want[1].shape[0]
        assert _same(got, w)


def test_noalloc_join_at_the_limits():
    """Exactly 2^18 rows on the smaller input (six value columns, 4096 distinct
    keys, so large key groups) and 2^20 on the larger: the worst case the fixed
    array is sized for, compared with mapsq_join; then inputs with only the
    larger side one row over its limit are rejected."""
    from paper_1702_03484_gb300 import Context
    r = gen.Rng(78)
    nb, np_ = 1 << 18, 1 << 20
    B = gen.Table([0, 1, 2, 3, 4, 5, 6], [r.below(nb, 4096).astype(np.uint32)] + [r.u32(nb) for _ in range(6)])
    P = gen.Table([0, 10, 11], [r.below(np_, 1 << 16).astype(np.uint32), r.u32(np_), r.u32(np_)])
    with Context(device=0) as ctx:
        for L, R in ((P, B), (B, P)):
            want = _reference(ctx, L, R)
            rc, got, rows = _noalloc_join(L, R, capacity=want[1].shape[0] + 5)
            assert rc == 0, rc
            assert rows == want[1].shape[0] > 1 << 21
            assert _same(got, want)
    over = gen.Table([0, 10], [np.zeros(np_ + 1, np.uint32)] * 2)
    small = gen.Table([0, 1], [np.zeros(16, np.uint32)] * 2)
    for L, R in ((over, small), (small, over)):
        rc, _, _ = _noalloc_join(L, R, capacity=16)
        assert rc == -1                      # MAPSQ_ERR_INVALID: the larger input is over its limit
