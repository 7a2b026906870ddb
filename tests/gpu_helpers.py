"""Shared helpers of the GPU parity tests (device tables, canonical compare)."""
import numpy as np

import oracle


def device_table(ctx, t):
    """Copy a generator table (``.vars``, ``.cols``) into a library table on the GPU."""
    import torch
    if not t.vars:
        return ctx.table([], [], nrows=t.nrows)
    return ctx.table(t.vars, [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in t.cols])


def host_rows(ref):
    """A library table (TableRef) copied to the host as the oracle's (vars, rows)."""
    vars_, cols = ref.to_host()
    if not cols:
        return vars_, np.zeros((ref.nrows, 0), np.uint32)
    return vars_, np.stack(cols, axis=1)


def assert_same_multiset(got, want, what=""):
    """``got`` is a library table (TableRef); ``want`` an oracle table."""
    gv, gr = oracle.canonical(host_rows(got))
    wv, wr = oracle.canonical(want)
    assert gv == wv, f"{what}: variables {gv} != {wv}"
    assert gr.shape == wr.shape, f"{what}: {gr.shape[0]} rows, expected {wr.shape[0]}"
    if gr.shape[0]:
        bad = np.flatnonzero(np.any(gr != wr, axis=1))
        assert bad.size == 0, f"{what}: {bad.size} rows differ, first at {bad[0]}: {gr[bad[0]]} vs {wr[bad[0]]}"


def join_and_check(ctx, L, R, what="", opts=None):
    tl, tr = device_table(ctx, L), device_table(ctx, R)
    out = ctx.join(tl, tr, opts)
    try:
        assert_same_multiset(out, oracle.join_mapreduce(L, R), what)
        return out.nrows
    finally:
        out.free()
        tl.free()
        tr.free()


def sort_rows_device(rows):
    """Rows of a (n, c) int32 device tensor holding uint32 values, in
    lexicographic uint32 order (stable LSD passes of torch.sort over 64-bit
    keys packing two columns each; a permutation of the rows, so it cannot make
    two different multisets equal)."""
    import torch
    n, c = rows.shape
    if n == 0 or c == 0:
        return rows
    perm = torch.arange(n, device=rows.device)
    for a in reversed(range(0, c, 2)):
        # the high column with its top bit flipped is in signed order, so
        # hi * 2^32 + lo (lo as an unsigned value) orders the pair and never overflows
        k = (rows[:, a] ^ -(1 << 31)).to(torch.int64) * (1 << 32)
        if a + 1 < c:
            k = k + (rows[:, a + 1].to(torch.int64) & 0xFFFFFFFF)
        _, idx = torch.sort(k[perm], stable=True)
        perm = perm[idx]
        del k, idx
    return rows[perm]


def assert_rows_equal_device(got, want_rows, what=""):
    """``got``: (n, c) int32 device tensor of output rows (uint32 values) with
    the columns in the oracle's order; ``want_rows``: the oracle's (n, c) uint32
    rows.  Compares the two canonically sorted multisets element by element."""
    import torch
    want = torch.from_numpy(np.ascontiguousarray(want_rows).view(np.int32)).to(got.device)
    assert got.shape == want.shape, f"{what}: {tuple(got.shape)} rows x cols, expected {tuple(want.shape)}"
    if got.shape[0] == 0:
        return
    g, w = sort_rows_device(got), sort_rows_device(want)
    bad = torch.nonzero(torch.any(g != w, dim=1)).flatten()
    if bad.numel():
        i = int(bad[0])
        raise AssertionError(f"{what}: {bad.numel()} rows differ, first at {i}: "
                             f"{g[i].cpu().numpy().view(np.uint32)} vs {w[i].cpu().numpy().view(np.uint32)}")


def oracle_pool(processes=None, initializer=None, initargs=()):
    """A pool of spawned host processes for oracle work (the test process has a
    CUDA context, so workers are spawned, never forked)."""
    import multiprocessing as mp
    import os
    n = processes or max(1, min(16, os.cpu_count() or 1))
    return mp.get_context("spawn").Pool(n, initializer=initializer, initargs=initargs)
