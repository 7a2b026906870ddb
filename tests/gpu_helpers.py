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
