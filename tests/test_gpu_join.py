"""GPU parity of mapsq_join against the CPU oracle (bit-exact multisets)."""
import numpy as np
import pytest

import gen
import oracle
from gpu_helpers import assert_same_multiset, device_table, join_and_check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_1702_03484_gb300 import Context
    assert torch.cuda.is_available()
    c = Context(device=0)
    yield c
    c.close()


def test_pairwise_uniform_full_size(ctx):
    """Tp1 16384 rows joined with Tp2 8192 rows on a key over 4096 ids."""
    L, R = gen.pairwise_uniform(seed=1)
    n = join_and_check(ctx, L, R, "pairwise uniform")
    assert n > 30000


def test_worked_example_table1(ctx):
    from golden_example import Dictionary, load
    g = load()
    d = Dictionary()
    tp1 = gen.Table([0, 1], [np.array([d.id(r[i]) for r in g["Tp1"]], np.uint32) for i in range(2)])
    tp2 = gen.Table([0, 2], [np.array([d.id(r[i]) for r in g["Tp2"]], np.uint32) for i in range(2)])
    out = ctx.join(device_table(ctx, tp1), device_table(ctx, tp2))
    vars_, cols = out.to_host()
    assert vars_ == [0, 1, 2]
    rows = sorted(tuple(d.term(c[i]) for c in cols) for i in range(out.nrows))
    assert rows == sorted(tuple(r) for r in g["RS"])


def _random_pair(seed, n_shared, max_rows):
    r = gen.Rng(seed, 21)
    nl = int(r.below(1, max_rows + 1)[0])
    nr = int(r.below(1, max_rows + 1)[0])
    dom = int(r.between(1, 1, max(2, max_rows // 4))[0])
    lv = list(range(n_shared)) + [8 + i for i in range(int(r.between(1, 0, 3)[0]))]
    rv = list(range(n_shared)) + [12 + i for i in range(int(r.between(1, 0, 3)[0]))]
    lv = lv or [8]
    rv = rv or [12]
    lv = [lv[i] for i in r.permutation(len(lv))]
    rv = [rv[i] for i in r.permutation(len(rv))]
    return gen.random_table(r, nl, lv, dom), gen.random_table(r, nr, rv, dom)


@pytest.mark.parametrize("n_shared", [0, 1, 2])
def test_random_joins_ragged(ctx, n_shared):
    """Random sizes (ragged tails, several write tiles), shuffled column orders."""
    max_rows = 300 if n_shared == 0 else 6000
    for seed in range(25):
        L, R = _random_pair(seed * 3 + n_shared, n_shared, max_rows)
        join_and_check(ctx, L, R, f"seed {seed} shared {n_shared}")


def test_extreme_ids_and_sentinel_key(ctx):
    big = 0xFFFFFFFF
    L = gen.Table([0, 1, 2], [np.array([big, big, 0, 5, big], np.uint32), np.array([big, 0, 0, 5, big], np.uint32),
                              np.arange(5, dtype=np.uint32)])
    R = gen.Table([1, 0, 3], [np.array([big, 0, big, 5], np.uint32), np.array([big, 0, big, 5], np.uint32),
                              np.array([7, 8, 9, 10], np.uint32)])
    join_and_check(ctx, L, R, "two-variable key with all-ones ids")
    L1 = gen.Table([0, 1], [np.array([big, 0, big], np.uint32), np.array([1, 2, 3], np.uint32)])
    R1 = gen.Table([0, 2], [np.array([0, big], np.uint32), np.array([4, 5], np.uint32)])
    join_and_check(ctx, L1, R1, "one-variable key with ids 0 and 2^32-1")


def test_hot_key_on_build_side(ctx):
    """One key holds most of the smaller side: its group spans many output tiles."""
    r = gen.Rng(5)
    rk = np.concatenate((np.full(3000, 7, np.uint32), r.below(1000, 50).astype(np.uint32)))
    R = gen.Table([0, 2], [rk, r.u32(rk.shape[0])])
    lk = np.concatenate((np.full(40, 7, np.uint32), r.below(9000, 50).astype(np.uint32)))
    L = gen.Table([0, 1], [lk, r.u32(lk.shape[0])])
    n = join_and_check(ctx, L, R, "hot key")
    assert n >= 40 * 3000


def test_large_build_sides(ctx):
    """Build sides of 2^16 rows and more take the region-partitioned build and,
    when no key group exceeds sixteen rows, the fused write: ragged sizes, many
    value columns, one- and two-variable keys, a hot build key (one region far
    larger than the others, and the partitioned write) and all build rows in
    one key."""
    r = gen.Rng(15)
    n = 70_001
    # many value columns, key groups of at most a few rows: partitioned build, fused write
    B = gen.Table([0, 1, 2, 3, 4, 5], [r.below(n, 40_000).astype(np.uint32)] + [r.u32(n) for _ in range(5)])
    P = gen.Table([0, 9], [r.below(150_003, 40_000).astype(np.uint32), r.u32(150_003)])
    join_and_check(ctx, P, B, "five build value columns")
    # two-variable key, probe side of one partial tile
    x, y = r.below(n, 300).astype(np.uint32), r.below(n, 300).astype(np.uint32)
    B2 = gen.Table([0, 1, 6], [x, y, r.u32(n)])
    P2 = gen.Table([7, 1, 0], [r.u32(90_017), r.below(90_017, 300).astype(np.uint32),
                               r.below(90_017, 300).astype(np.uint32)])
    join_and_check(ctx, B2, P2, "two-variable key")
    # a hot key with 40% of the build rows
    hk = r.below(n, 60_000).astype(np.uint32)
    hk[r.below(28_000, n)] = 12345
    B3 = gen.Table([0, 2], [hk, r.u32(n)])
    P3 = gen.Table([0, 1], [np.concatenate((np.full(30, 12345, np.uint32), r.below(100_000, 60_000).astype(np.uint32))),
                            r.u32(100_030)])
    assert join_and_check(ctx, P3, B3, "hot build key") >= 30 * 20_000
    # every build row in one key
    B4 = gen.Table([0, 2], [np.full(1 << 16, 77, np.uint32), r.u32(1 << 16)])
    P4 = gen.Table([0, 1], [np.array([77, 1, 77], np.uint32), r.u32(3)])
    assert join_and_check(ctx, P4, B4, "one key") == 2 << 16


def test_build_side_either_way(ctx):
    r = gen.Rng(6)
    small = gen.Table([0, 1, 3], [r.below(100, 64).astype(np.uint32), r.u32(100), r.u32(100)])
    large = gen.Table([4, 0], [r.u32(5000), r.below(5000, 64).astype(np.uint32)])
    join_and_check(ctx, small, large, "left smaller")
    join_and_check(ctx, large, small, "right smaller")


def test_cross_product_unit_and_empty(ctx):
    r = gen.Rng(8)
    A = gen.Table([0, 1], [r.u32(123), r.u32(123)])
    B = gen.Table([2], [r.u32(77)])
    join_and_check(ctx, A, B, "cross product")
    join_and_check(ctx, A, gen.Table.unit(1), "unit table")
    join_and_check(ctx, gen.Table.unit(1), A, "unit table on the left")
    join_and_check(ctx, A, gen.Table.unit(0), "empty 0-column table")
    E = gen.Table([0, 5], [np.zeros(0, np.uint32), np.zeros(0, np.uint32)])
    join_and_check(ctx, A, E, "empty right")
    join_and_check(ctx, E, A, "empty left")
    join_and_check(ctx, gen.Table.unit(1), gen.Table.unit(1), "unit x unit")


def test_disjoint_keys_give_empty(ctx):
    A = gen.Table([0, 1], [np.arange(100, dtype=np.uint32), np.arange(100, dtype=np.uint32)])
    B = gen.Table([0, 2], [np.arange(100, 200, dtype=np.uint32), np.arange(100, dtype=np.uint32)])
    assert join_and_check(ctx, A, B, "disjoint") == 0


def test_skewed_two_key_reduced(ctx):
    """The skewed large-join workload at 2^18 x 2^16 rows: exactly 4 * 2^18 output rows."""
    A, B = gen.skewed_two_key(seed=3, log_a=18, log_b=16, log_keys=14)
    assert join_and_check(ctx, A, B, "skewed two-key") == 4 << 18


def test_uneven_batch_reduced(ctx):
    for i, (L, R, s) in enumerate(gen.uneven_batch(seed=4, n_joins=10, log_lo=8.0, log_hi=15.0)):
        join_and_check(ctx, L, R, f"batch join {i} (s={s})")


def test_result_tables_chain(ctx):
    """A join result is a valid input of the next join (three-way chain)."""
    r = gen.Rng(9)
    A = gen.Table([0, 1], [r.below(500, 40).astype(np.uint32), r.below(500, 40).astype(np.uint32)])
    B = gen.Table([1, 2], [r.below(400, 40).astype(np.uint32), r.below(400, 40).astype(np.uint32)])
    C = gen.Table([2, 0], [r.below(300, 40).astype(np.uint32), r.below(300, 40).astype(np.uint32)])
    ab = ctx.join(device_table(ctx, A), device_table(ctx, B))
    abc = ctx.join(ab, device_table(ctx, C))
    want = oracle.join_mapreduce(oracle.join_mapreduce(A, B), C)
    assert_same_multiset(abc, want, "chain")


def test_three_shared_variables_unsupported(ctx):
    from paper_1702_03484_gb300 import MapsqError
    A = gen.Table([0, 1, 2], [np.arange(4, dtype=np.uint32)] * 3)
    with pytest.raises(MapsqError) as e:
        ctx.join(device_table(ctx, A), device_table(ctx, A))
    assert e.value.name == "UNSUPPORTED"


def test_budget_and_allocator_failures():
    import torch
    from paper_1702_03484_gb300 import Context, MapsqError, mapsq
    L, R = gen.pairwise_uniform(seed=1)
    with Context(device=0, budget=600 << 10) as small:  # inputs fit, the join does not
        tl, tr = device_table(small, L), device_table(small, R)
        with pytest.raises(MapsqError) as e:
            small.join(tl, tr)
        assert e.value.name == "BUDGET"
    calls = {"n": 0}

    def refuse(nbytes, user, stream):
        calls["n"] += 1
        return None

    def release(ptr, nbytes, user, stream):
        pass

    a = mapsq.Allocator(mapsq.ALLOC_FN(refuse), mapsq.FREE_FN(release), None)
    a._keep = (refuse, release)
    with pytest.raises(MapsqError) as e:
        Context(device=0, allocator=a)
    assert e.value.name == "OOM" and calls["n"] >= 1
    torch.cuda.synchronize()


def test_torch_caching_allocator():
    from paper_1702_03484_gb300 import Context, torch_allocator
    L, R = gen.pairwise_uniform(seed=1)
    with Context(device=0, allocator=torch_allocator()) as c:
        join_and_check(c, L, R, "torch allocator")
        assert c.memory_in_use()[1] > 0


def test_profiling_reports_kernels(ctx):
    L, R = gen.pairwise_uniform(seed=1)
    ctx.reset_stats()
    ctx.set_profiling(True)
    join_and_check(ctx, L, R, "profiled")
    stats = ctx.kernel_stats()
    ctx.set_profiling(False)
    write = next(w for w in ("join_write", "dense_write") if w in stats)
    for k in ("hash_insert", "hash_scatter", "probe_count", "prefix_sum", write):
        assert stats[k]["launches"] >= 1 and stats[k]["device_ms"] > 0
    assert stats[write]["alg_bytes"] > 12 * 30000


def test_dense_write_path(ctx):
    """Joins of at most sixteen matches per probe row take the dense write (a
    thread per probe row): rows of exactly four aligned matches (16-byte
    stores) and of 0-3 matches (single stores), against the oracle."""
    ctx.reset_stats()
    ctx.set_profiling(True)
    try:
        r = gen.Rng(91)
        # every build key exactly four times: probe rows match 0 or 4 rows
        keys = np.repeat(np.unique(r.below(3000, 1 << 20).astype(np.uint32)), 4)
        B = gen.Table([0, 12, 13], [keys, r.u32(keys.shape[0]), r.u32(keys.shape[0])])
        A = gen.Table([0, 8], [np.concatenate((keys[::4][:2000], r.below(20000, 1 << 20).astype(np.uint32))),
                               r.u32(22000)])
        assert A.nrows > B.nrows  # B is the build side
        join_and_check(ctx, A, B, "four matches")
        # 1-3 copies per key: ragged runs
        uk = np.unique(r.below(2000, 1 << 16).astype(np.uint32))
        keys2 = np.concatenate([np.full(int(c), k, np.uint32) for k, c in zip(uk, r.between(uk.shape[0], 1, 3))])
        B2 = gen.Table([0, 12], [keys2, r.u32(keys2.shape[0])])
        A2 = gen.Table([0, 8, 9], [r.below(30000, 1 << 16).astype(np.uint32), r.u32(30000), r.u32(30000)])
        join_and_check(ctx, A2, B2, "one to three matches")
        assert ctx.kernel_stats()["dense_write"]["launches"] >= 2
    finally:
        ctx.set_profiling(False)


def test_join_batch_matches_oracle(ctx):
    """Batched form: uneven joins plus special cases in one batch, each exact."""
    batch = [(L, R) for L, R, s in gen.uneven_batch(seed=4, n_joins=12, log_lo=6.0, log_hi=14.0)]
    r = gen.Rng(14)
    A = gen.Table([0, 1], [r.u32(123), r.u32(123)])
    batch += [
        (A, gen.Table([2], [r.u32(77)])),                                   # cross product
        (A, gen.Table.unit(1)),                                             # unit
        (A, gen.Table([0, 5], [np.zeros(0, np.uint32)] * 2)),                # empty side
        gen.skewed_two_key(seed=3, log_a=14, log_b=12, log_keys=10),        # two-variable key
        (gen.Table([0, 1], [np.full(50, 7, np.uint32), r.u32(50)]),         # one hot key
         gen.Table([0, 2], [np.full(3000, 7, np.uint32), r.u32(3000)])),
    ]
    lefts = [device_table(ctx, L) for L, R in batch]
    rights = [device_table(ctx, R) for L, R in batch]
    outs = ctx.join_batch(lefts, rights)
    assert len(outs) == len(batch)
    for i, ((L, R), o) in enumerate(zip(batch, outs)):
        assert_same_multiset(o, oracle.join_mapreduce(L, R), f"batch item {i}")
        o.free()
    assert ctx.join_batch([], []) == []


def _sorted_join(ctx, X, Y, x_left, sorted_col=0, algorithm=0):
    """Join through caller-described tables, X marked sorted on ``sorted_col``."""
    import ctypes as C
    import torch
    from paper_1702_03484_gb300 import JoinOpts, TableRef, mapsq
    xc = [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in X.cols]
    yc = [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in Y.cols]
    xv = mapsq.table_view(X.vars, xc, X.nrows, sorted_cols=(sorted_col,))
    yv = mapsq.table_view(Y.vars, yc, Y.nrows)
    a, b = (xv, yv) if x_left else (yv, xv)
    before = ctx.kernel_stats().get("sorted_count", {}).get("launches", 0)
    out = TableRef(ctx, mapsq.mapsq_join(ctx.handle, C.pointer(a), C.pointer(b), JoinOpts(algorithm=algorithm)))
    torch.cuda.synchronize()
    used = ctx.kernel_stats().get("sorted_count", {}).get("launches", 0) > before
    return out, used


def _sorted_table(r, n, vars_, key_col, dom):
    cols = [r.below(n, dom).astype(np.uint32) for _ in vars_]
    cols[key_col] = np.sort(cols[key_col])
    return gen.Table(vars_, cols)


def test_sorted_build_side(ctx):
    """A side sorted on the key column and at least four times the other's rows
    is used as the grouped side (the sorted join); results equal the oracle,
    with keys absent, below and above its range, extreme ids and long runs."""
    ctx.set_profiling(True)
    try:
        r = gen.Rng(77)
        for seed, (nx, ny, dom) in enumerate([(100_000, 1000, 5000), (50, 12, 40), (300_000, 70_000, 1 << 20),
                                              (4096, 1024, 3)]):
            X = _sorted_table(r, nx, [3, 0, 9], 1, dom)
            X.cols[1][:5] = 0
            X.cols[1][-3:] = 0xFFFFFFFF
            Y = gen.Table([0, 12], [r.below(ny, dom + 10).astype(np.uint32), r.u32(ny)])
            Y.cols[0][:3] = [0, 0xFFFFFFFF, dom + 5]
            want = oracle.join_mapreduce(X, Y)
            for x_left in (True, False):
                out, used = _sorted_join(ctx, X, Y, x_left, sorted_col=1)
                assert used, "sorted join not chosen"
                assert_same_multiset(out, want if x_left else oracle.join_mapreduce(Y, X), f"case {seed} {x_left}")
                out.free()
        # too small a ratio: AUTO takes the hash join; SORTED forces the search;
        # HASH never searches
        X = _sorted_table(r, 1000, [0, 5], 0, 300)
        Y = gen.Table([0, 6], [r.below(800, 300).astype(np.uint32), r.u32(800)])
        want = oracle.join_mapreduce(X, Y)
        for algorithm, expect in ((0, False), (2, True), (1, False)):
            out, used = _sorted_join(ctx, X, Y, True, algorithm=algorithm)
            assert used == expect, algorithm
            assert_same_multiset(out, want, f"algorithm {algorithm}")
            out.free()
        X = _sorted_table(r, 40_000, [0, 5], 0, 3000)
        out, used = _sorted_join(ctx, X, Y, False, algorithm=1)
        assert not used
        assert_same_multiset(out, oracle.join_mapreduce(Y, X), "hash forced")
        out.free()
    finally:
        ctx.set_profiling(False)


def test_sorted_count_both_search_modes(ctx):
    """A probe side of a few tiles (the count searches K-ary, both ends of a
    run together) and one of more than 152 tiles (bisection for the start,
    galloping for the end) give the oracle's rows, with long runs, keys below
    and above the sorted column's range and the largest id."""
    r = gen.Rng(78)
    X = _sorted_table(r, 2_000_000, [0, 4], 0, 1 << 20)
    X.cols[0][:2000] = 0                     # a long run at the start
    X.cols[0][-700:] = 0xFFFFFFFF            # and at the end
    X.cols[0][1_000_000:1_050_000] = X.cols[0][1_000_000]  # one in the middle
    X.cols[0].sort()
    for ny in (5_000, 700_000):
        Y = gen.Table([0, 7], [r.below(ny, (1 << 20) + 50).astype(np.uint32), r.u32(ny)])
        Y.cols[0][:4] = [0, 0xFFFFFFFF, 0xFFFFFFFE, int(X.cols[0][1_000_000])]
        out, used = _sorted_join(ctx, X, Y, False, algorithm=2)
        assert_same_multiset(out, oracle.join_mapreduce(Y, X), f"probe rows {ny}")
        out.free()


def test_one_pass_dense_join(ctx):
    """A large probe side against a build side of even key groups takes the
    one-pass join (lookups, scan, look-back and write in one launch, the output
    allocated at probe rows x the largest group): exact rows with probe keys
    that miss, a ragged last tile and the all-ones key, on one and two key
    columns; a build side with one large group takes the count and write
    passes, exact too."""
    r = gen.Rng(79)
    ctx.set_profiling(True)
    try:
        for nkey, groups, n_probe, hot in ((2, 3, (1 << 20) + 777, False), (1, 2, (1 << 21) + 5, False),
                                           (2, 3, (1 << 20) + 1, True)):
            ids = np.repeat(np.arange(60_000, dtype=np.uint32), groups)
            if hot:
                ids[:5000] = 7  # one group of about 5000 rows: no one-pass bound
            ids = ids[r.permutation(ids.shape[0])]
            ids[-1] = 0xFFFFFFFF
            nb = ids.shape[0]
            pid = r.below(n_probe, 70_000).astype(np.uint32)  # ids from 60000 on miss
            pid[:3] = [0xFFFFFFFF, 7, 69_999]
            if nkey == 2:
                second = (ids * 3 + 1).astype(np.uint32)
                second[-1] = 0xFFFFFFFF
                psecond = (pid * 3 + 1).astype(np.uint32)
                psecond[0] = 0xFFFFFFFF
                B = gen.Table([0, 1, 5, 6], [ids, second, r.u32(nb), r.u32(nb)])
                P = gen.Table([0, 1, 7], [pid, psecond, r.u32(n_probe)])
            else:
                B = gen.Table([0, 5], [ids, r.u32(nb)])
                P = gen.Table([0, 7, 8], [pid, r.u32(n_probe), r.u32(n_probe)])
            tb, tp = device_table(ctx, B), device_table(ctx, P)
            before = ctx.kernel_stats().get("fused_join", {}).get("launches", 0)
            out = ctx.join(tp, tb)
            used = ctx.kernel_stats().get("fused_join", {}).get("launches", 0) > before
            assert used == (not hot), (nkey, groups, hot)
            assert_same_multiset(out, oracle.join_mapreduce(P, B), f"one pass nkey {nkey} hot {hot}")
            for t in (out, tb, tp):
                t.free()
    finally:
        ctx.set_profiling(False)


def test_autotune_sets_ratio_and_joins_stay_exact():
    from paper_1702_03484_gb300 import Context, MapsqError
    with Context(device=0) as c:
        res = c.autotune(sorted_rows=1 << 18)
        assert res["sorted_rows"] == 1 << 18 and len(res["points"]) == 12
        assert [p["ratio"] for p in res["points"]] == [1 << i for i in range(12)]
        assert all(p["hash_ms"] > 0 and p["sorted_ms"] > 0 for p in res["points"])
        ratio = res["sorted_ratio"]
        assert ratio == 0xFFFFFFFF or ratio in [p["ratio"] for p in res["points"]]
        # size axis: 2^16 .. 2^22 build rows; skew axis: groups of 4 .. 64 rows
        assert [p["build_rows"] for p in res["size_points"]] == [1 << 16, 1 << 18, 1 << 20, 1 << 22, 1 << 24]
        assert [p["group_rows"] for p in res["skew_points"]] == [4, 8, 16, 32, 64]
        assert res["part_min_build"] == (1 << 64) - 1 or res["part_min_build"] in [p["build_rows"]
                                                                                    for p in res["size_points"]]
        assert 1 <= res["dense_max"] <= 64
        L, R = gen.pairwise_uniform(seed=1)
        join_and_check(c, L, R, "after autotune")
        # the choices apply to later joins: a large build side and large key groups stay exact
        r = gen.Rng(71)
        B = gen.Table([0, 2], [r.below(1 << 17, 3000).astype(np.uint32), r.u32(1 << 17)])
        P = gen.Table([0, 1], [r.below(9000, 3000).astype(np.uint32), r.u32(9000)])
        join_and_check(c, P, B, "build of 2^17 rows, about 44 rows per key, after autotune")
        with pytest.raises(MapsqError):
            c.autotune(sorted_rows=100)


def test_to_host_into_caller_arrays(ctx):
    """mapsq_table_to_host into caller-provided (pinned) arrays equals the copy into new arrays."""
    import torch
    L, R = gen.pairwise_uniform(seed=1)
    out = ctx.join(device_table(ctx, L), device_table(ctx, R))
    vars_a, cols_a = out.to_host()
    bufs = [torch.empty(out.nrows + 100, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
            for _ in range(len(out.vars))]
    vars_b, cols_b = out.to_host(bufs)
    assert vars_a == vars_b
    assert all(np.array_equal(a, b) for a, b in zip(cols_a, cols_b))
    with pytest.raises(ValueError):
        out.to_host([np.zeros(3, np.uint32)] * len(out.vars))
    out.free()


def test_bounded_wait_gives_up_and_context_stays_usable(ctx):
    """A prefix scan whose first tile is never taken: every look-back waits for
    a predecessor that is never published, gives up after the wait limit, and
    the call returns TIMEOUT; afterwards the status word is clear and joins
    are exact again."""
    from paper_1702_03484_gb300 import mapsq
    from paper_1702_03484_gb300.mapsq import MapsqError
    for spins in (1, 1000):
        with pytest.raises(MapsqError) as e:
            mapsq.mapsq_selftest_wait(ctx.handle, spins)
        assert e.value.name == "TIMEOUT"
        ctx.sync()  # the status word was cleared when the timeout was reported
        L, R = gen.pairwise_uniform(seed=1, n_left=3000, n_right=2000, key_domain=500)
        join_and_check(ctx, L, R, "after a timeout")
    mapsq.mapsq_set_wait_limit(ctx.handle, 1 << 20)


def test_join_to_host_in_slices_under_a_small_budget():
    """A join whose result is several times the context's memory budget is
    computed slice by slice into host columns and equals the oracle; a count
    without host columns gives the same row count; too small host columns give
    BUDGET with the row count."""
    import ctypes as C
    import torch
    from paper_1702_03484_gb300 import Context, mapsq
    from paper_1702_03484_gb300.mapsq import MapsqError
    r = gen.Rng(17)
    nl, nr = 1 << 18, 1 << 13
    L = gen.Table([0, 1, 2], [r.below(nl, 1 << 11).astype(np.uint32), r.u32(nl), r.u32(nl)])
    R = gen.Table([3, 0], [r.u32(nr), r.below(nr, 1 << 11).astype(np.uint32)])
    want = oracle.join_mapreduce(L, R)
    out_bytes = want[1].nbytes
    lc = [torch.from_numpy(c).cuda() for c in L.cols]
    rc = [torch.from_numpy(c).cuda() for c in R.cols]
    lv, rv = mapsq.table_view(L.vars, lc), mapsq.table_view(R.vars, rc)
    with Context(device=0, budget=out_bytes // 6) as small:
        with pytest.raises(MapsqError) as e:
            mapsq.mapsq_join(small.handle, C.pointer(lv), C.pointer(rv))
        assert e.value.name == "BUDGET"  # the plain join does not fit
        vars_, cols, slices = mapsq.mapsq_join_to_host(small.handle, lv, rv)
        assert slices >= 6
        class Host:
            nrows = cols[0].shape[0]
            @staticmethod
            def to_host():
                return vars_, cols
        assert_same_multiset(Host, want, "sliced join")
        with pytest.raises(MapsqError) as e:
            mapsq.mapsq_join_to_host(small.handle, lv, rv, capacity=want[1].shape[0] - 1)
        assert e.value.name == "BUDGET"
        # the right side as the larger one, sliced the other way
        vars2, cols2, _ = mapsq.mapsq_join_to_host(small.handle, rv, lv)
        class Host2:
            nrows = cols2[0].shape[0]
            @staticmethod
            def to_host():
                return vars2, cols2
        assert_same_multiset(Host2, oracle.join_mapreduce(R, L), "sliced join, larger side right")
