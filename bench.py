"""Benchmark of the MapSQ join path on GB300.

Default workload: the skewed large join, A = 2^26 rows x B = 2^24 rows of four
uint32 columns, two shared variables packed into a 64-bit key, Zipf(1.1) key
frequencies on A, exactly 2^28 output rows (one step = one mapsq_join).
Metric: output bindings/s (one binding = one output row).  After the headline,
the same line carries the other join workloads measured in the same process
(``other_workloads``): the 256-join uneven batch (batched against plain), the
32 BGPs over a 1e7-triple university graph (plain against batched), the
16384 x 8192 pairwise join and a 3-second served stream over the 1e8-triple
graph (p50/p99 latency, against the same queries one after another).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload skewed_join|university_bgp|pairwise_uniform|uneven_batch|serving]

``--impl reference`` times the CPU oracle on the host cores (one process per
core) on bounded samples of the same workload per step (the paper has no code
to run).
Under torchrun (N > 1) every rank evaluates the whole workload on its own GPU
(independent replicas; weak scaling, no collective on the data path).

Other workloads alone: ``university_bgp`` (32 BGPs through mapsq_query, against
mapsq_query_batch), ``pairwise_uniform`` (16384 x 8192), ``uneven_batch`` (256
joins of uneven size in one mapsq_join_batch, against the same joins one by
one) and ``serving`` (a Poisson stream of 2000 queries/s over 1e8 triples
through the serving loop; p50/p99 latency, against serial mapsq_query).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gen  # noqa: E402
from gen.bgp import GraphIndex, generate_bgps  # noqa: E402

METRIC = "output bindings/s"
UNIT = "bindings/s"
L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)  # at least 2: the last one is profiled
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="skewed_join",
                    choices=["university_bgp", "skewed_join", "pairwise_uniform", "uneven_batch", "serving"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skewed_join only: skip the other workloads measured after the headline")
    ap.add_argument("--sorted-ratio", type=int, default=0,
                    help="fix the hash-vs-sorted crossover instead of autotuning it (profiler captures)")
    ap.add_argument("--size", default="full", choices=["full", "small"],
                    help="small: a reduced case of the workload for profiler captures (skewed_join: "
                         "2^24 x 2^22 rows over 2^20 key ids; uneven_batch: rows per side up to 2^20)")
    return ap.parse_args()


# ---------------------------------------------------------------- workloads

class Pinned:
    """Page-locked host arrays for the end-to-end copies (host <-> device DMA
    without a bounce through pageable memory): inputs copied in once at setup,
    result buffers grown on first use (the untimed warm-up) and reused."""

    def __init__(self):
        self.keep = {}

    def array(self, key, n):
        import torch
        a = self.keep.get(key)
        if a is None or a[1].shape[0] < n:
            t = torch.empty(max(int(n), 1), dtype=torch.int32, pin_memory=True)
            a = (t, t.numpy().view(np.uint32))
            self.keep[key] = a
        return a[1]

    def copy_of(self, key, col):
        dst = self.array(key, col.shape[0])[: col.shape[0]]
        dst[:] = col
        return dst

    def out(self, ncols, n):
        return [self.array(("out", c), n) for c in range(ncols)]


PINNED = Pinned()


class Workload:
    name = ""
    config = {}
    oracle_unit = "units"

    def release(self, ctx):
        """Free the workload's device tables."""
        for key in ("tA", "tB", "tL", "tR"):
            t = self.__dict__.pop(key, None)
            if t is not None:
                t.free()
        for a, b in self.__dict__.pop("dev", []):
            a.free()
            b.free()

    def setup_gpu(self, ctx):
        pass

    def run_gpu(self, ctx):
        """One step through the device-resident path; returns output rows."""
        raise NotImplementedError

    def run_e2e(self, ctx):
        """One step through the C ABI with host buffers; returns (rows, h2d, d2h)."""
        raise NotImplementedError

    def run_oracle(self, sample_index):
        """The oracle on a bounded sample; returns (rows, description)."""
        raise NotImplementedError


class UniversityBGP(Workload):
    name = "university_bgp"
    oracle_unit = "whole BGPs"

    def __init__(self, n_triples=10_000_000, n_bgps=32, seed=2):
        self.s, self.p, self.o = gen.university_graph(n_triples, seed=seed)
        self.bgps = [b["patterns"] for b in generate_bgps(GraphIndex(self.s, self.p, self.o), n_bgps, seed=seed)]
        self.config = {"workload": "university_bgp", "triples": n_triples, "predicates": 18, "bgps": n_bgps,
                       "patterns_per_bgp": "3-6", "graph_seed": seed, "bgp_seed": seed,
                       "l2": "flushed between steps (256 MiB write)"}
        self._graph_set = None

    def setup_gpu(self, ctx):
        """Loads the store (a1: dedup and the two sorted orders), timed apart
        from the metric: host arrays in, store resident."""
        t0 = time.perf_counter()
        ctx.load_triples(self.s, self.p, self.o)
        self.store_build_s = time.perf_counter() - t0

    def run_gpu(self, ctx):
        if not hasattr(self, "arrays"):  # the BGPs as C pattern arrays, built once
            from paper_1702_03484_gb300 import mapsq
            self.arrays = [mapsq.pattern_array(b) for b in self.bgps]
        rows = 0
        for a in self.arrays:
            t = ctx.query(a)
            rows += t.nrows
            t.free()
        return rows

    def run_gpu_alt(self, ctx):
        rows = 0
        for t in ctx.query_batch(self.bgps):
            rows += t.nrows
            t.free()
        return rows

    alt_form = "batched: mapsq_query_batch, all BGPs of the step in one batch, one batched join per level"

    def run_e2e(self, ctx):
        rows = h2d = d2h = 0
        for b in self.bgps:
            t = ctx.query(b)
            h2d += 16 * len(b)
            vars_, cols = t.to_host(PINNED.out(len(t.vars), t.nrows))
            d2h += sum(c.nbytes for c in cols)
            rows += t.nrows
            t.free()
        return rows, h2d, d2h

    def run_oracle(self, sample_index, budget_s=2.0):
        import oracle
        if self._graph_set is None:
            self._graph_set = oracle.distinct_triples(self.s, self.p, self.o)
        rows, done, t0 = 0, 0, time.perf_counter()
        k = sample_index
        while time.perf_counter() - t0 < budget_s and done < len(self.bgps):
            b = self.bgps[k % len(self.bgps)]
            rows += oracle.evaluate_bgp(self._graph_set, b, is_set=True)[1].shape[0]
            k += 1
            done += 1
        return rows, done


class SkewedJoin(Workload):
    name = "skewed_join"
    oracle_unit = "key buckets: the rows of A and B whose x has the same top 10 bits, joined"

    def __init__(self, log_a=26, log_b=24, log_keys=22):
        self.A, self.B = gen.skewed_two_key(seed=3, log_a=log_a, log_b=log_b, log_keys=log_keys)
        self.config = {"workload": "skewed_join", "rows_a": 1 << log_a, "rows_b": 1 << log_b,
                       "key": "two shared variables packed in 64 bits", "zipf_s": 1.1, "key_ids": 1 << log_keys,
                       "l2": "inputs larger than L2, flushed between steps"}

    def setup_gpu(self, ctx):
        import torch
        self.tA = ctx.table(self.A.vars, [torch.from_numpy(c).cuda() for c in self.A.cols])
        self.tB = ctx.table(self.B.vars, [torch.from_numpy(c).cuda() for c in self.B.cols])

    def run_gpu(self, ctx):
        t = ctx.join(self.tA, self.tB)
        n = t.nrows
        t.free()
        return n

    def run_e2e(self, ctx):
        if not hasattr(self, "hA"):  # the inputs in pinned host memory (setup, not timed)
            self.hA = [PINNED.copy_of(("A", i), c) for i, c in enumerate(self.A.cols)]
            self.hB = [PINNED.copy_of(("B", i), c) for i, c in enumerate(self.B.cols)]
        tA = ctx.table(self.A.vars, self.hA)
        tB = ctx.table(self.B.vars, self.hB)
        t = ctx.join(tA, tB)
        vars_, cols = t.to_host(PINNED.out(len(t.vars), t.nrows))
        n = t.nrows
        h2d = sum(c.nbytes for c in self.A.cols + self.B.cols)
        d2h = sum(c.nbytes for c in cols)
        for x in (t, tA, tB):
            x.free()
        return n, h2d, d2h

    def alg_bytes(self, rows):
        """Compulsory bytes of one join: both inputs read once, the output written once."""
        return 4 * (self.A.nrows * 4 + self.B.nrows * 4) + 4 * rows * 6

    ORACLE_BUCKETS = 1024  # oracle units: the keys whose x has the same top 10 bits

    def run_oracle(self, sample_index, budget_s=2.0):
        """The oracle on one key bucket: the rows of A and B whose keys fall in
        it, joined (the bucket's share of the whole join's output)."""
        import oracle
        if not hasattr(self, "_parts"):  # rows grouped by bucket, once (not timed)
            nb = self.ORACLE_BUCKETS
            shift = np.uint32(32 - int(np.log2(nb)))
            self._parts = []
            for T in (self.A, self.B):
                b = (T.cols[0] >> shift).astype(np.uint16)
                order = np.argsort(b, kind="stable")  # a radix sort for 16-bit keys
                cut = np.searchsorted(b[order], np.arange(nb + 1))
                self._parts.append((T, [c[order] for c in T.cols], cut))
        k = sample_index % self.ORACLE_BUCKETS
        (TA, ca, cuta), (TB, cb, cutb) = self._parts
        A = gen.Table(TA.vars, [c[cuta[k]:cuta[k + 1]] for c in ca])
        B = gen.Table(TB.vars, [c[cutb[k]:cutb[k + 1]] for c in cb])
        return oracle.join_mapreduce(A, B)[1].shape[0], 1


class PairwiseUniform(Workload):
    name = "pairwise_uniform"
    oracle_unit = "whole joins"

    def alg_bytes(self, rows):
        return 4 * (self.L.nrows * 2 + self.R.nrows * 2) + 12 * rows

    def __init__(self):
        self.L, self.R = gen.pairwise_uniform(seed=1)
        self.config = {"workload": "pairwise_uniform", "rows_left": 16384, "rows_right": 8192, "key_ids": 4096,
                       "l2": "flushed between steps"}

    def setup_gpu(self, ctx):
        import torch
        self.tL = ctx.table(self.L.vars, [torch.from_numpy(c).cuda() for c in self.L.cols])
        self.tR = ctx.table(self.R.vars, [torch.from_numpy(c).cuda() for c in self.R.cols])

    def run_gpu(self, ctx):
        t = ctx.join(self.tL, self.tR)
        n = t.nrows
        t.free()
        return n

    def run_e2e(self, ctx):
        if not hasattr(self, "hL"):  # the inputs in pinned host memory (setup, not timed)
            self.hL = [PINNED.copy_of(("L", i), c) for i, c in enumerate(self.L.cols)]
            self.hR = [PINNED.copy_of(("R", i), c) for i, c in enumerate(self.R.cols)]
        tL = ctx.table(self.L.vars, self.hL)
        tR = ctx.table(self.R.vars, self.hR)
        t = ctx.join(tL, tR)
        vars_, cols = t.to_host(PINNED.out(len(t.vars), t.nrows))
        n = t.nrows
        for x in (t, tL, tR):
            x.free()
        return n, sum(c.nbytes for c in self.L.cols + self.R.cols), sum(c.nbytes for c in cols)

    def run_oracle(self, sample_index, budget_s=2.0):
        import oracle
        return oracle.join_mapreduce(self.L, self.R)[1].shape[0], 1


class UnevenBatch(Workload):
    """256 independent joins of uneven size (rows log-uniform in [2^8, 2^22] per
    side, 2-4 columns, left keys uniform or Zipf(0.8 / 1.2)): one step = the
    whole batch through ``mapsq_join_batch`` (every phase one launch for all
    joins); the alternative form runs the same joins one ``mapsq_join`` after
    another."""
    name = "uneven_batch"
    oracle_unit = "whole joins"

    def alg_bytes(self, rows):
        """Compulsory bytes of the batch: every input read once, every output
        written once (output bytes of the last step)."""
        ins = sum(4 * (L.nrows * len(L.cols) + R.nrows * len(R.cols)) for L, R in self.joins)
        return ins + getattr(self, "out_bytes", 0)

    def __init__(self, seed=4, n_joins=256, log_hi=22.0):
        self.joins = [(L, R) for L, R, _ in gen.uneven_batch(seed=seed, n_joins=n_joins, log_hi=log_hi)]
        self.config = {"workload": "uneven_batch", "joins": n_joins, "rows_per_side": f"2^U[8,{log_hi:g}]",
                       "columns": "2-4", "zipf_s": "0 / 0.8 / 1.2 per join", "seed": seed,
                       "form": "mapsq_join_batch (all joins in one batch)",
                       "l2": "inputs larger than L2, flushed between steps"}

    def setup_gpu(self, ctx):
        import torch
        self.dev = [(ctx.table(L.vars, [torch.from_numpy(c).cuda() for c in L.cols]),
                     ctx.table(R.vars, [torch.from_numpy(c).cuda() for c in R.cols])) for L, R in self.joins]

    def run_gpu(self, ctx):
        rows = out = 0
        for t in ctx.join_batch([a for a, _ in self.dev], [b for _, b in self.dev]):
            rows += t.nrows
            out += 4 * t.nrows * len(t.vars)
            t.free()
        self.out_bytes = out
        return rows

    def run_gpu_alt(self, ctx):
        rows = 0
        for a, b in self.dev:
            t = ctx.join(a, b)
            rows += t.nrows
            t.free()
        return rows

    alt_form = "plain: the same 256 joins one mapsq_join after another"

    def run_e2e(self, ctx):
        if not hasattr(self, "hosts"):  # the inputs in pinned host memory (setup, not timed)
            self.hosts = [([PINNED.copy_of(("L", j, i), c) for i, c in enumerate(L.cols)],
                           [PINNED.copy_of(("R", j, i), c) for i, c in enumerate(R.cols)])
                          for j, (L, R) in enumerate(self.joins)]
        tabs = [(ctx.table(L.vars, hl), ctx.table(R.vars, hr)) for (L, R), (hl, hr) in zip(self.joins, self.hosts)]
        h2d = sum(c.nbytes for L, R in self.joins for c in L.cols + R.cols)
        rows = d2h = 0
        for t in ctx.join_batch([a for a, _ in tabs], [b for _, b in tabs]):
            vars_, cols = t.to_host(PINNED.out(len(t.vars), t.nrows))
            d2h += sum(c.nbytes for c in cols)
            rows += t.nrows
            t.free()
        for a, b in tabs:
            a.free()
            b.free()
        return rows, h2d, d2h

    def run_oracle(self, sample_index, budget_s=2.0):
        import oracle
        rows, done, t0 = 0, 0, time.perf_counter()
        k = sample_index
        while time.perf_counter() - t0 < budget_s and done < len(self.joins):
            L, R = self.joins[k % len(self.joins)]
            rows += oracle.join_mapreduce(L, R)[1].shape[0]
            k += 1
            done += 1
        return rows, done


WORKLOADS = {"university_bgp": UniversityBGP, "skewed_join": SkewedJoin, "pairwise_uniform": PairwiseUniform,
             "uneven_batch": UnevenBatch}


class Serving(UniversityBGP):
    """Served form: a Poisson stream of BGP queries (mean ``rate`` per second,
    3-8 patterns, star and chain, 1-2 constants, drawn from a pool of witness
    BGPs) over a device-resident university graph of 1e8 triples, evaluated by
    the library's serving loop with continuous batching and a 40 GB budget for
    the tables in flight.  One step = ``step_s`` seconds of arrivals."""
    name = "serving"
    oracle_unit = "queries of the stream"

    def __init__(self, n_triples=100_000_000, pool=2048, seed=5, rate=2000.0, step_s=1.5, budget=40 << 30):
        self.s, self.p, self.o = gen.university_graph(n_triples, seed=2)
        g = GraphIndex(self.s, self.p, self.o)
        self.bgps = [b["patterns"] for b in generate_bgps(g, pool, seed=seed, k_range=(3, 8), var_range=None)]
        del g
        self.seed, self.rate, self.step_s, self.budget = seed, rate, step_s, budget
        self.config = {"workload": "serving", "triples": n_triples, "predicates": 18, "arrivals": "Poisson",
                       "rate_qps": rate, "step_s": step_s, "patterns_per_bgp": "3-8", "bgp_pool": pool,
                       "bgp_seed": seed, "mem_budget_gb": budget / (1 << 30), "max_active": 256,
                       "l2": "store (1e8 triples, 1.6 GB) larger than L2"}
        self._graph_set = None

    def stream(self, n_steps, part):
        """Arrival offsets (s) and pool indices of ``n_steps`` steps of arrivals."""
        r = gen.Rng(self.seed, 100 + part)
        n = int(self.rate * self.step_s * n_steps * 1.3) + 64
        t = np.cumsum(-np.log1p(-r.unit(n)) / self.rate)
        t = t[t < n_steps * self.step_s]
        return t, r.below(t.shape[0], len(self.bgps))

    def serve(self, ctx, n_steps, part, to_host=False):
        """Serve one stream; returns (rows, seconds, device ms, h2d, d2h, counters)."""
        import torch
        arrivals, idx = self.stream(n_steps, part)
        ctx.serve_start(max_active=256, mem_budget_bytes=self.budget)
        tickets = []
        h2d = [0]

        def producer():
            t0 = time.perf_counter()
            for a, i in zip(arrivals.tolist(), idx.tolist()):
                wait = t0 + a - time.perf_counter()
                if wait > 0:
                    time.sleep(wait)
                b = self.bgps[i]
                tickets.append(ctx.submit(b))
                h2d[0] += 16 * len(b)

        stream = torch.cuda.current_stream()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        th = threading.Thread(target=producer)
        ev0.record(stream)
        w0 = time.perf_counter()
        th.start()
        rows = d2h = seen = failed = 0
        pending = []
        while th.is_alive() or seen < len(tickets) or pending:
            while seen < len(tickets):
                pending.append(tickets[seen])
                seen += 1
            still = []
            for tk in pending:
                try:
                    res = ctx.poll(tk)
                except Exception:
                    failed += 1
                    continue
                if res is None:
                    still.append(tk)
                    continue
                rows += res.nrows
                if to_host:
                    _, cols = res.to_host(PINNED.out(len(res.vars), res.nrows))
                    d2h += sum(c.nbytes for c in cols)
                res.free()
            pending = still
            time.sleep(0.0005)
        th.join()
        ev1.record(stream)
        ev1.synchronize()
        wall = time.perf_counter() - w0
        counters = ctx.serve_stats()
        ctx.serve_stop()
        counters["poll_failed"] = failed
        return rows, wall, ev0.elapsed_time(ev1), h2d[0], d2h, counters, idx

    def burst(self, ctx, idx):
        """Every query of ``idx`` submitted at once (the serving loop saturated):
        returns (rows, seconds, counters)."""
        ctx.serve_start(max_active=256, mem_budget_bytes=self.budget)
        t0 = time.perf_counter()
        tickets = [ctx.submit(self.bgps[i]) for i in idx.tolist()]
        rows, pending = 0, tickets
        while pending:
            still = []
            for tk in pending:
                res = ctx.poll(tk)
                if res is None:
                    still.append(tk)
                else:
                    rows += res.nrows
                    res.free()
            pending = still
            time.sleep(0.0005)
        dt = time.perf_counter() - t0
        counters = ctx.serve_stats()
        ctx.serve_stop()
        return rows, dt, counters

    def run_serial(self, ctx, idx, budget_s=8.0):
        """The same queries one mapsq_query after another (bounded sample)."""
        import torch
        stream = torch.cuda.current_stream()
        rows, n, ms = 0, 0, 0.0
        t0 = time.perf_counter()
        for i in idx.tolist():
            if time.perf_counter() - t0 > budget_s:
                break
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            t = ctx.query(self.bgps[i])
            rows += t.nrows
            t.free()
            b.record(stream)
            b.synchronize()
            ms += a.elapsed_time(b)
            n += 1
        return rows, n, ms

    def run_oracle(self, sample_index, budget_s=2.0):
        import oracle
        if self._graph_set is None:
            self._graph_set = oracle.distinct_triples(self.s, self.p, self.o)
        _, idx = self.stream(1, 0)
        rows, done, t0 = 0, 0, time.perf_counter()
        k = sample_index
        while time.perf_counter() - t0 < budget_s and done < idx.shape[0]:
            b = self.bgps[int(idx[k % idx.shape[0]])]
            rows += oracle.evaluate_bgp(self._graph_set, b, is_set=True)[1].shape[0]
            k += 1
            done += 1
        return rows, done


WORKLOADS["serving"] = Serving


def _oracle_worker(job):
    """One host process of the all-cores oracle baseline: builds the workload
    from its seeds, then runs the oracle on its share of samples for ``budget_s``."""
    workload, size, first, stride, budget_s = job
    import types
    w = make_workload(types.SimpleNamespace(workload=workload, size=size))
    w.run_oracle(first, budget_s=0.0)  # one-off setup (the oracle's triple set), not timed
    rows, units, k, t0 = 0, 0, first, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        r, u = w.run_oracle(k, budget_s=budget_s - (time.perf_counter() - t0))
        rows += r
        units += u
        k += stride
    return rows, units, time.perf_counter() - t0


def oracle_all_cores(args, budget_s=10.0):
    """The oracle on every host core (one process per core, spawned), each on its
    own samples of the workload; returns (bindings/s, cores, units)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    jobs = [(args.workload, args.size, i, cores, budget_s) for i in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_worker, jobs)
    rows = sum(r for r, _, _ in res)
    units = sum(u for _, u, _ in res)
    return rows / max(dt for _, _, dt in res), cores, units


def autotune_summary(tune):
    """The autotuner's choices and the times they come from (ms, best of three)."""
    if tune.get("fixed"):
        return tune
    return {"sorted_ratio": tune["sorted_ratio"],
            "points": [(p["ratio"], round(p["hash_ms"], 3), round(p["sorted_ms"], 3)) for p in tune["points"]],
            "partitioned_build_from_rows": tune["part_min_build"],
            "size_points": [(p["build_rows"], round(p["partitioned_ms"], 3), round(p["plain_ms"], 3))
                            for p in tune["size_points"]],
            "dense_write_up_to_matches": tune["dense_max"],
            "skew_points": [(p["group_rows"], round(p["dense_ms"], 3), round(p["partitioned_write_ms"], 3))
                            for p in tune["skew_points"]]}


def tuned(ctx, args):
    """The hash-vs-sorted crossover for this GPU: measured (not timed), or fixed."""
    if args.sorted_ratio:
        ctx.set_sorted_ratio(args.sorted_ratio)
        return {"sorted_ratio": args.sorted_ratio, "points": [], "fixed": True}
    return ctx.autotune()


def make_workload(args):
    if args.size == "small":
        if args.workload == "skewed_join":
            return SkewedJoin(log_a=24, log_b=22, log_keys=20)
        if args.workload == "uneven_batch":
            return UnevenBatch(log_hi=20.0)
        raise SystemExit("--size small exists for skewed_join and uneven_batch only")
    return WORKLOADS[args.workload]()


# ---------------------------------------------------------------- helpers

def combine_ranks(total_ms, rows, world, device):
    """Whole-job figures of N independent replicas: the slowest rank's timed
    milliseconds and the sum of every rank's rows (max / sum all-reduces over
    the default process group; ``device`` holds the tensors: a GPU for NCCL,
    the CPU for gloo)."""
    if world == 1:
        return total_ms, rows
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    r = torch.tensor([float(rows)], dtype=torch.float64, device=device)
    dist.all_reduce(r)
    return float(t.item()), float(r.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t0 = time.perf_counter()  # sampling is live before the timed region starts
            while not self.lines and time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        # the first sample was taken before the timed region: keep it only if it is the only one
        lines = self.lines[1:] if len(self.lines) > 1 else self.lines
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for name, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_traffic(kernel, workload):
    """DRAM bytes per launch of ``kernel`` from a committed ncu summary, if the
    summary was taken from the current kernel sources (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if ":" in line and line.startswith("- "):
            k, v = line[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    src = os.path.join(ROOT, "paper_1702_03484_gb300", "csrc", fields.get("source", "join.cu"))
    if not os.path.exists(src):
        return None
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if fields.get("source_sha256") != digest:
        return None
    try:
        return float(fields["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# ---------------------------------------------------------------- arms

_REF = None  # the workload of a reference-arm worker process


def _ref_init(workload, size):
    global _REF
    import types
    _REF = make_workload(types.SimpleNamespace(workload=workload, size=size))
    _REF.run_oracle(0, budget_s=0.0)  # one-off setup (the oracle's triple set)


def _ref_config(_):
    return _REF.name, _REF.config, _REF.oracle_unit


def _ref_sample(job):
    """Oracle units from ``first`` on (every ``stride``-th) for about ``budget_s``."""
    first, stride, budget_s = job
    rows, units, k, t0 = 0, 0, first, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        r, u = _REF.run_oracle(k, budget_s=budget_s - (time.perf_counter() - t0))
        rows += r
        units += u
        k += stride
    return rows, units


def run_reference(args):
    """The reference arm: the oracle as it stands on the host's cores, one
    spawned process per core (at most 4 for the 1e8-triple serving graph, for
    memory), each on its own bounded samples of the workload per step."""
    import multiprocessing as mp
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    if args.workload == "serving":
        cores = min(cores, 4)
    with mp.get_context("spawn").Pool(cores, initializer=_ref_init, initargs=(args.workload, args.size)) as pool:
        name, config, unit_desc = pool.map(_ref_config, [0])[0]
        for i in range(args.warmup):
            pool.map(_ref_sample, [(i * cores + c, cores * (args.warmup + args.steps), 0.5) for c in range(cores)])
        rows, units, t0 = 0, 0, time.perf_counter()
        for i in range(args.steps):
            res = pool.map(_ref_sample, [((args.warmup + i) * cores + c, cores * (args.warmup + args.steps), 2.0)
                                         for c in range(cores)])
            rows += sum(r for r, _ in res)
            units += sum(u for _, u in res)
        dt = time.perf_counter() - t0
    value = rows / dt
    sample = (f"per step about 2 s of the {name} workload on each of {cores} host processes ({units} units in "
              f"{args.steps} steps; units: {unit_desc}), oracle in numpy")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": config,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_steps(w, ctx, fn, steps, flush, stream):
    """``steps`` calls of ``fn(ctx)``, each bracketed by CUDA events on the
    context's stream, the L2 flushed before each (outside the events).  Returns
    (total ms, rows, per-step ms)."""
    import torch
    total_ms, rows, step_ms = 0.0, 0, []
    for _ in range(steps):
        flush.fill_(1)  # evict the L2 between timed steps (not timed)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rows += fn(ctx)
        b.record(stream)
        b.synchronize()
        step_ms.append(a.elapsed_time(b))
        total_ms += step_ms[-1]
    return total_ms, rows, step_ms


def kernel_roofline(ctx, w, fn, steps, flush, stream, peak, peak_kind):
    """The dominant kernel's roofline, measured in its own pass after the timed
    steps: one step profiled in full names the kernel with the most device time,
    then ``steps`` steps time that kernel alone (CUDA events around each of its
    launches, on the launching stream).  Returns (roofline, per-kernel table of
    the fully profiled step)."""
    ctx.reset_stats()
    ctx.set_profiling(True)
    fn(ctx)
    full = ctx.kernel_stats()
    ctx.set_profiling(False)
    if not full:
        return None, {}
    dominant = max(full.items(), key=lambda kv: kv[1]["device_ms"])[0]
    ctx.reset_stats()
    ctx.profile_only(dominant)
    ctx.set_profiling(True)
    timed_steps(w, ctx, fn, steps, flush, stream)
    st = ctx.kernel_stats()[dominant]
    ctx.set_profiling(False)
    ctx.profile_only(None)
    per_launch_s = st["device_ms"] / 1000.0 / st["launches"]
    achieved = st["alg_bytes"] / st["launches"] / per_launch_s / 1e9
    total = sum(v["device_ms"] for v in full.values())
    roof = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak,
            "peak_kind": f"{peak_kind} copy bandwidth", "unit": "GB/s", "frac": achieved / peak,
            "traffic": ncu_traffic(dominant, w.name), "launches": st["launches"],
            "alg_bytes_per_launch": st["alg_bytes"] / st["launches"],
            "ms_per_launch": per_launch_s * 1000.0, "share_of_device_time": full[dominant]["device_ms"] / total}
    table = {k: {"launches": v["launches"], "ms": round(v["device_ms"], 4)} for k, v in full.items()}
    return roof, table


def measure(ctx, w, args, flush, stream, peak, peak_kind, steps, e2e_steps):
    """One workload of the line's ``other_workloads``: warm-up, ``steps`` timed
    steps, then the passes of ``measure_rest``."""
    import torch
    for _ in range(args.warmup):
        w.run_gpu(ctx)
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    total_ms, rows, step_ms = timed_steps(w, ctx, w.run_gpu, steps, flush, stream)
    launches = ctx.launch_count() - launches0
    res = {"value": rows / (total_ms / 1000.0), "unit": UNIT, "ms_per_step": total_ms / steps,
           "rows_per_step": rows / steps, "step_ms_p50": float(np.percentile(step_ms, 50)),
           "step_ms_p99": float(np.percentile(step_ms, 99)), "gpu_launches": launches}
    if hasattr(w, "alg_bytes"):
        res["roofline_whole_step"] = whole_step_roofline(w, rows / steps, total_ms / steps, peak)
    res.update(measure_rest(ctx, w, steps, e2e_steps, flush, stream, peak, peak_kind))
    return res


def whole_step_roofline(w, rows_per_step, ms_per_step, peak):
    alg = w.alg_bytes(rows_per_step)
    achieved = alg / (ms_per_step / 1000.0) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "alg_bytes_per_step": alg,
            "what": "compulsory bytes of the whole step (inputs read once, output written once) / step time, "
                    "every kernel included"}


EXTRAS = ("uneven_batch", "university_bgp", "pairwise_uniform")


def measure_serving_short(ctx, steps=2, pool=256):
    """A short served stream over the 1e8-triple graph (the serving config with
    a smaller BGP pool and ``steps`` x 1.5 s of Poisson arrivals at 2000
    queries/s): latency percentiles, throughput, and the same queries one
    mapsq_query after another (2 s sample)."""
    w = Serving(pool=pool)
    w.setup_gpu(ctx)
    w.serve(ctx, 1, part=1)  # warm-up stream
    rows, wall, dev_ms, _, _, counters, idx = w.serve(ctx, steps, part=2)
    s_rows, s_n, s_ms = w.run_serial(ctx, idx, budget_s=2.0)
    res = {"value": rows / (dev_ms / 1000.0), "unit": UNIT, "queries": counters["submitted"],
           "completed": counters["completed"], "failed": counters["failed"], "p50_ms": counters["p50_ms"],
           "p99_ms": counters["p99_ms"], "mean_ms": counters["mean_ms"], "achieved_qps": counters["submitted"] / wall,
           "rounds": counters["rounds"], "batched_joins": counters["batched_joins"],
           "preempted": counters["preempted"], "wall_s": wall,
           "serial_plain": {"value": s_rows / (s_ms / 1000.0) if s_ms else None, "unit": UNIT, "queries": s_n,
                            "ms_per_query": s_ms / max(s_n, 1)},
           "config": dict(w.config, bgp_pool=pool, steps=steps),
           "form": "mapsq_serve_*: continuous batching of the queries in flight, 40 GB admission budget"}
    w.release(ctx)
    return res


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1702_03484_gb300 import Context

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = make_workload(args)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
    peak, peak_kind = measured_peaks()

    def barrier():
        if world > 1:
            dist.barrier()

    with Context(device=local) as ctx:
        w.setup_gpu(ctx)
        tune = tuned(ctx, args)
        stream = torch.cuda.current_stream(dev)
        for _ in range(args.warmup):
            w.run_gpu(ctx)
        launches0 = ctx.launch_count()
        barrier()
        torch.cuda.synchronize()
        # clocks are sampled over the timed steps and the passes after them
        with ClockSampler(local) as clocks:
            total_ms, rows, step_ms = timed_steps(w, ctx, w.run_gpu, args.steps, flush, stream)
            torch.cuda.synchronize()
            barrier()
            launches = ctx.launch_count() - launches0
            head = measure_rest(ctx, w, args.steps, max(1, min(args.steps, 5)), flush, stream, peak, peak_kind)
        extras = {}
        if args.workload == "skewed_join" and args.size == "full" and not args.no_extras and world == 1:
            w.release(ctx)
            for name in EXTRAS:
                x = WORKLOADS[name]()
                x.setup_gpu(ctx)
                r = measure(ctx, x, args, flush, stream, peak, peak_kind, steps=min(args.steps, 10),
                            e2e_steps=2)
                r["config"] = x.config
                for k in ("total_ms", "rows"):
                    r.pop(k, None)
                if "other_form" in r:
                    r["other_over_this"] = r["other_form"]["value"] / r["value"]
                extras[name] = r
                x.release(ctx)
            extras["serving"] = measure_serving_short(ctx)

    t_max, rows_all = combine_ranks(total_ms, rows, world, dev)
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return
    value = rows_all / (t_max / 1000.0)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic", "config": w.config,
            "rows_per_step": rows / args.steps,
            "step_ms_p50": float(np.percentile(step_ms, 50)), "step_ms_p99": float(np.percentile(step_ms, 99)),
            "e2e": head["e2e"], "gpu_launches": launches, "roofline": head["roofline"],
            "clocks": clocks.summary()}
    if hasattr(w, "alg_bytes"):
        line["roofline_whole_step"] = whole_step_roofline(w, rows / args.steps, t_max / args.steps, peak)
    if "other_form" in head:
        line["other_form"] = head["other_form"]
    line.update({
        "store_build": ({"seconds": w.store_build_s, "triples_per_s": len(w.s) / w.store_build_s}
                        if hasattr(w, "store_build_s") else None),
        "autotune": autotune_summary(tune),
        "kernels_one_step": head["kernels_one_step"]})
    if extras:
        line["other_workloads"] = extras
    if not args.no_cpu_baseline and world == 1:
        t0 = time.perf_counter()
        crow, cunits = 0, 0
        k = 0
        w.run_oracle(0, budget_s=0.0)  # one-off setup of the oracle's inputs, not timed
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 15.0:
            r, u = w.run_oracle(k, budget_s=15.0 - (time.perf_counter() - t0))
            crow += r
            cunits += u
            k += u
        cdt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": crow / cdt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{cunits} units of the {w.name} workload ({w.oracle_unit}) in "
                                          f"{cdt:.1f} s, numpy oracle, single thread"}
        v, cores, units = oracle_all_cores(args)
        line["cpu_baseline_all_cores"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                          "sample": f"{units} units of the {w.name} workload ({w.oracle_unit}), "
                                                    f"one spawned process per core for about 10 s each"}
    print(json.dumps(line), flush=True)


def measure_rest(ctx, w, steps, e2e_steps, flush, stream, peak, peak_kind):
    """After a workload's timed steps, each in its own pass: the other form
    (batched or plain) when the workload has one, end to end through host
    buffers, and the dominant kernel's roofline."""
    import torch
    res = {}
    if hasattr(w, "run_gpu_alt"):
        for _ in range(2):
            w.run_gpu_alt(ctx)
        bms, brows, bstep = timed_steps(w, ctx, w.run_gpu_alt, steps, flush, stream)
        res["other_form"] = {"value": brows / (bms / 1000.0), "unit": UNIT, "ms_per_step": bms / steps,
                             "step_ms_p50": float(np.percentile(bstep, 50)),
                             "step_ms_p99": float(np.percentile(bstep, 99)), "form": w.alt_form}
    for _ in range(2):
        w.run_e2e(ctx)
    torch.cuda.synchronize()
    e_rows, h2d, d2h = 0, 0, 0
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        r, hi, ho = w.run_e2e(ctx)
        e_rows += r
        h2d += hi
        d2h += ho
    torch.cuda.synchronize()
    e_dt = time.perf_counter() - t0
    res["e2e"] = {"value": e_rows / e_dt, "unit": UNIT, "h2d_bytes_per_step": h2d // e2e_steps,
                  "d2h_bytes_per_step": d2h // e2e_steps}
    res["roofline"], res["kernels_one_step"] = kernel_roofline(ctx, w, w.run_gpu, steps, flush, stream,
                                                               peak, peak_kind)
    return res


def run_serving(args):
    """The served form: Poisson arrivals through mapsq_submit / mapsq_poll."""
    import torch
    from paper_1702_03484_gb300 import Context

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    w = Serving()
    with Context(device=local) as ctx:
        w.setup_gpu(ctx)
        tune = tuned(ctx, args)
        # warm-up stream, profiled in full: it names the kernel with the most device time
        ctx.reset_stats()
        ctx.set_profiling(True)
        w.serve(ctx, max(1, args.warmup // 2), part=1)
        warm_stats = ctx.kernel_stats()
        ctx.set_profiling(False)
        dominant = max(warm_stats.items(), key=lambda kv: kv[1]["device_ms"])[0] if warm_stats else None
        launches0 = ctx.launch_count()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clocks:
            rows, wall, dev_ms, _, _, counters, idx = w.serve(ctx, args.steps, part=2)
        torch.cuda.synchronize()
        launches = ctx.launch_count() - launches0
        # the dominant kernel timed alone, on a separate stream of arrivals after the timed one
        ctx.reset_stats()
        ctx.profile_only(dominant)
        ctx.set_profiling(True)
        w.serve(ctx, max(1, args.warmup // 2), part=4)
        stats = ctx.kernel_stats()
        ctx.set_profiling(False)
        ctx.profile_only(None)
        # the same stream's queries one after another (bounded sample)
        s_rows, s_n, s_ms = w.run_serial(ctx, idx)
        # saturation: the first 8000 of them submitted at once
        b_idx = idx[:8000]
        b_rows, b_dt, b_counters = w.burst(ctx, b_idx)
        # end to end: a shorter stream whose every result is copied to the host
        e_steps = max(1, min(args.steps, 4))
        e_rows, e_wall, _, h2d, d2h, e_counters, _ = w.serve(ctx, e_steps, part=3, to_host=True)

    t_max, rows_all = combine_ranks(dev_ms, rows, world, "cuda")
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return
    peak, peak_kind = measured_peaks()
    roofline = None
    if stats:
        name, st = max(stats.items(), key=lambda kv: kv[1]["device_ms"])
        per_launch_s = st["device_ms"] / 1000.0 / st["launches"]
        achieved = st["alg_bytes"] / st["launches"] / per_launch_s / 1e9
        roofline = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak,
                    "peak_kind": f"{peak_kind} copy bandwidth", "unit": "GB/s", "frac": achieved / peak,
                    "traffic": ncu_traffic(name, w.name), "launches": st["launches"],
                    "alg_bytes_per_launch": st["alg_bytes"] / st["launches"],
                    "share_of_device_time": warm_stats[name]["device_ms"] / sum(v["device_ms"]
                                                                                for v in warm_stats.values())}
    line = {"metric": METRIC, "value": rows_all / (t_max / 1000.0), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": w.config,
            "serving": {"queries": counters["submitted"], "completed": counters["completed"],
                        "failed": counters["failed"], "p50_ms": counters["p50_ms"], "p99_ms": counters["p99_ms"],
                        "mean_ms": counters["mean_ms"], "rounds": counters["rounds"],
                        "batched_joins": counters["batched_joins"], "preempted": counters["preempted"],
                        "achieved_qps": counters["submitted"] / wall, "wall_s": wall},
            "serial_plain": {"value": s_rows / (s_ms / 1000.0) if s_ms else None, "unit": UNIT, "queries": s_n,
                             "ms_per_query": s_ms / max(s_n, 1), "qps": 1000.0 * s_n / s_ms if s_ms else None,
                             "form": "the same stream's queries one mapsq_query after another"},
            "saturated": {"value": b_rows / b_dt, "unit": UNIT, "queries": int(b_idx.shape[0]),
                          "qps": b_idx.shape[0] / b_dt, "p50_ms": b_counters["p50_ms"],
                          "p99_ms": b_counters["p99_ms"], "rounds": b_counters["rounds"],
                          "form": "the stream's first queries submitted at once (wall clock to the last result)"},
            "e2e": {"value": e_rows / e_wall, "unit": UNIT, "h2d_bytes_per_step": h2d // e_steps,
                    "d2h_bytes_per_step": d2h // e_steps, "p50_ms": e_counters["p50_ms"],
                    "p99_ms": e_counters["p99_ms"]},
            "gpu_launches": launches, "roofline": roofline, "clocks": clocks.summary(),
            "autotune": {"sorted_ratio": tune["sorted_ratio"]},
            "store_build": {"seconds": w.store_build_s, "triples_per_s": len(w.s) / w.store_build_s},
            "kernels_warmup_stream": {k: {"launches": v["launches"], "ms": round(v["device_ms"], 4)}
                                      for k, v in warm_stats.items()}}
    if not args.no_cpu_baseline and world == 1:
        w.run_oracle(0, budget_s=0.0)  # builds the oracle's triple set, not timed
        t0 = time.perf_counter()
        crow, cunits, k = 0, 0, 0
        while time.perf_counter() - t0 < 15.0:
            r, u = w.run_oracle(k, budget_s=15.0 - (time.perf_counter() - t0))
            crow += r
            cunits += u
            k += u
        cdt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": crow / cdt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{cunits} queries of the serving stream in {cdt:.1f} s, evaluated "
                                          f"one after another by the numpy oracle, single thread"}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serving":
        run_serving(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
