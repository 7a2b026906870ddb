"""Oracle work items run in spawned host processes by the full-size parity
tests (test infrastructure; no device code).  Each job takes plain arrays and
returns the oracle's table as (vars, rows)."""
import os

import numpy as np

import gen
import oracle

_GRAPH = None


def join_job(job):
    """oracle.join_mapreduce of two tables given as (vars, columns) pairs."""
    (lv, lc), (rv, rc) = job
    return oracle.join_mapreduce(gen.Table(list(lv), list(lc)), gen.Table(list(rv), list(rc)))


def save_split_graph(split, path):
    """Write a graph split by predicate (oracle.split_by_predicate) to ``path``
    as .npy files that the workers map read-only."""
    os.makedirs(path, exist_ok=True)
    keys = np.array(sorted(split), np.int64)
    np.save(os.path.join(path, "preds.npy"), keys)
    for k in keys.tolist():
        for name, arr in zip("spo", split[k]):
            np.save(os.path.join(path, f"{name}{k}.npy"), arr)


def load_split_graph(path):
    """Pool initializer: map the split graph written by save_split_graph."""
    global _GRAPH
    keys = np.load(os.path.join(path, "preds.npy")).tolist()
    _GRAPH = {k: tuple(np.load(os.path.join(path, f"{n}{k}.npy"), mmap_mode="r") for n in "spo") for k in keys}


def bgp_job(bgp):
    """oracle.evaluate_bgp of one BGP over the mapped graph, canonical form."""
    return oracle.canonical(oracle.evaluate_bgp(_GRAPH, [tuple(x) for x in bgp]))
