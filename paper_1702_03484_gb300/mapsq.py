"""Python binding of libmapsq (ctypes): argument marshalling only.

Every function named ``mapsq_*`` here calls the C entry point of the same name
declared in ``include/mapsq.h`` and raises :class:`MapsqError` on a negative
status.  :class:`Context` and :class:`TableRef` are thin conveniences over
them.  All device work happens in the library's CUDA kernels; there is no
fallback: if ``libmapsq.so`` is missing or cannot be loaded, importing the
library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# MAPSQ_LIB selects another build of the library (libmapsq_checked.so: the
# kernels check their device indexes)
LIB_PATH = os.environ.get("MAPSQ_LIB") or os.path.join(_HERE, "libmapsq.so")

MAX_VARS = 16
VAR_S, VAR_P, VAR_O = 1, 2, 4
JOIN_AUTO, JOIN_HASH, JOIN_SORTED = 0, 1, 2
DISTINCT = 1

STATUS = {
    0: "OK", -1: "INVALID", -2: "UNSUPPORTED", -3: "OOM", -4: "BUDGET",
    -5: "CUDA", -6: "TIMEOUT", -7: "BUSY", -8: "NOT_FOUND",
}


class MapsqError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{STATUS.get(code, code)}: {message}")
        self.code = code
        self.name = STATUS.get(code, str(code))


class Pattern(C.Structure):
    _fields_ = [("s", C.c_uint32), ("p", C.c_uint32), ("o", C.c_uint32), ("var_mask", C.c_uint32)]


class Table(C.Structure):
    _fields_ = [("nrows", C.c_uint64), ("ncols", C.c_uint32), ("var", C.c_int32 * MAX_VARS),
                ("col", C.c_void_p * MAX_VARS), ("on_device", C.c_int32), ("sorted_mask", C.c_uint32)]


class JoinOpts(C.Structure):
    _fields_ = [("algorithm", C.c_int32), ("reserved", C.c_int32 * 3)]


class AutotuneResult(C.Structure):
    _fields_ = [("sorted_ratio", C.c_uint32), ("points", C.c_uint32), ("ratio", C.c_uint32 * 12),
                ("hash_ms", C.c_double * 12), ("sorted_ms", C.c_double * 12), ("sorted_rows", C.c_uint64),
                ("part_min_build", C.c_uint64), ("part_points", C.c_uint32), ("dense_max", C.c_uint32),
                ("part_rows", C.c_uint64 * 6), ("part_on_ms", C.c_double * 6), ("part_off_ms", C.c_double * 6),
                ("dense_points", C.c_uint32), ("group", C.c_uint32 * 6), ("dense_ms", C.c_double * 6),
                ("partitioned_ms", C.c_double * 6)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


class KernelStat(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_uint64), ("device_ms", C.c_double),
                ("alg_bytes", C.c_double)]


class ServeOpts(C.Structure):
    _fields_ = [("max_active", C.c_uint32), ("reserved0", C.c_uint32), ("mem_budget_bytes", C.c_uint64),
                ("reserved", C.c_uint64 * 4)]


class ServeCounters(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("in_flight", C.c_uint64), ("rounds", C.c_uint64), ("batched_joins", C.c_uint64),
                ("result_rows", C.c_uint64), ("preempted", C.c_uint64), ("p50_ms", C.c_double),
                ("p99_ms", C.c_double), ("mean_ms", C.c_double)]


_P = C.c_void_p
_TP = C.POINTER(Table)
_SIGNATURES = {
    "mapsq_create": (C.c_int, [C.POINTER(_P), C.c_int, C.POINTER(Allocator), _P, C.c_uint64]),
    "mapsq_destroy": (C.c_int, [_P]),
    "mapsq_set_stream": (C.c_int, [_P, _P]),
    "mapsq_last_error": (C.c_char_p, [_P]),
    "mapsq_strerror": (C.c_char_p, [C.c_int]),
    "mapsq_build_info": (C.c_char_p, []),
    "mapsq_load_triples": (C.c_int, [_P, _P, _P, _P, C.c_uint64, C.c_int]),
    "mapsq_store_info": (C.c_int, [_P, C.POINTER(C.c_uint64), C.POINTER(C.c_uint32)]),
    "mapsq_scan_pattern": (C.c_int, [_P, C.POINTER(Pattern), C.POINTER(_TP)]),
    "mapsq_join": (C.c_int, [_P, _TP, _TP, C.POINTER(_TP), C.POINTER(JoinOpts)]),
    "mapsq_query": (C.c_int, [_P, C.POINTER(Pattern), C.c_uint32, C.POINTER(_TP)]),
    "mapsq_query_batch": (C.c_int, [_P, C.c_uint32, C.POINTER(C.POINTER(Pattern)), C.POINTER(C.c_uint32),
                                    C.POINTER(_TP)]),
    "mapsq_join_batch": (C.c_int, [_P, C.c_uint32, C.POINTER(_TP), C.POINTER(_TP), C.POINTER(_TP),
                                   C.POINTER(JoinOpts)]),
    "mapsq_table_from_columns": (C.c_int, [_P, C.c_uint64, C.c_uint32, C.POINTER(C.c_int32), C.POINTER(_P), C.c_int,
                                           C.POINTER(_TP)]),
    "mapsq_table_to_host": (C.c_int, [_P, _TP, C.POINTER(_P)]),
    "mapsq_table_free": (None, [_P, _TP]),
    "mapsq_sync": (C.c_int, [_P]),
    "mapsq_memory_in_use": (C.c_int, [_P, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
    "mapsq_set_profiling": (C.c_int, [_P, C.c_int]),
    "mapsq_kernel_stats": (C.c_int, [_P, C.POINTER(KernelStat), C.c_uint32, C.POINTER(C.c_uint32)]),
    "mapsq_reset_stats": (C.c_int, [_P]),
    "mapsq_profile_only": (C.c_int, [_P, C.c_char_p]),
    "mapsq_launch_count": (C.c_int, [_P, C.POINTER(C.c_uint64)]),
    "mapsq_join_noalloc": (C.c_int, [_TP, _TP, C.POINTER(_P), C.c_uint64, _TP, C.POINTER(C.c_uint64), _P]),
    "mapsq_autotune": (C.c_int, [_P, C.c_uint64, C.POINTER(AutotuneResult)]),
    "mapsq_set_sorted_ratio": (C.c_int, [_P, C.c_uint32]),
    "mapsq_serve_start": (C.c_int, [_P, C.POINTER(ServeOpts)]),
    "mapsq_submit": (C.c_int, [_P, C.POINTER(Pattern), C.c_uint32, C.POINTER(C.c_uint64)]),
    "mapsq_poll": (C.c_int, [_P, C.c_uint64, C.POINTER(_TP)]),
    "mapsq_serve_stats": (C.c_int, [_P, C.POINTER(ServeCounters)]),
    "mapsq_serve_stop": (C.c_int, [_P]),
    "mapsq_join_to_host": (C.c_int, [_P, _TP, _TP, C.POINTER(JoinOpts), C.POINTER(_P), C.c_uint64,
                                     C.POINTER(C.c_uint64), _TP, C.POINTER(C.c_uint32)]),
    "mapsq_join_star": (C.c_int, [_P, C.c_uint32, C.POINTER(_TP), C.c_int32, C.POINTER(_TP)]),
    "mapsq_set_wait_limit": (C.c_int, [_P, C.c_uint32]),
    "mapsq_selftest_wait": (C.c_int, [_P, C.c_uint32]),
    "mapsq_project": (C.c_int, [_P, _TP, C.c_uint32, C.POINTER(C.c_int32), C.c_uint32, C.POINTER(_TP)]),
    "mapsq_query_select": (C.c_int, [_P, C.POINTER(Pattern), C.c_uint32, C.c_uint32, C.POINTER(C.c_int32),
                                     C.c_uint32, C.POINTER(_TP)]),
    "mapsq_dict_load": (C.c_int, [_P, C.POINTER(C.c_uint64), C.c_char_p, C.c_uint32]),
    "mapsq_decode": (C.c_int, [_P, _TP, C.c_uint32, C.POINTER(C.c_uint64), _P, C.c_uint64,
                               C.POINTER(C.c_uint64)]),
}

_lib = None


def lib():
    """The loaded libmapsq (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_1702_03484_gb300.build.build()")
        handle = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def _check(ctx, rc):
    if rc != 0:
        msg = lib().mapsq_last_error(ctx).decode() if ctx else lib().mapsq_strerror(rc).decode()
        raise MapsqError(rc, msg)


def _ptr(x):
    """Device or host address of a torch tensor / numpy array (contiguous)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return x.data_ptr()
    assert isinstance(x, np.ndarray) and x.flags.c_contiguous
    return x.ctypes.data


def _is_device(x):
    return hasattr(x, "is_cuda") and x.is_cuda


# ------------------------------------------------------------------ entry points

def mapsq_create(device=0, allocator=None, stream=None, budget=0):
    ctx = _P()
    _check(None, lib().mapsq_create(C.byref(ctx), device, C.byref(allocator) if allocator else None, stream, budget))
    return ctx


def mapsq_destroy(ctx):
    _check(None, lib().mapsq_destroy(ctx))


def mapsq_set_stream(ctx, stream):
    _check(ctx, lib().mapsq_set_stream(ctx, stream))


def mapsq_strerror(code):
    return lib().mapsq_strerror(code).decode()


def mapsq_last_error(ctx):
    return lib().mapsq_last_error(ctx).decode()


def mapsq_load_triples(ctx, s, p, o):
    n = int(s.shape[0])
    dev = _is_device(s)
    if not dev:
        s, p, o = (np.ascontiguousarray(x, dtype=np.uint32) for x in (s, p, o))
    _check(ctx, lib().mapsq_load_triples(ctx, _ptr(s), _ptr(p), _ptr(o), n, 1 if dev else 0))


def mapsq_store_info(ctx):
    n, k = C.c_uint64(), C.c_uint32()
    _check(ctx, lib().mapsq_store_info(ctx, C.byref(n), C.byref(k)))
    return n.value, k.value


def _pattern(tp):
    return Pattern(*(int(x) for x in tp))


def mapsq_scan_pattern(ctx, tp):
    out = _TP()
    _check(ctx, lib().mapsq_scan_pattern(ctx, C.byref(_pattern(tp)), C.byref(out)))
    return out


def mapsq_join(ctx, left, right, opts=None):
    out = _TP()
    _check(ctx, lib().mapsq_join(ctx, left, right, C.byref(out), C.byref(opts) if opts else None))
    return out


def mapsq_join_batch(ctx, lefts, rights, opts=None):
    k = len(lefts)
    la = (_TP * max(k, 1))(*lefts)
    ra = (_TP * max(k, 1))(*rights)
    outs = (_TP * max(k, 1))()
    _check(ctx, lib().mapsq_join_batch(ctx, k, la, ra, outs, C.byref(opts) if opts else None))
    return [outs[j] for j in range(k)]


def mapsq_query_batch(ctx, bgps):
    nq = len(bgps)
    arrs = [(Pattern * len(b))(*[_pattern(tp) for tp in b]) for b in bgps]
    ptrs = (C.POINTER(Pattern) * max(nq, 1))(*[C.cast(a, C.POINTER(Pattern)) for a in arrs])
    ns = (C.c_uint32 * max(nq, 1))(*[len(b) for b in bgps])
    outs = (_TP * max(nq, 1))()
    _check(ctx, lib().mapsq_query_batch(ctx, nq, ptrs, ns, outs))
    return [outs[q] for q in range(nq)]


def pattern_array(bgp):
    """A BGP as the C array of mapsq_pattern that mapsq_query takes (build it
    once to query the same BGP repeatedly without converting it each time)."""
    if isinstance(bgp, C.Array):
        return bgp
    return (Pattern * len(bgp))(*[_pattern(tp) for tp in bgp])


def mapsq_query(ctx, bgp):
    arr = pattern_array(bgp)
    out = _TP()
    _check(ctx, lib().mapsq_query(ctx, arr, len(arr), C.byref(out)))
    return out


def mapsq_join_to_host(ctx, left, right, capacity=None, opts=None):
    """Join into host numpy columns slice by slice (see include/mapsq.h).
    ``capacity=None`` counts first (a call with no host columns), then joins
    into arrays of exactly that size.  Returns (vars, [uint32 columns], slices)."""
    lp = left if isinstance(left, _TP) else C.pointer(left)
    rp = right if isinstance(right, _TP) else C.pointer(right)
    o = C.byref(opts) if opts else None
    rows = C.c_uint64()
    slices = C.c_uint32()
    if capacity is None:
        _check(ctx, lib().mapsq_join_to_host(ctx, lp, rp, o, None, 0, C.byref(rows), None, C.byref(slices)))
        capacity = rows.value
    ncols = len(set(lp.contents.var[: lp.contents.ncols]) | set(rp.contents.var[: rp.contents.ncols]))
    cols = [np.zeros(max(int(capacity), 1), np.uint32) for _ in range(ncols)]
    arr = (_P * max(ncols, 1))(*[c.ctypes.data for c in cols])
    out = Table()
    _check(ctx, lib().mapsq_join_to_host(ctx, lp, rp, o, arr, capacity, C.byref(rows), C.pointer(out),
                                         C.byref(slices)))
    n = rows.value
    return list(out.var[: out.ncols]), [c[:n] for c in cols], slices.value


def mapsq_join_star(ctx, tables, key_var):
    arr = (_TP * len(tables))(*[t if isinstance(t, _TP) else C.pointer(t) for t in tables])
    out = _TP()
    _check(ctx, lib().mapsq_join_star(ctx, len(tables), arr, key_var, C.byref(out)))
    return out


def mapsq_build_info():
    """Which build of the library is loaded ("sm_103a" or "sm_103a checked")."""
    return lib().mapsq_build_info().decode()


def mapsq_set_wait_limit(ctx, spins):
    _check(ctx, lib().mapsq_set_wait_limit(ctx, spins))


def mapsq_selftest_wait(ctx, spins):
    """Raises MapsqError TIMEOUT when the bounded waits give up as designed."""
    _check(ctx, lib().mapsq_selftest_wait(ctx, spins))


def mapsq_project(ctx, t, vars_, distinct=False):
    arr = (C.c_int32 * max(len(vars_), 1))(*vars_)
    out = _TP()
    _check(ctx, lib().mapsq_project(ctx, t, len(vars_), arr, DISTINCT if distinct else 0, C.byref(out)))
    return out


def mapsq_query_select(ctx, bgp, vars_, distinct=False):
    pats = pattern_array(bgp)
    arr = (C.c_int32 * max(len(vars_), 1))(*vars_)
    out = _TP()
    _check(ctx, lib().mapsq_query_select(ctx, pats, len(pats), len(vars_), arr, DISTINCT if distinct else 0,
                                         C.byref(out)))
    return out


def mapsq_dict_load(ctx, terms):
    """``terms[i]``: the string of term id i (encoded as UTF-8)."""
    enc = [t.encode() for t in terms]
    offsets = np.zeros(len(enc) + 1, np.uint64)
    offsets[1:] = np.cumsum([len(b) for b in enc], dtype=np.uint64)
    blob = b"".join(enc)
    _check(ctx, lib().mapsq_dict_load(ctx, offsets.ctypes.data_as(C.POINTER(C.c_uint64)), blob, len(enc)))


def mapsq_decode(ctx, t, col):
    """The strings of column ``col`` (a list of str, one per row)."""
    n = int(t.contents.nrows)
    offsets = np.zeros(n + 1, np.uint64)
    total = C.c_uint64()
    optr = offsets.ctypes.data_as(C.POINTER(C.c_uint64))
    _check(ctx, lib().mapsq_decode(ctx, t, col, optr, None, 0, C.byref(total)))
    buf = C.create_string_buffer(max(total.value, 1))
    _check(ctx, lib().mapsq_decode(ctx, t, col, optr, C.cast(buf, _P), total.value, C.byref(total)))
    raw = buf.raw[: total.value]
    return [raw[int(offsets[r]):int(offsets[r + 1])].decode() for r in range(n)]


def mapsq_table_from_columns(ctx, vars_, cols, nrows=None):
    ncols = len(vars_)
    if nrows is None:
        nrows = int(cols[0].shape[0]) if ncols else 0
    dev = ncols > 0 and _is_device(cols[0])
    if not dev:
        cols = [np.ascontiguousarray(c, dtype=np.uint32) for c in cols]
    var_arr = (C.c_int32 * max(ncols, 1))(*vars_)
    col_arr = (_P * max(ncols, 1))(*[_ptr(c) for c in cols])
    out = _TP()
    _check(ctx, lib().mapsq_table_from_columns(ctx, nrows, ncols, var_arr, col_arr, 1 if dev else 0, C.byref(out)))
    return out


def mapsq_table_to_host(ctx, t, out=None):
    """Copy the columns to host memory: new numpy arrays, or the caller's
    ``out`` arrays (uint32, at least nrows long each; pinned memory copies
    fastest), of which the first nrows entries are returned as views."""
    tab = t.contents
    if out is None:
        cols = [np.empty(tab.nrows, dtype=np.uint32) for _ in range(tab.ncols)]
    else:
        if len(out) < tab.ncols or any(o.dtype != np.uint32 or o.shape[0] < tab.nrows or not o.flags.c_contiguous
                                       for o in out[: tab.ncols]):
            raise ValueError("out: one contiguous uint32 array of at least nrows entries per column")
        cols = [o[: tab.nrows] for o in out[: tab.ncols]]
    arr = (_P * max(tab.ncols, 1))(*[c.ctypes.data for c in cols])
    _check(ctx, lib().mapsq_table_to_host(ctx, t, arr))
    return list(tab.var[: tab.ncols]), cols


def mapsq_table_free(ctx, t):
    lib().mapsq_table_free(ctx, t)


def mapsq_sync(ctx):
    _check(ctx, lib().mapsq_sync(ctx))


def mapsq_memory_in_use(ctx):
    a, b = C.c_uint64(), C.c_uint64()
    _check(ctx, lib().mapsq_memory_in_use(ctx, C.byref(a), C.byref(b)))
    return a.value, b.value


def mapsq_set_profiling(ctx, enable):
    _check(ctx, lib().mapsq_set_profiling(ctx, 1 if enable else 0))


def mapsq_kernel_stats(ctx):
    cap = 64
    arr = (KernelStat * cap)()
    n = C.c_uint32()
    _check(ctx, lib().mapsq_kernel_stats(ctx, arr, cap, C.byref(n)))
    return {arr[i].name.decode(): {"launches": arr[i].launches, "device_ms": arr[i].device_ms,
                                   "alg_bytes": arr[i].alg_bytes} for i in range(min(n.value, cap))}


def mapsq_reset_stats(ctx):
    _check(ctx, lib().mapsq_reset_stats(ctx))


def mapsq_profile_only(ctx, name=None):
    _check(ctx, lib().mapsq_profile_only(ctx, name.encode() if name else None))


def mapsq_launch_count(ctx):
    n = C.c_uint64()
    _check(ctx, lib().mapsq_launch_count(ctx, C.byref(n)))
    return n.value


def mapsq_join_noalloc(left, right, out_cols, capacity, stream=None):
    """Join caller-described tables into caller-owned output buffers without any
    allocation (see include/mapsq.h).  ``left``/``right`` are ``Table`` structs
    (or pointers to them), ``out_cols`` device addresses.  Returns (status,
    Table describing the result, row count); the status is not raised so that a
    caller can retry with larger buffers after MAPSQ_ERR_BUDGET."""
    cols = (_P * max(len(out_cols), 1))(*out_cols)
    out = Table()
    rows = C.c_uint64()
    lp = left if isinstance(left, _TP) else C.pointer(left)
    rp = right if isinstance(right, _TP) else C.pointer(right)
    rc = lib().mapsq_join_noalloc(lp, rp, cols, capacity, C.pointer(out), C.byref(rows), stream)
    return rc, out, rows.value


def mapsq_autotune(ctx, sorted_rows=0):
    r = AutotuneResult()
    _check(ctx, lib().mapsq_autotune(ctx, sorted_rows, C.byref(r)))
    n = r.points
    return {"sorted_ratio": r.sorted_ratio, "sorted_rows": r.sorted_rows,
            "points": [{"ratio": r.ratio[i], "hash_ms": r.hash_ms[i], "sorted_ms": r.sorted_ms[i]} for i in range(n)],
            "part_min_build": r.part_min_build, "dense_max": r.dense_max,
            "size_points": [{"build_rows": r.part_rows[i], "partitioned_ms": r.part_on_ms[i],
                             "plain_ms": r.part_off_ms[i]} for i in range(r.part_points)],
            "skew_points": [{"group_rows": r.group[i], "dense_ms": r.dense_ms[i],
                             "partitioned_write_ms": r.partitioned_ms[i]} for i in range(r.dense_points)]}


def mapsq_set_sorted_ratio(ctx, ratio):
    _check(ctx, lib().mapsq_set_sorted_ratio(ctx, ratio))


def mapsq_serve_start(ctx, max_active=0, mem_budget_bytes=0):
    opts = ServeOpts(max_active=max_active, mem_budget_bytes=mem_budget_bytes)
    _check(ctx, lib().mapsq_serve_start(ctx, C.byref(opts)))


def mapsq_submit(ctx, bgp):
    arr = (Pattern * len(bgp))(*[_pattern(tp) for tp in bgp])
    ticket = C.c_uint64()
    rc = lib().mapsq_submit(ctx, arr, len(bgp), C.byref(ticket))
    if rc != 0:
        raise MapsqError(rc, lib().mapsq_strerror(rc).decode())
    return ticket.value


def mapsq_poll(ctx, ticket):
    """The query's result table once done (None while it runs); raises its error."""
    out = _TP()
    rc = lib().mapsq_poll(ctx, ticket, C.byref(out))
    if rc != 0:
        raise MapsqError(rc, lib().mapsq_strerror(rc).decode())
    return out if out else None


def mapsq_serve_stats(ctx):
    st = ServeCounters()
    _check(ctx, lib().mapsq_serve_stats(ctx, C.byref(st)))
    return {name: getattr(st, name) for name, _ in ServeCounters._fields_}


def mapsq_serve_stop(ctx):
    _check(ctx, lib().mapsq_serve_stop(ctx))


def table_view(vars_, cols, nrows=None, sorted_cols=()):
    """A ``Table`` struct describing caller-owned device columns (no copy);
    ``sorted_cols`` lists the columns the caller knows to be nondecreasing."""
    t = Table()
    for c in sorted_cols:
        t.sorted_mask |= 1 << c
    t.nrows = int(cols[0].shape[0]) if cols else int(nrows or 0)
    t.ncols = len(vars_)
    for c in range(MAX_VARS):
        t.var[c] = vars_[c] if c < len(vars_) else -1
        t.col[c] = _ptr(cols[c]) if c < len(cols) else None
    t.on_device = 1
    return t


# ------------------------------------------------------------------ conveniences

class _CudaArray:
    """Exposes one device column through __cuda_array_interface__ (no copy)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<u4", "data": (int(ptr or 0), False),
                                         "version": 3, "strides": None, "stream": None}


class TableRef:
    """A table owned by the library, freed with its context or by :meth:`free`."""

    def __init__(self, ctx: "Context", ptr):
        self.ctx = ctx
        self.ptr = ptr

    @property
    def nrows(self) -> int:
        return int(self.ptr.contents.nrows)

    @property
    def vars(self):
        t = self.ptr.contents
        return list(t.var[: t.ncols])

    def to_host(self, out=None):
        """(vars, [numpy uint32 column, ...]); ``out``: caller's arrays to fill."""
        return mapsq_table_to_host(self.ctx.handle, self.ptr, out)

    def device_columns(self):
        """Zero-copy torch views of the device columns (valid until free)."""
        import torch
        t = self.ptr.contents
        return [torch.as_tensor(_CudaArray(t.col[c], t.nrows), device="cuda") for c in range(t.ncols)]

    def decode(self, col):
        """The strings of column ``col`` through the context's dictionary."""
        return mapsq_decode(self.ctx.handle, self.ptr, col)

    def free(self):
        if self.ptr:
            mapsq_table_free(self.ctx.handle, self.ptr)
            self.ptr = None


class Context:
    """One library context on one GPU; its device work runs on ``stream``
    (default: torch's current stream when torch has a GPU, else a private one)."""

    def __init__(self, device=0, stream=None, budget=0, allocator=None):
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    # torch's default stream is the legacy default stream (handle 1 for the runtime)
                    stream = torch.cuda.current_stream(device).cuda_stream or 1
            except ImportError:
                pass
        self._allocator = allocator
        self.handle = mapsq_create(device, allocator, stream, budget)

    def close(self):
        if self.handle:
            mapsq_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def load_triples(self, s, p, o):
        mapsq_load_triples(self.handle, s, p, o)

    def store_info(self):
        return mapsq_store_info(self.handle)

    def scan_pattern(self, tp) -> TableRef:
        return TableRef(self, mapsq_scan_pattern(self.handle, tp))

    def join(self, left: TableRef, right: TableRef, opts=None) -> TableRef:
        return TableRef(self, mapsq_join(self.handle, left.ptr, right.ptr, opts))

    def join_star(self, tables, key_var) -> TableRef:
        return TableRef(self, mapsq_join_star(self.handle, [t.ptr for t in tables], key_var))

    def join_batch(self, lefts, rights, opts=None):
        return [TableRef(self, p) for p in mapsq_join_batch(self.handle, [x.ptr for x in lefts],
                                                             [x.ptr for x in rights], opts)]

    def query_batch(self, bgps):
        return [TableRef(self, p) for p in mapsq_query_batch(self.handle, bgps)]

    def query(self, bgp, select=None, distinct=False) -> TableRef:
        """Solutions of a BGP; ``select``: the variables to keep (SELECT), with
        ``distinct`` for SELECT DISTINCT."""
        if select is None:
            return TableRef(self, mapsq_query(self.handle, bgp))
        return TableRef(self, mapsq_query_select(self.handle, bgp, list(select), distinct))

    def project(self, t: TableRef, vars_, distinct=False) -> TableRef:
        return TableRef(self, mapsq_project(self.handle, t.ptr, list(vars_), distinct))

    def dict_load(self, terms):
        mapsq_dict_load(self.handle, terms)

    def table(self, vars_, cols, nrows=None) -> TableRef:
        return TableRef(self, mapsq_table_from_columns(self.handle, list(vars_), list(cols), nrows))

    def sync(self):
        mapsq_sync(self.handle)

    def memory_in_use(self):
        return mapsq_memory_in_use(self.handle)

    def set_profiling(self, on: bool):
        mapsq_set_profiling(self.handle, on)

    def kernel_stats(self):
        return mapsq_kernel_stats(self.handle)

    def reset_stats(self):
        mapsq_reset_stats(self.handle)

    def profile_only(self, name=None):
        mapsq_profile_only(self.handle, name)

    def launch_count(self):
        return mapsq_launch_count(self.handle)

    def autotune(self, sorted_rows=0):
        return mapsq_autotune(self.handle, sorted_rows)

    def set_sorted_ratio(self, ratio):
        mapsq_set_sorted_ratio(self.handle, ratio)

    def serve_start(self, max_active=0, mem_budget_bytes=0):
        mapsq_serve_start(self.handle, max_active, mem_budget_bytes)

    def submit(self, bgp) -> int:
        return mapsq_submit(self.handle, bgp)

    def poll(self, ticket):
        p = mapsq_poll(self.handle, ticket)
        return TableRef(self, p) if p is not None else None

    def serve_stats(self):
        return mapsq_serve_stats(self.handle)

    def serve_stop(self):
        mapsq_serve_stop(self.handle)


def torch_allocator():
    """An allocator that takes device memory from torch's caching allocator."""
    import torch

    sizes = {}

    def _alloc(nbytes, user, stream):
        try:
            p = torch.cuda.caching_allocator_alloc(int(nbytes))
        except RuntimeError:
            return None
        sizes[p] = nbytes
        return p

    def _free(ptr, nbytes, user, stream):
        sizes.pop(ptr, None)
        torch.cuda.caching_allocator_delete(ptr)

    a = Allocator(ALLOC_FN(_alloc), FREE_FN(_free), None)
    a._keep = (_alloc, _free, sizes)
    return a
