/*
 * mapsq.h - C ABI of a GB300-native implementation of MapSQ's MapReduce-based
 * join of SPARQL triple-pattern partial matches (Feng, Zhang, Feng,
 * "MapSQ: A MapReduce-based Framework for SPARQL Queries on GPU",
 * arXiv 1702.03484).
 *
 * Model.  A graph is a set of dictionary-encoded triples (s, p, o), every term
 * a uint32 id (0 .. 0xFFFFFFFF are all valid).  A triple pattern binds some of
 * s, p, o to constants and the others to variables (ids 0..15).  Matching a
 * pattern gives its partial-match table (Section 1, Table 1(a), 1(b)); two
 * tables are joined on their shared variables (Algorithm 1); a basic graph
 * pattern (BGP) is evaluated one pattern at a time, joining after each match
 * (Section 2).  The host plans subqueries and join order; the device matches
 * and joins (the paper's CPU/GPU coprocessing split, Section 2).
 *
 * Tables.  A table is structure-of-arrays: ``ncols`` uint32 columns of
 * ``nrows`` rows; column c holds variable ``var[c]``.  Tables returned by the
 * library are owned by the library until ``mapsq_table_free``; their columns
 * are device pointers (256-byte aligned, except scan results, which may be
 * read-only slices of the triple store).  A caller may also describe its own
 * device columns in a ``mapsq_table`` it fills itself and pass it as an input;
 * such columns must be 4-byte aligned and the caller keeps ownership (never
 * pass such a table to ``mapsq_table_free``).
 *
 * Results are multisets of rows (bag semantics, no DISTINCT); row order is
 * unspecified.
 *
 * Citations.  Every call that computes a step of the method names the passage
 * of the paper (Section, Algorithm or Table) that defines it.  The others
 * (context and stream, errors, table memory, statistics, profiling) are
 * infrastructure with no counterpart in the paper.
 *
 * Conventions.  Every int-returning call returns MAPSQ_OK (0) or a negative
 * MAPSQ_ERR_* code; after an error, output arguments are left untouched and
 * ``mapsq_last_error`` describes it.  Input pointers are borrowed for the call
 * only.  All device work of a context is ordered on its CUDA stream; calls on
 * one context must not run concurrently from several threads.  Calls that
 * return a row count synchronise with that stream.
 */
#ifndef MAPSQ_H
#define MAPSQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MAPSQ_MAX_VARS 16

#if defined(__GNUC__)
#define MAPSQ_API __attribute__((visibility("default")))
#else
#define MAPSQ_API
#endif

/* Status codes. */
#define MAPSQ_OK 0
#define MAPSQ_ERR_INVALID (-1)     /* bad argument (NULL, bad var id, bad size) */
#define MAPSQ_ERR_UNSUPPORTED (-2) /* valid SPARQL outside the path: variable predicate, >2 join keys */
#define MAPSQ_ERR_OOM (-3)         /* the allocator returned NULL */
#define MAPSQ_ERR_BUDGET (-4)      /* the step needs more than the context's memory budget */
#define MAPSQ_ERR_CUDA (-5)        /* a CUDA runtime call failed */
#define MAPSQ_ERR_TIMEOUT (-6)     /* a bounded device wait gave up (device status word) */
#define MAPSQ_ERR_BUSY (-7)        /* the serving loop is not accepting work */
#define MAPSQ_ERR_NOT_FOUND (-8)   /* unknown ticket */

/* var_mask bits of a pattern: the field holds a variable id instead of a term. */
#define MAPSQ_VAR_S 1u
#define MAPSQ_VAR_P 2u
#define MAPSQ_VAR_O 4u

/* Join algorithms for mapsq_join_opts.algorithm.  Both compute Algorithm 1's
 * result; they differ in how equal keys are brought together (its Sort step):
 * HASH groups the smaller side by key in a hash table; SORTED uses a side
 * whose key column is already sorted (sorted_mask) as the groups and searches
 * it with the other side's keys.  AUTO takes SORTED when a side is sorted on
 * the (single) key column and at least the context's sorted ratio times the
 * other side's rows (see mapsq_autotune), else HASH. */
#define MAPSQ_JOIN_AUTO 0
#define MAPSQ_JOIN_HASH 1
#define MAPSQ_JOIN_SORTED 2

typedef struct mapsq_ctx mapsq_ctx;

/* Device memory provider.  ``alloc`` returns device memory of at least
 * ``bytes`` bytes usable on ``stream`` (a cudaStream_t) or NULL; ``free``
 * releases a block obtained from ``alloc``.  NULL allocator: the library uses
 * its own stream-ordered pool (cudaMallocAsync). */
typedef struct {
  void* (*alloc)(size_t bytes, void* user, void* stream);
  void (*free)(void* ptr, size_t bytes, void* user, void* stream);
  void* user;
} mapsq_allocator;

/* One triple pattern (Section 1).  A field whose MAPSQ_VAR_* bit is set in
 * ``var_mask`` holds a variable id (0..15), otherwise a term id.  The predicate
 * must be a constant (a variable predicate gives MAPSQ_ERR_UNSUPPORTED). */
typedef struct {
  uint32_t s, p, o, var_mask;
} mapsq_pattern;

/* A binding table (structure of arrays), see "Tables" above.  A table with
 * ncols == 0 is a set of empty bindings: nrows is 0 (no solution) or 1 (the
 * pattern held, no variable bound).  Bit c of ``sorted_mask`` says that column
 * c is in nondecreasing order: scan results carry it (a run of the store is
 * sorted, Section 2's partial matches come from a sorted index here), and a
 * join whose key is such a column may use it as the grouped side instead of a
 * hash table (the Sort step of Algorithm 1, already done).  Zero is always
 * correct; a caller filling its own table must not set a bit for a column
 * that is not sorted. */
typedef struct {
  uint64_t nrows;
  uint32_t ncols;
  int32_t var[MAPSQ_MAX_VARS];
  uint32_t* col[MAPSQ_MAX_VARS];
  int32_t on_device;
  uint32_t sorted_mask;
} mapsq_table;

/* Join options; a NULL pointer or zero fields choose defaults. */
typedef struct {
  int32_t algorithm;     /* MAPSQ_JOIN_AUTO, _HASH or _SORTED (SORTED falls back to HASH when no
                            side is sorted on a single key column) */
  int32_t reserved[3];   /* zero */
} mapsq_join_opts;

/* What mapsq_autotune measured (times: best of three joins, milliseconds).
 * Shuffle axis: per tested ratio r of sorted-side rows to other-side rows,
 * one join by each algorithm.  Size axis: hash joins of part_rows[i] build
 * rows (two per key) probed by four times as many rows, with and without the
 * region partition of the build side.  Skew axis: hash joins whose keys have
 * group[i] build rows each (2^20 build rows, 2^20 probe rows, every probe row
 * matching a whole group), written by the dense write (a thread per probe
 * row) or by the partitioned write (output tiles spread over all SMs).  Size
 * axis points: 2^16, 2^18, 2^20, 2^22 and 2^24 build rows. */
typedef struct {
  uint32_t sorted_ratio;   /* chosen: AUTO takes SORTED from this ratio up (0xFFFFFFFF = never) */
  uint32_t points;         /* tested ratios */
  uint32_t ratio[12];
  double hash_ms[12];
  double sorted_ms[12];
  uint64_t sorted_rows;    /* rows of the sorted side in the test joins */
  uint64_t part_min_build; /* chosen: hash builds of at least this many rows are partitioned (UINT64_MAX = never) */
  uint32_t part_points;
  uint32_t dense_max;      /* chosen: the dense write for joins of at most this many matches per probe row
                              on average (and at most 64 in any row) */
  uint64_t part_rows[6];
  double part_on_ms[6];
  double part_off_ms[6];
  uint32_t dense_points;
  uint32_t group[6];
  double dense_ms[6];
  double partitioned_ms[6];
} mapsq_autotune_result;

/* Autotune the context's join choices on this GPU (the paper has no
 * counterpart; every choice computes Algorithm 1's same result):
 * (1) hash vs sorted join (two ways of Algorithm 1's Sort step): joins a
 * sorted side of ``sorted_rows`` rows (0 = 2^22; keys k / 2, so every key
 * twice) with other sides of sorted_rows / r rows (keys uniform over the same
 * range) for r = 1, 2, 4, ..., 2048 and sets the sorted ratio to the smallest r
 * from which SORTED is never slower; (2) per build size, whether a hash
 * build is partitioned by region first (build sides of 2^16 to 2^22 rows):
 * the smallest size from which partitioning is never slower; (3) per skew
 * (rows per key group, 4 to 64), the dense or the partitioned write: the
 * dense write up to the largest group size at which it is not slower, applied
 * to a join's mean number of matches per probe row.  Times are the best of
 * three joins, host synchronisation included.  ``out`` may be NULL.  Uses
 * about 2.5 GB of device memory at most.  Errors: BUSY (serving), OOM,
 * BUDGET, CUDA. */
MAPSQ_API int mapsq_autotune(mapsq_ctx* ctx, uint64_t sorted_rows, mapsq_autotune_result* out);

/* Set the context's sorted ratio directly (what mapsq_autotune measures; the
 * default is 4; 0xFFFFFFFF never takes the sorted join).  Errors: INVALID
 * (ratio 0), BUSY (serving). */
MAPSQ_API int mapsq_set_sorted_ratio(mapsq_ctx* ctx, uint32_t ratio);

/* Serving loop options (mapsq_serve_start); zero fields choose defaults. */
typedef struct {
  uint32_t max_active;        /* queries in flight at once (default 256) */
  uint32_t reserved0;
  uint64_t mem_budget_bytes;  /* bytes of intermediate and result tables in flight (0 = unbounded) */
  uint64_t reserved[4];
} mapsq_serve_opts;

/* Serving loop counters (mapsq_serve_stats).  Latency is measured from
 * mapsq_submit to the query's completion, over completed and failed queries. */
typedef struct {
  uint64_t submitted, completed, failed, in_flight;
  uint64_t rounds;         /* worker rounds (each at most one batched join) */
  uint64_t batched_joins;  /* joins run inside those batches */
  uint64_t result_rows;    /* rows of the completed results */
  uint64_t preempted;      /* queries put back in the queue for memory */
  double p50_ms, p99_ms, mean_ms;
} mapsq_serve_counters;

/* Per-kernel device time, collected while profiling is on (mapsq_set_profiling).
 * ``alg_bytes`` sums each launch's algorithmic bytes: the bytes the step must
 * read and write at minimum (inputs once, outputs once). */
typedef struct {
  char name[48];
  uint64_t launches;
  double device_ms;
  double alg_bytes;
} mapsq_kernel_stat;

/* Create a context on CUDA device ``device``.  ``cuda_stream`` (a cudaStream_t)
 * orders all device work; NULL creates a private non-blocking stream (pass
 * cudaStreamLegacy, (void*)1, for the legacy default stream).
 * ``mem_budget_bytes`` bounds the device memory of intermediate and result
 * tables plus scratch (0 = unbounded).  Errors: INVALID (out == NULL, bad
 * device), CUDA. */
MAPSQ_API int mapsq_create(mapsq_ctx** out, int device, const mapsq_allocator* allocator, void* cuda_stream,
                 uint64_t mem_budget_bytes);

/* Synchronise, free the triple store and every table still owned by ``ctx``, and
 * the context itself.  NULL is a no-op returning MAPSQ_OK. */
MAPSQ_API int mapsq_destroy(mapsq_ctx* ctx);

/* Replace the stream that orders the context's work (a cudaStream_t; NULL =
 * the private stream).  Earlier work is not waited for. */
MAPSQ_API int mapsq_set_stream(mapsq_ctx* ctx, void* cuda_stream);

/* Description of the last error on this context (never NULL). */
MAPSQ_API const char* mapsq_last_error(const mapsq_ctx* ctx);

/* Which build of the library this is: "sm_103a", or "sm_103a checked" for
 * libmapsq_checked.so, whose kernels check their device indexes (a failed
 * check sets a bit of the device status word, skips the access and makes the
 * call return MAPSQ_ERR_CUDA; joins then synchronise once more).  Never NULL. */
MAPSQ_API const char* mapsq_build_info(void);

/* Name of a status code. */
MAPSQ_API const char* mapsq_strerror(int status);

/* Load a graph: ``n`` triples given as three uint32 columns (host pointers, or
 * device pointers when ``ptrs_on_device`` is nonzero).  The graph is a set
 * (RDF): duplicate triples are dropped.  Builds the device-resident store: per
 * predicate, the (s, o) pairs sorted by s then o, and the (o, s) pairs sorted by
 * o then s (the index that replaces the paper's partial-matching engine,
 * Section 2).  Replaces any previous store; tables from earlier scans stay
 * valid.  Synchronises.  Errors: INVALID, OOM, BUDGET, CUDA. */
MAPSQ_API int mapsq_load_triples(mapsq_ctx* ctx, const uint32_t* s, const uint32_t* p, const uint32_t* o, uint64_t n,
                       int ptrs_on_device);

/* Number of distinct triples and predicates of the loaded store. */
MAPSQ_API int mapsq_store_info(mapsq_ctx* ctx, uint64_t* n_triples, uint32_t* n_predicates);

/* Partial matches of one triple pattern (Section 1, Table 1(a) and 1(b);
 * Section 2, first step of query answering).  The result has one column per
 * distinct variable, in the order s, o; a variable in both places keeps the
 * triples with s == o.  Both constants: a 0-column table of 0 or 1 rows.  The
 * result may be a read-only view of the store's sorted columns (no copy); it
 * stays valid after the store is replaced, until it is freed.  Its
 * sorted_mask marks the column the store keeps sorted.
 * Synchronises.  Errors: INVALID (NULL, var id > 15), UNSUPPORTED (variable
 * predicate), OOM, BUDGET, CUDA; INVALID if no store is loaded. */
MAPSQ_API int mapsq_scan_pattern(mapsq_ctx* ctx, const mapsq_pattern* tp, mapsq_table** out);

/* Join two tables on their shared variables (Algorithm 1, the MapReduce-based
 * join: map each row to (key = shared variables, value = other columns, label
 * LEFT/RIGHT), shuffle by key, and reduce each key to every LEFT x RIGHT pair).
 * Output columns: the shared variables in ascending id, then the left table's
 * other columns in order, then the right table's (Table 1(c)).  No shared
 * variable: the cross product.  Input columns must be on the device.  The
 * shuffle is a hash build or, for a side sorted on the key column, the sorted
 * join (``opts``: NULL or MAPSQ_JOIN_AUTO lets the context choose, see
 * MAPSQ_JOIN_SORTED); the result is the same.  Synchronises once to size the
 * output (twice when a hash build side has 2^16 rows or more: its distinct
 * keys are estimated first, to size the table).  Errors: INVALID (also an
 * unknown algorithm), UNSUPPORTED (more than two shared variables), OOM,
 * BUDGET, CUDA. */
MAPSQ_API int mapsq_join(mapsq_ctx* ctx, const mapsq_table* left, const mapsq_table* right, mapsq_table** out,
               const mapsq_join_opts* opts);

/* A join whose result need not fit in device memory (the paper's GPU had
 * 1536 MB, Section 3): Algorithm 1 on slices of the larger input, whose
 * results together are the join, since every row of one slice finds all its
 * matches in the other, whole input.  Each slice's result is computed on the
 * device, copied to the caller's host columns (``host_cols[c]``, room for
 * ``capacity_rows`` rows; columns in mapsq_join's order) after the slices
 * before it, and freed; a slice whose count or result exceeds the context's
 * memory budget or the device memory is halved and retried.  The smaller input
 * is whole in every slice and must fit.  ``*out_rows`` receives the join's
 * row count; ``host_cols`` NULL only counts; if the count exceeds
 * capacity_rows the call returns MAPSQ_ERR_BUDGET after counting every slice
 * (``*out_rows`` set, the host columns partly written).  On success ``*out``
 * (may be NULL) describes the host result (on_device 0, columns =
 * host_cols) and ``*slices`` (may be NULL) the number of slices.  Input
 * columns must be on the device.  Synchronises at least once per slice.
 * Errors: INVALID, UNSUPPORTED, BUDGET, OOM (a one-row slice does not fit),
 * CUDA. */
MAPSQ_API int mapsq_join_to_host(mapsq_ctx* ctx, const mapsq_table* left, const mapsq_table* right,
                                 const mapsq_join_opts* opts, uint32_t* const* host_cols, uint64_t capacity_rows,
                                 uint64_t* out_rows, mapsq_table* out, uint32_t* slices);

/* Multi-way join of ``k`` (2 to 8) tables that share exactly one variable,
 * ``key_var`` (the partial matches of a star of triple patterns around it):
 * the key/value framing of Section 1 and Algorithm 1 with k inputs instead of
 * two, in one count and write round instead of k - 1 pairwise joins.  Result:
 * for every key value, every combination of one row from each table holding
 * it; columns: the key, then each table's other columns in table order (the
 * order k - 1 pairwise joins give).  Every table but one must be sorted on
 * the key (sorted_mask; scan results sorted on it are); otherwise the tables
 * are joined pairwise, with the same result.  Synchronises once.  Errors:
 * INVALID (NULL, k out of range, a table without the key, a variable other
 * than the key in two tables, more than 16 result columns), UNSUPPORTED (one
 * key's product beyond 2^32 rows), OOM, BUDGET, CUDA. */
MAPSQ_API int mapsq_join_star(mapsq_ctx* ctx, uint32_t k, const mapsq_table* const* tables, int32_t key_var,
                              mapsq_table** out);

/* Batched form: ``k`` independent joins (each as mapsq_join, Algorithm 1;
 * evaluating many at once has no counterpart in the paper) evaluated
 * together.  Every phase of the join (hash build, count, partition, write) is
 * one launch for the whole batch, the write phase a persistent kernel fed by a
 * device work queue, and the batch synchronises once to size all outputs
 * (twice with large hash build sides, as mapsq_join), so many small joins cost
 * about as much as one.  out[j] receives join j's table.  With k > 1 the k
 * tables share one device allocation: each is freed with mapsq_table_free as
 * usual, and their memory returns when the last of them is freed.
 * Errors: as mapsq_join (then no table is returned). */
MAPSQ_API int mapsq_join_batch(mapsq_ctx* ctx, uint32_t k, const mapsq_table* const* left,
                               const mapsq_table* const* right, mapsq_table** out, const mapsq_join_opts* opts);

/* Evaluate a BGP of ``n`` patterns (Section 2: match each pattern, join the
 * partial results after each match).  The host orders the patterns: the one
 * with fewest matches first, then repeatedly the one with fewest matches among
 * those sharing a variable with the joined ones.  A star of 3 to 8 patterns
 * (one variable in every pattern, no other variable in two) is joined in one
 * round instead (mapsq_join_star).  Result columns are the BGP's variables in
 * ascending id.  Errors: as mapsq_scan_pattern and mapsq_join. */
MAPSQ_API int mapsq_query(mapsq_ctx* ctx, const mapsq_pattern* bgp, uint32_t n, mapsq_table** out);

/* Batched form of mapsq_query: ``nq`` BGPs (bgps[q] with n[q] patterns, each
 * evaluated as in Section 2; batching has no counterpart in the paper)
 * evaluated together.  Their range searches are one launch; at each level,
 * every query's next join goes into one batched join (mapsq_join_batch), so
 * the batch synchronises about once per level instead of once per join.
 * out[q] receives query q's result (columns in ascending variable id).  The
 * results of the queries whose last join falls in the same level share one
 * device allocation with that level's other results (as mapsq_join_batch's),
 * returned when the last of them is freed.
 * All or nothing: on error no table is returned.  Errors: as mapsq_query. */
MAPSQ_API int mapsq_query_batch(mapsq_ctx* ctx, uint32_t nq, const mapsq_pattern* const* bgps, const uint32_t* n,
                                mapsq_table** out);

/* Start the serving loop: a worker thread that evaluates submitted BGP queries
 * with continuous batching over the loaded store.  Each query is evaluated as
 * in mapsq_query (Section 2: the host hands the partial-match tables of one
 * query, pattern after pattern, to the device join); running many queries at
 * once, in shared launches under a memory budget, has no counterpart in the
 * paper.  In every round it admits
 * waiting queries (while fewer than max_active are in flight and the tables
 * in flight stay under mem_budget_bytes), gives the new ones their range
 * searches in one launch, and puts the next join of every query in flight into
 * one batched join; after that batch's count pass, results are written in
 * arrival order while they fit in the budget, the others wait for a later
 * round.  When no join fits, the youngest query in flight is put back in the
 * queue (its tables freed) and admissions pause until a join is written; a
 * query whose next result cannot fit beside its own tables even alone fails
 * with MAPSQ_ERR_BUDGET.  While serving, only the serve calls, mapsq_table_to_host,
 * mapsq_table_free, mapsq_memory_in_use and the statistics calls may be made
 * on the context; the others return MAPSQ_ERR_BUSY.  Errors: BUSY (already
 * serving), INVALID (no store), OOM. */
MAPSQ_API int mapsq_serve_start(mapsq_ctx* ctx, const mapsq_serve_opts* opts);

/* Queue a BGP of ``n`` patterns (copied; evaluated as in Section 2 by the
 * serving loop); *ticket identifies it.  Thread-safe.
 * Errors: BUSY (not serving or stopping), INVALID, UNSUPPORTED. */
MAPSQ_API int mapsq_submit(mapsq_ctx* ctx, const mapsq_pattern* bgp, uint32_t n, uint64_t* ticket);

/* Collect a query: MAPSQ_OK with *out = its result (written on the device;
 * columns in ascending variable id; owned by the caller until
 * mapsq_table_free) once done, MAPSQ_OK
 * with *out = NULL while it runs, the query's error code if it failed,
 * NOT_FOUND for a ticket never issued.  A result is returned once.
 * Thread-safe. */
MAPSQ_API int mapsq_poll(mapsq_ctx* ctx, uint64_t ticket, mapsq_table** out);

/* Counters and latency percentiles of the serving loop.  Thread-safe. */
MAPSQ_API int mapsq_serve_stats(mapsq_ctx* ctx, mapsq_serve_counters* out);

/* Finish every submitted query, then stop the worker.  Results not yet
 * collected stay owned by the context.  Not to be called while another thread
 * is inside mapsq_submit, mapsq_poll or mapsq_serve_stats on this context.
 * Errors: BUSY (not serving). */
MAPSQ_API int mapsq_serve_stop(mapsq_ctx* ctx);

/* Copy ``ncols`` columns of ``nrows`` rows (host pointers, or device pointers if
 * ``on_device``) into a new library-owned device table with variables ``var``.
 * ncols == 0 makes a 0-column table of ``nrows`` (0 or 1) empty bindings.
 * Errors: INVALID (ncols > 16, duplicate or out-of-range var ids, NULL), OOM,
 * BUDGET, CUDA. */
MAPSQ_API int mapsq_table_from_columns(mapsq_ctx* ctx, uint64_t nrows, uint32_t ncols, const int32_t* var,
                             const uint32_t* const* cols, int on_device, mapsq_table** out);

/* Copy every column of ``t`` to caller-owned host buffers (host_cols[c] holds
 * t->nrows uint32).  Synchronises.  Errors: INVALID, CUDA. */
MAPSQ_API int mapsq_table_to_host(mapsq_ctx* ctx, const mapsq_table* t, uint32_t* const* host_cols);

/* Release a table returned by the library (NULL is a no-op). */
MAPSQ_API void mapsq_table_free(mapsq_ctx* ctx, mapsq_table* t);

/* Wait for the context's stream and check the device status word.  Errors:
 * CUDA, TIMEOUT. */
MAPSQ_API int mapsq_sync(mapsq_ctx* ctx);

/* Bound every wait of a device thread on another (the look-back of the prefix
 * scans) at ``spins`` polls of about 30-50 ns each (default 2^20, about 50
 * ms); a wait that runs out sets
 * the context's device status word and the kernel ends, and the next call
 * that synchronises returns MAPSQ_ERR_TIMEOUT (the context stays usable).
 * Infrastructure; the paper has no counterpart.  Errors: INVALID (spins == 0). */
MAPSQ_API int mapsq_set_wait_limit(mapsq_ctx* ctx, uint32_t spins);

/* Self-test of the bounded waits: runs a prefix scan of four tiles whose first
 * tile no block ever takes, so each later tile's look-back waits for a
 * predecessor that is never published; with the wait limit ``spins`` every
 * such wait gives up, the kernel ends and the call returns MAPSQ_ERR_TIMEOUT
 * (the expected result), after which the status word is clear and the context
 * usable.  MAPSQ_OK would mean a wait did not give up.  Synchronises.
 * Infrastructure; the paper has no counterpart.  Errors: INVALID, BUSY, OOM,
 * BUDGET, CUDA; TIMEOUT as described. */
MAPSQ_API int mapsq_selftest_wait(mapsq_ctx* ctx, uint32_t spins);

/* Device memory currently held for tables and scratch, and its high-water mark. */
MAPSQ_API int mapsq_memory_in_use(mapsq_ctx* ctx, uint64_t* bytes, uint64_t* peak_bytes);

/* Turn per-kernel timing on (1) or off (0).  While on, every launch is bracketed
 * by CUDA events on the context's stream. */
MAPSQ_API int mapsq_set_profiling(mapsq_ctx* ctx, int enable);

/* Per-kernel totals since profiling was last turned on or reset: writes up to
 * ``cap`` entries and their number to ``*n``.  Synchronises. */
MAPSQ_API int mapsq_kernel_stats(mapsq_ctx* ctx, mapsq_kernel_stat* out, uint32_t cap, uint32_t* n);

/* Restrict profiling to the kernel kind named ``name`` (as reported by
 * mapsq_kernel_stats); NULL profiles every kind again.  Errors: INVALID
 * (unknown name). */
MAPSQ_API int mapsq_profile_only(mapsq_ctx* ctx, const char* name);

/* Clear the per-kernel totals. */
MAPSQ_API int mapsq_reset_stats(mapsq_ctx* ctx);

/* Number of CUDA kernels this context has launched since it was created. */
MAPSQ_API int mapsq_launch_count(mapsq_ctx* ctx, uint64_t* launches);

/* Flags of mapsq_project and mapsq_query_select. */
#define MAPSQ_DISTINCT 1u

/* The SELECT clause of a query (Section 1: query Q selects ?person from the
 * solutions of its patterns): a new table holding the columns of ``t`` whose
 * variables are ``vars[0 .. nvars)``, in that order.  Without MAPSQ_DISTINCT
 * every row is kept (SPARQL's default bag semantics: one row per solution);
 * with it each distinct row is kept once (SELECT DISTINCT; which of several
 * equal rows survives is unspecified, their values being equal), in the
 * order of the rows kept.  Columns of ``t`` must be on the device.  DISTINCT
 * synchronises once (to size its result) and uses 12 bytes of scratch per row
 * of ``t`` plus 4 per slot of its table (a power of two of at least twice the
 * rows).  Errors: INVALID (NULL, nvars == 0, a variable not in ``t`` or given
 * twice, unknown flags), UNSUPPORTED (DISTINCT over more than 2^31 rows), OOM,
 * BUDGET, CUDA. */
MAPSQ_API int mapsq_project(mapsq_ctx* ctx, const mapsq_table* t, uint32_t nvars, const int32_t* vars,
                            uint32_t flags, mapsq_table** out);

/* A BGP query with a SELECT clause: mapsq_query (Section 2) followed by
 * mapsq_project of its solutions (Section 1, query Q); the full solution table
 * is freed.  Errors: as mapsq_query and mapsq_project. */
MAPSQ_API int mapsq_query_select(mapsq_ctx* ctx, const mapsq_pattern* bgp, uint32_t n, uint32_t nvars,
                                 const int32_t* vars, uint32_t flags, mapsq_table** out);

/* Load a term dictionary for mapsq_decode: term id i is the byte string
 * ``bytes[offsets[i] .. offsets[i + 1])`` (host pointers; ``offsets`` has
 * n_terms + 1 nondecreasing entries from 0; both are copied to the device).
 * The dictionary is the inverse of the encoding that turned an RDF graph's
 * terms into the uint32 ids of the triples (the paper's tables, Table 1, show
 * terms as strings).  Replaces any previous dictionary.  Synchronises.
 * Errors: INVALID, BUSY (serving), OOM, BUDGET, CUDA. */
MAPSQ_API int mapsq_dict_load(mapsq_ctx* ctx, const uint64_t* offsets, const char* bytes, uint32_t n_terms);

/* Decode column ``col`` of ``t`` (device columns) through the loaded
 * dictionary: row r's string is written to ``bytes[offsets[r] .. offsets[r +
 * 1])``.  ``offsets`` (host, caller-owned, t->nrows + 1 entries) is always
 * filled and ``*nbytes`` receives offsets[t->nrows]; the bytes are written only
 * when ``bytes`` is not NULL and *nbytes <= ``cap``, so a caller can size its
 * buffer with a first call.  Synchronises.  Errors: INVALID (NULL, no
 * dictionary, col out of range, an id with no term), OOM, BUDGET, CUDA. */
MAPSQ_API int mapsq_decode(mapsq_ctx* ctx, const mapsq_table* t, uint32_t col, uint64_t* offsets, char* bytes,
                           uint64_t cap, uint64_t* nbytes);

/* Join two tables without allocating any memory.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc (a host that
 * owns all device memory and lends only fixed buffers, or a path where an
 * allocation could block or fail).  It computes the same result as mapsq_join
 * (same column layout) with no context: every intermediate lives in one
 * 64 MiB device array inside the library, which each GPU that loads the
 * library holds until the process exits.  Nothing is allocated: no cudaMalloc,
 * no cudaFree, no allocating library routine.
 *
 * ``left``/``right``: caller-described tables, columns on the current device,
 * 4-byte aligned.  The smaller input may have at most 262,144 rows and the
 * larger at most 1,048,576, whatever their order or sorted_mask (the join
 * always groups the smaller input in a hash table); larger inputs give
 * MAPSQ_ERR_INVALID before any device work.  A result of more than 2^32 rows
 * gives MAPSQ_ERR_UNSUPPORTED (after the count, with ``*out_rows`` set).
 * ``out_cols``: one caller-owned device buffer per output column
 * (shared variables, then the left table's other columns, then the right
 * table's), each 16-byte aligned with room for ``out_capacity_rows`` rows.  On
 * return ``*out_rows`` holds the join's row count; if it exceeds the capacity
 * the call returns MAPSQ_ERR_BUDGET without writing the outputs, so the caller
 * can retry with larger buffers.  On success ``*out`` describes the result
 * (its columns are ``out_cols``; the caller keeps ownership).
 *
 * Work runs on ``cuda_stream`` (a cudaStream_t of the current device).  The
 * call synchronises that stream after each copy of its descriptors from host
 * memory (it has no pinned buffer) and to read the row count; the output
 * columns are complete when the stream's later work is.  The first call on a device
 * also looks up the array's device address, so make it before any stream
 * capture.  Every call shares the one array, and each call clears what must
 * start at zero, so calls whose device work overlaps (on two streams or two
 * threads) race and must be serialised by the caller.  Errors: INVALID (NULL,
 * sizes beyond the limits, unaligned buffers), UNSUPPORTED (more than two
 * shared variables, more than 2^32 result rows), BUDGET (output larger than
 * the capacity), CUDA, TIMEOUT. */
MAPSQ_API int mapsq_join_noalloc(const mapsq_table* left, const mapsq_table* right, uint32_t* const* out_cols,
                                 uint64_t out_capacity_rows, mapsq_table* out, uint64_t* out_rows,
                                 void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* MAPSQ_H */
