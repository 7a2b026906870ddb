// Internal declarations shared by the translation units of libmapsq.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "mapsq.h"

// Device bounds checks of the checked build (compiled with -DMAPSQ_CHECKED,
// libmapsq_checked.so): a failed check sets bit 4 (16) of the given status
// word and the access is skipped, never a trap; the call that launched the
// kernel reports it after a synchronisation.  In the regular build the checks
// are not compiled.
#ifdef MAPSQ_CHECKED
#define MQ_IN_BOUNDS(cond, status) ((cond) || (atomicOr((status), 16u), false))
#else
#define MQ_IN_BOUNDS(cond, status) true
#endif

namespace mapsq {

constexpr size_t kPinnedWords = 4096;
constexpr size_t kReadWords = 4096;      // words one published read carries (read_words)
constexpr size_t kMappedWords = 2 + kReadWords;
constexpr uint32_t kStatusBounds = 16u;  // status bit of a failed bounds check (checked build)

// Kernels timed by the profiling switch (mapsq_set_profiling).
enum KernelId {
  K_STORE_HIST = 0,
  K_STORE_SCATTER,
  K_STORE_DEDUP,
  K_PRED_HEADS,
  K_SCAN_RANGES,
  K_SCAN_EMIT,
  K_SCAN_FILTER,
  K_PREFIX_SUM,
  K_HASH_INSERT,
  K_HASH_SCATTER,
  K_PROBE_COUNT,
  K_JOIN_WRITE,
  K_CROSS_WRITE,
  K_COPY,
  K_HLL,
  K_PARTITION,
  K_SORTED_COUNT,
  K_DENSE_WRITE,
  K_PARTITION_BUILD,
  K_STAR_COUNT,
  K_STAR_WRITE,
  K_FUSED_JOIN,
  K_COUNT_KERNELS
};

extern const char* const kKernelNames[K_COUNT_KERNELS];

// A device allocation shared by its owner and the tables that alias it (the
// triple store and the scan results that are slices of it); freed when the
// last reference goes.
struct SharedBlock {
  void* ptr = nullptr;
  size_t bytes = 0;
  int refs = 0;
};

// A library-owned table: the public struct first, so a mapsq_table* handed out
// by the library converts back to its TableImpl.
struct TableImpl {
  mapsq_table pub;
  void* block;         // one allocation holding every column, or NULL for a view
  size_t bytes;
  uint32_t magic;
  SharedBlock* view;   // the block a view's columns alias, or NULL
};
constexpr uint32_t kTableMagic = 0x7AB1E5u;

// Device-resident triple store: per predicate, SO- and OS-sorted column pairs.
struct Store {
  bool loaded = false;
  uint64_t n = 0;                   // distinct triples
  std::vector<uint32_t> pred_id;    // sorted distinct predicate ids (host mirror)
  std::vector<uint64_t> pred_begin; // segment [pred_begin[k], pred_begin[k+1]) of predicate pred_id[k]
  uint32_t* so_s = nullptr;         // sorted by (p, s, o)
  uint32_t* so_o = nullptr;
  uint32_t* os_o = nullptr;         // sorted by (p, o, s)
  uint32_t* os_s = nullptr;
  SharedBlock* shared = nullptr;    // the four columns' allocation
};

struct LaunchRecord {
  int kid;
  cudaEvent_t start, stop;
  double bytes;
};

struct KernelTotals {
  uint64_t launches = 0;
  double ms = 0.0;
  double bytes = 0.0;
};

}  // namespace mapsq

namespace mapsq {
struct Server;
}

struct mapsq_ctx {
  int device = 0;
  std::recursive_mutex mu;           // held by the serving loop for a round, and by calls that may run meanwhile
  mapsq::Server* server = nullptr;   // serving loop, while started
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  bool has_allocator = false;
  mapsq_allocator allocator{};
  cudaMemPool_t pool = nullptr;
  uint64_t budget = 0;
  uint64_t in_use = 0;
  uint64_t peak = 0;
  std::string err;
  mapsq::Store store;
  uint32_t* d_status = nullptr;    // device status word: 0 = fine
  uint64_t* h_pinned = nullptr;    // pinned buffer for device->host reads (kPinnedWords words)
  // host memory the device writes directly (mapped): [0] sequence number of
  // the last published read, [1] status word, [2..] the read's words
  uint64_t* h_mapped = nullptr;
  uint64_t* d_mapped = nullptr;    // the same memory's device address
  uint64_t mapped_seq = 0;
  // ring of pinned staging buffers for host->device uploads; an upload reuses a
  // buffer only after the copy that last read it has run
  static constexpr int kStageSlots = 8;
  void* h_stage[kStageSlots] = {};
  size_t h_stage_bytes[kStageSlots] = {};
  cudaEvent_t stage_done[kStageSlots] = {};
  int stage_next = 0;
  bool profiling = false;
  int profile_only = -1;          // kernel id to profile alone, or -1 for all
  uint64_t launches = 0;          // kernels launched by this context
  std::vector<mapsq::LaunchRecord> pending;
  std::vector<cudaEvent_t> free_events;
  mapsq::KernelTotals totals[mapsq::K_COUNT_KERNELS];
  std::vector<mapsq::TableImpl*> live_tables;
  uint32_t sorted_ratio = 4;      // AUTO joins: sorted side rows / other side rows from which SORTED runs
  uint32_t wait_spins = 1u << 20; // polls of a bounded device wait before it gives up (mapsq_set_wait_limit)
  uint64_t part_min_build = 1u << 16;  // hash builds of at least this many rows are partitioned first (autotuned)
  uint64_t dense_max = 16;             // joins of at most this many matches per probe row: dense write (autotuned)
  // term dictionary for mapsq_decode (device): id i is dict_bytes[dict_off[i] .. dict_off[i + 1])
  uint64_t* dict_off = nullptr;
  char* dict_bytes = nullptr;
  uint32_t dict_terms = 0;
  uint64_t dict_nbytes = 0;
  // scratch chunks kept for the next call (reused in stream order on ``stream``)
  static constexpr int kChunkCache = 4;
  std::vector<void*> chunk_cache;
};

namespace mapsq {

using Ctx = mapsq_ctx;

int set_error(Ctx* ctx, int code, const char* fmt, ...);
int cuda_fail(Ctx* ctx, cudaError_t e, const char* what, const char* file, int line);

#define MQ_CUDA(call)                                                     \
  do {                                                                    \
    cudaError_t e_ = (call);                                              \
    if (e_ != cudaSuccess) return ::mapsq::cuda_fail(ctx, e_, #call, __FILE__, __LINE__); \
  } while (0)

#define MQ_TRY(call)         \
  do {                       \
    int rc_ = (call);        \
    if (rc_ != MAPSQ_OK) return rc_; \
  } while (0)

// Device memory through the context's allocator, counted against its budget.
int dev_alloc(Ctx* ctx, size_t bytes, void** out);
void dev_free(Ctx* ctx, void* p, size_t bytes);

// RAII holder for scratch allocations inside one call: requests are carved
// (256-byte aligned) from chunks of at least kChunk bytes, so that a join's
// dozen small arrays cost one allocation and one free.
struct Scratch {
  static constexpr size_t kChunk = size_t(256) << 10;
  Ctx* ctx;
  std::vector<std::pair<void*, size_t>> blocks;
  char* cur = nullptr;
  size_t left = 0;
  explicit Scratch(Ctx* c) : ctx(c) {}
  ~Scratch() {
    for (auto& b : blocks) {
      if (b.second == kChunk && int(ctx->chunk_cache.size()) < Ctx::kChunkCache)
        ctx->chunk_cache.push_back(b.first);  // work queued on the stream still reads it: reuse is stream-ordered
      else
        dev_free(ctx, b.first, b.second);
    }
  }
  // Carved regions stay allocated until the destructor: a rewind is a no-op
  // (the interface matches the fixed-array carver, which reuses its space).
  size_t mark() const { return 0; }
  void rewind(size_t) {}
  // One block for the requests that follow (a batch's per-join arrays), so
  // that they cost one device allocation instead of one each.  A hint: if the
  // block cannot be had, each request allocates as before.
  int reserve(size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes <= left || bytes <= kChunk) return MAPSQ_OK;
    void* p = nullptr;
    const std::string before = ctx->err;
    if (dev_alloc(ctx, bytes, &p) != MAPSQ_OK) {
      ctx->err = before;  // not an error of the call: its requests allocate one by one
      return MAPSQ_OK;
    }
    blocks.push_back({p, bytes});
    cur = static_cast<char*>(p);
    left = bytes;
    return MAPSQ_OK;
  }
  template <class T>
  int get(size_t count, T** out) {
    size_t bytes = count * sizeof(T);
    bytes = ((bytes ? bytes : 16) + 255) & ~size_t(255);
    if (bytes > left) {
      void* p = nullptr;
      size_t chunk = bytes < kChunk ? kChunk : bytes;
      int rc = MAPSQ_OK;
      if (chunk == kChunk && !ctx->chunk_cache.empty()) {
        p = ctx->chunk_cache.back();
        ctx->chunk_cache.pop_back();
      } else {
        rc = dev_alloc(ctx, chunk, &p);
      }
      if (rc == MAPSQ_ERR_BUDGET && chunk > bytes) rc = dev_alloc(ctx, chunk = bytes, &p);  // just what fits
      if (rc != MAPSQ_OK) return rc;
      blocks.push_back({p, chunk});
      cur = static_cast<char*>(p);
      left = chunk;
    }
    *out = reinterpret_cast<T*>(cur);
    cur += bytes;
    left -= bytes;
    return MAPSQ_OK;
  }
};

// Allocate a library-owned table with room for nrows x ncols (columns 256-byte aligned).
int table_alloc(Ctx* ctx, uint64_t nrows, uint32_t ncols, const int32_t* var, TableImpl** out);
// A table whose columns alias ``owner`` (which gains a reference).
int table_view(Ctx* ctx, uint64_t nrows, uint32_t ncols, const int32_t* var, uint32_t* const* cols,
               SharedBlock* owner, TableImpl** out);
void table_release(Ctx* ctx, TableImpl* t);
void shared_release(Ctx* ctx, SharedBlock* b);
int tables_alloc_shared(Ctx* ctx, uint32_t k, const uint64_t* nrows, const uint32_t* ncols,
                        const int32_t* const* var, TableImpl** out);

// Profiling brackets around one launch (no-ops while profiling is off).
int prof_begin(Ctx* ctx, int kid);
void prof_end(Ctx* ctx, int rec, double alg_bytes);

// Copy ``bytes`` host bytes to device memory ``dst`` on the context's stream
// through the pinned staging buffer (waits for the previous upload to leave it).
int stage_upload(Ctx* ctx, void* dst, const void* src, size_t bytes);

// Read a few 64-bit words back from the device (synchronises the stream).
int read_u64(Ctx* ctx, const void* dptr, uint64_t* host, int count);
// ``n`` (at most kReadWords) 64-bit words at ``dptr`` into host[0, n), with the
// status word checked, once every earlier operation of the stream has run: a
// one-block kernel writes them and a sequence number into mapped host memory,
// the host polls that number for a short while, then falls back to a stream
// synchronisation (long steps, and errors).  Costs one launch and no copy.
int read_words(Ctx* ctx, const void* dptr, size_t n, uint64_t* host);

// Frees the term dictionary (mapsq_dict_load, mapsq_destroy).
void dict_release(Ctx* ctx);

// SELECT (select.cu): columns of ``t`` holding ``vars``, DISTINCT with MAPSQ_DISTINCT.
int project_table(Ctx* ctx, const mapsq_table* t, uint32_t nvars, const int32_t* vars, uint32_t flags,
                  TableImpl** out);

// Serving loop (serve.cu): stops and frees it (mapsq_destroy).
void server_shutdown(Ctx* ctx);

// Device status word check after a synchronisation.
int check_status(Ctx* ctx);
// In the checked build: synchronise and report the context's status word (no-op otherwise).
int checked_sync(Ctx* ctx);

// Primitives (prim.cu).
// out[0..n] = exclusive prefix sums of in[0..n), out[n] = total.
int prefix_sum_u32_u64(Ctx* ctx, const uint32_t* in, uint64_t* out, uint64_t n);
int prefix_sum_u32_u32(Ctx* ctx, const uint32_t* in, uint32_t* out, uint64_t n);
// The same scan with its first tile withheld (every look-back wait runs out).
int prefix_sum_withheld(Ctx* ctx, const uint32_t* in, uint64_t* out, uint64_t n);
int copy_u32(Ctx* ctx, uint32_t* dst, const uint32_t* src, uint64_t n);

// Store (store.cu).
int store_build(Ctx* ctx, const uint32_t* s, const uint32_t* p, const uint32_t* o, uint64_t n, int on_device);
void store_release(Ctx* ctx);

// Pattern scan (scan.cu).
enum ScanKind : int32_t {
  KIND_NONE = 0,    // predicate not in the store: no match
  KIND_EXIST = 1,   // s and o constant
  KIND_S_BOUND = 2, // s constant, o variable
  KIND_O_BOUND = 3, // o constant, s variable
  KIND_TWO_VARS = 4,
  KIND_SAME_VAR = 5
};
struct PatternRange {
  uint64_t lo, hi;  // row range in the chosen order; hi - lo = matches (before the s==o filter)
  int32_t order;    // 0: SO columns, 1: OS columns, -1: no match
  int32_t kind;     // a ScanKind
};
int validate_pattern(Ctx* ctx, const mapsq_pattern& tp);
int scan_ranges(Ctx* ctx, const mapsq_pattern* tps, uint32_t n, PatternRange* out);
// ``key_var``: the variable the result will be joined on (or -1); a pattern
// with two variables is returned in the store order sorted by it.
int scan_emit(Ctx* ctx, const mapsq_pattern& tp, const PatternRange& r, TableImpl** out, int32_t key_var = -1);
// Columns of ``t`` reordered by ascending variable id (sorted_mask follows).
void canonical_columns(mapsq_table* t);
// The one variable that table ``t`` shares with pattern ``tp``, or -1 (none or two).
int32_t shared_var(const mapsq_table& t, const mapsq_pattern& tp);

// Join (join.cu): k independent joins in one batch of launches.
int join_tables(Ctx* ctx, const mapsq_table* L, const mapsq_table* R, const mapsq_join_opts* opts,
                TableImpl** out);
int join_batch(Ctx* ctx, uint32_t k, const mapsq_table* const* L, const mapsq_table* const* R,
               const mapsq_join_opts* opts, TableImpl** out);

// Star join (star.cu): k tables sharing only ``key_var``, in one count and write round.
int join_star(Ctx* ctx, uint32_t k, const mapsq_table* const* tabs, int32_t key_var, TableImpl** out);

// A join into caller host columns, slice by slice of its larger input (mapsq_join_to_host).
int join_to_host(Ctx* ctx, const mapsq_table* L, const mapsq_table* R, const mapsq_join_opts* opts,
                 uint32_t* const* host_cols, uint64_t capacity, uint64_t* out_rows, mapsq_table* out,
                 uint32_t* slices);

// Counts k joins, then writes, in order, those whose results fit together in
// ``budget_bytes`` (0 = all): status[j] = 0 written (out[j] set), 1 deferred;
// need[j] = bytes of join j's result table.
int join_batch_admit(Ctx* ctx, uint32_t k, const mapsq_table* const* L, const mapsq_table* const* R,
                     uint64_t budget_bytes, TableImpl** out, int* status, uint64_t* need);

// BGP evaluation (query.cu): pattern order, and many BGPs level by level.
std::vector<uint32_t> plan_order(const mapsq_pattern* bgp, uint32_t n, const PatternRange* ranges);
int query_batch(Ctx* ctx, uint32_t nq, const mapsq_pattern* const* bgps, const uint32_t* ns, TableImpl** out);

inline uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

}  // namespace mapsq
