// C ABI entry points: contexts, memory, tables, profiling, and the BGP planner
// (the host side of the paper's CPU/GPU coprocessing split, Section 2).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <new>

#include "internal.cuh"

namespace mapsq {

const char* const kKernelNames[K_COUNT_KERNELS] = {
    "store_radix_histogram", "store_radix_scatter", "store_dedup", "store_predicate_heads",
    "scan_ranges",           "scan_emit",           "scan_filter", "prefix_sum",
    "hash_insert",           "hash_scatter",        "probe_count", "join_write",
    "cross_write",           "copy",        "hll_sketch",  "write_partition", "sorted_count", "dense_write",
    "partition_build", "star_count", "star_write", "fused_join"};

int set_error(Ctx* ctx, int code, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return code;
}

int cuda_fail(Ctx* ctx, cudaError_t e, const char* what, const char* file, int line) {
  return set_error(ctx, MAPSQ_ERR_CUDA, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

int dev_alloc(Ctx* ctx, size_t bytes, void** out) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  if (ctx->budget && ctx->in_use + bytes > ctx->budget)
    return set_error(ctx, MAPSQ_ERR_BUDGET, "allocation of %zu bytes exceeds the budget (%llu in use of %llu)",
                     bytes, (unsigned long long)ctx->in_use, (unsigned long long)ctx->budget);
  void* p = nullptr;
  if (ctx->has_allocator) {
    p = ctx->allocator.alloc(bytes, ctx->allocator.user, ctx->stream);
  } else {
    cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, ctx->pool, ctx->stream);
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      p = nullptr;
    } else if (e != cudaSuccess) {
      return cuda_fail(ctx, e, "cudaMallocFromPoolAsync", __FILE__, __LINE__);
    }
  }
  if (!p) return set_error(ctx, MAPSQ_ERR_OOM, "device allocation of %zu bytes failed", bytes);
  ctx->in_use += bytes;
  ctx->peak = std::max(ctx->peak, ctx->in_use);
  *out = p;
  return MAPSQ_OK;
}

void dev_free(Ctx* ctx, void* p, size_t bytes) {
  if (!p) return;
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  if (ctx->has_allocator)
    ctx->allocator.free(p, bytes, ctx->allocator.user, ctx->stream);
  else
    cudaFreeAsync(p, ctx->stream);
  ctx->in_use -= std::min<uint64_t>(ctx->in_use, bytes);
}

int table_alloc(Ctx* ctx, uint64_t nrows, uint32_t ncols, const int32_t* var, TableImpl** out) {
  if (ncols > MAPSQ_MAX_VARS) return set_error(ctx, MAPSQ_ERR_INVALID, "table with %u columns", ncols);
  TableImpl* t = new (std::nothrow) TableImpl();
  if (!t) return set_error(ctx, MAPSQ_ERR_OOM, "host allocation failed");
  t->magic = kTableMagic;
  t->pub.nrows = nrows;
  t->pub.ncols = ncols;
  t->pub.on_device = 1;
  for (uint32_t c = 0; c < MAPSQ_MAX_VARS; ++c) {
    t->pub.var[c] = c < ncols ? var[c] : -1;
    t->pub.col[c] = nullptr;
  }
  // stride rounded to 64 rows: every column starts 256-byte aligned
  uint64_t stride = (nrows + 63) & ~uint64_t(63);
  size_t bytes = size_t(stride) * ncols * sizeof(uint32_t);
  if (bytes) {
    int rc = dev_alloc(ctx, bytes, &t->block);
    if (rc != MAPSQ_OK) {
      delete t;
      return rc;
    }
    t->bytes = bytes;
    for (uint32_t c = 0; c < ncols; ++c) t->pub.col[c] = static_cast<uint32_t*>(t->block) + stride * c;
  }
  ctx->live_tables.push_back(t);
  *out = t;
  return MAPSQ_OK;
}

int table_view(Ctx* ctx, uint64_t nrows, uint32_t ncols, const int32_t* var, uint32_t* const* cols,
               SharedBlock* owner, TableImpl** out) {
  TableImpl* t = new (std::nothrow) TableImpl();
  if (!t) return set_error(ctx, MAPSQ_ERR_OOM, "host allocation failed");
  t->magic = kTableMagic;
  t->pub.nrows = nrows;
  t->pub.ncols = ncols;
  t->pub.on_device = 1;
  for (uint32_t c = 0; c < MAPSQ_MAX_VARS; ++c) {
    t->pub.var[c] = c < ncols ? var[c] : -1;
    t->pub.col[c] = c < ncols ? cols[c] : nullptr;
  }
  t->view = owner;
  ++owner->refs;
  ctx->live_tables.push_back(t);
  *out = t;
  return MAPSQ_OK;
}

// The result tables of a batch in one device allocation: each table is a
// view of its part (columns 256-byte aligned, as table_alloc lays them out),
// and the block goes when the last of the tables is released.
int tables_alloc_shared(Ctx* ctx, uint32_t k, const uint64_t* nrows, const uint32_t* ncols,
                        const int32_t* const* var, TableImpl** out) {
  std::vector<size_t> off(k, 0), stride(k, 0);
  size_t total = 0;
  for (uint32_t j = 0; j < k; ++j) {
    if (ncols[j] > MAPSQ_MAX_VARS) return set_error(ctx, MAPSQ_ERR_INVALID, "table with %u columns", ncols[j]);
    stride[j] = size_t((nrows[j] + 63) & ~uint64_t(63));
    off[j] = total;
    total += (stride[j] * ncols[j] * sizeof(uint32_t) + 255) & ~size_t(255);
  }
  if (total == 0) {  // no columns or no rows anywhere: nothing to share
    for (uint32_t j = 0; j < k; ++j) {
      const int rc = table_alloc(ctx, nrows[j], ncols[j], var[j], &out[j]);
      if (rc != MAPSQ_OK) {
        for (uint32_t i = 0; i < j; ++i) table_release(ctx, out[i]);
        return rc;
      }
    }
    return MAPSQ_OK;
  }
  SharedBlock* b = new (std::nothrow) SharedBlock();
  if (!b) return set_error(ctx, MAPSQ_ERR_OOM, "host allocation failed");
  int rc = dev_alloc(ctx, total, &b->ptr);
  if (rc != MAPSQ_OK) {
    delete b;
    return rc;
  }
  b->bytes = total;
  uint32_t made = 0;
  for (; made < k && rc == MAPSQ_OK; ++made) {
    uint32_t* cols[MAPSQ_MAX_VARS] = {};
    for (uint32_t c = 0; c < ncols[made]; ++c)
      cols[c] = reinterpret_cast<uint32_t*>(static_cast<char*>(b->ptr) + off[made]) + stride[made] * c;
    rc = table_view(ctx, nrows[made], ncols[made], var[made], cols, b, &out[made]);
    if (rc == MAPSQ_OK) out[made]->bytes = stride[made] * ncols[made] * sizeof(uint32_t);
    else break;
  }
  if (rc != MAPSQ_OK) {
    if (made == 0) {
      dev_free(ctx, b->ptr, b->bytes);
      delete b;
    }
    for (uint32_t i = 0; i < made; ++i) table_release(ctx, out[i]);  // the last one frees the block
    return rc;
  }
  return MAPSQ_OK;
}

void shared_release(Ctx* ctx, SharedBlock* b) {
  if (!b || --b->refs > 0) return;
  dev_free(ctx, b->ptr, b->bytes);
  delete b;
}

void table_release(Ctx* ctx, TableImpl* t) {
  if (!t) return;
  auto it = std::find(ctx->live_tables.begin(), ctx->live_tables.end(), t);
  if (it == ctx->live_tables.end()) return;  // not ours, or already released
  ctx->live_tables.erase(it);
  if (t->view)
    shared_release(ctx, t->view);
  else
    dev_free(ctx, t->block, t->bytes);
  t->magic = 0;
  delete t;
}

int prof_begin(Ctx* ctx, int kid) {
  if (!ctx->profiling || (ctx->profile_only >= 0 && ctx->profile_only != kid)) return -1;
  LaunchRecord r{kid, nullptr, nullptr, 0.0};
  for (cudaEvent_t* e : {&r.start, &r.stop}) {
    if (!ctx->free_events.empty()) {
      *e = ctx->free_events.back();
      ctx->free_events.pop_back();
    } else if (cudaEventCreate(e) != cudaSuccess) {
      return -1;
    }
  }
  cudaEventRecord(r.start, ctx->stream);
  ctx->pending.push_back(r);
  return int(ctx->pending.size()) - 1;
}

void prof_end(Ctx* ctx, int rec, double alg_bytes) {
  if (rec < 0 || !ctx->profiling || rec >= int(ctx->pending.size())) return;
  cudaEventRecord(ctx->pending[rec].stop, ctx->stream);
  ctx->pending[rec].bytes = alg_bytes;
}

static int drain_profile(Ctx* ctx) {
  if (ctx->pending.empty()) return MAPSQ_OK;
  MQ_CUDA(cudaStreamSynchronize(ctx->stream));
  for (auto& r : ctx->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.start, r.stop) == cudaSuccess) {
      ctx->totals[r.kid].launches += 1;
      ctx->totals[r.kid].ms += ms;
      ctx->totals[r.kid].bytes += r.bytes;
    }
    ctx->free_events.push_back(r.start);
    ctx->free_events.push_back(r.stop);
  }
  ctx->pending.clear();
  return MAPSQ_OK;
}

int stage_upload(Ctx* ctx, void* dst, const void* src, size_t bytes) {
  if (bytes == 0) return MAPSQ_OK;
  // Slots are used in order; an event is recorded after the last slot of each
  // half of the ring, and a slot is reused only after the event of its half
  // (recorded after the slot's previous copy was queued) has completed.
  const int s = ctx->stage_next;
  ctx->stage_next = (s + 1) % Ctx::kStageSlots;
  constexpr int kHalf = Ctx::kStageSlots / 2;
  const int mark = (s / kHalf) * kHalf + kHalf - 1;  // the slot whose event covers this half
  if (ctx->stage_done[mark]) MQ_CUDA(cudaEventSynchronize(ctx->stage_done[mark]));
  if (bytes > ctx->h_stage_bytes[s]) {
    if (ctx->h_stage[s]) cudaFreeHost(ctx->h_stage[s]);
    ctx->h_stage[s] = nullptr;
    ctx->h_stage_bytes[s] = 0;
    const size_t cap = std::max<size_t>(bytes, 64 << 10);
    MQ_CUDA(cudaMallocHost(&ctx->h_stage[s], cap));
    ctx->h_stage_bytes[s] = cap;
  }
  memcpy(ctx->h_stage[s], src, bytes);
  MQ_CUDA(cudaMemcpyAsync(dst, ctx->h_stage[s], bytes, cudaMemcpyHostToDevice, ctx->stream));
  if (s == mark) {
    if (!ctx->stage_done[s]) MQ_CUDA(cudaEventCreateWithFlags(&ctx->stage_done[s], cudaEventDisableTiming));
    MQ_CUDA(cudaEventRecord(ctx->stage_done[s], ctx->stream));
  }
  return MAPSQ_OK;
}

int read_u64(Ctx* ctx, const void* dptr, uint64_t* host, int count) {
  if (count < 1 || count > 32) return set_error(ctx, MAPSQ_ERR_INVALID, "read_u64 of %d words", count);
  return read_words(ctx, dptr, size_t(count), host);
}

namespace {

// Copies n words and the status word to mapped host memory, then (after a
// system-scope fence, so that the host sees them first) the sequence number.
__global__ void publish_kernel(const uint64_t* __restrict__ src, uint32_t n, const uint32_t* __restrict__ status,
                               uint64_t* dst, uint64_t seq) {
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) dst[2 + i] = src[i];
  if (threadIdx.x == 0) dst[1] = *status;
  __threadfence_system();
  __syncthreads();
  if (threadIdx.x == 0) *reinterpret_cast<volatile uint64_t*>(dst) = seq;
}

constexpr auto kPublishPoll = std::chrono::microseconds(500);  // then block in cudaStreamSynchronize

}  // namespace

int read_words(Ctx* ctx, const void* dptr, size_t n, uint64_t* host) {
  if (n > kReadWords) return set_error(ctx, MAPSQ_ERR_INVALID, "read of %zu words", n);
  const uint64_t seq = ++ctx->mapped_seq;
  publish_kernel<<<1, 256, 0, ctx->stream>>>(static_cast<const uint64_t*>(dptr), uint32_t(n), ctx->d_status,
                                             ctx->d_mapped, seq);
  ++ctx->launches;
  MQ_CUDA(cudaGetLastError());
  const auto t0 = std::chrono::steady_clock::now();
  bool seen = false;
  for (uint32_t i = 1;; ++i) {
    if (__atomic_load_n(ctx->h_mapped, __ATOMIC_ACQUIRE) == seq) {
      seen = true;
      break;
    }
    if (!(i & 63) && std::chrono::steady_clock::now() - t0 > kPublishPoll) break;
  }
  if (!seen) {
    MQ_CUDA(cudaStreamSynchronize(ctx->stream));
    if (__atomic_load_n(ctx->h_mapped, __ATOMIC_ACQUIRE) != seq)
      return set_error(ctx, MAPSQ_ERR_CUDA, "published read %llu missing after synchronisation",
                       (unsigned long long)seq);
  }
  if (n) memcpy(host, ctx->h_mapped + 2, n * sizeof(uint64_t));
  ctx->h_pinned[32] = ctx->h_mapped[1] & 0xFFFFFFFFu;
  return check_status(ctx);
}

void dict_release(Ctx* ctx) {
  if (ctx->dict_off) dev_free(ctx, ctx->dict_off, (uint64_t(ctx->dict_terms) + 1) * 8);
  if (ctx->dict_bytes) dev_free(ctx, ctx->dict_bytes, std::max<uint64_t>(ctx->dict_nbytes, 1));
  ctx->dict_off = nullptr;
  ctx->dict_bytes = nullptr;
  ctx->dict_terms = 0;
  ctx->dict_nbytes = 0;
}

int check_status(Ctx* ctx) {
  // h_pinned[32] holds the status word read by the last synchronising call
  uint32_t st = uint32_t(ctx->h_pinned[32] & 0xFFFFFFFFu);
  if (st == 0) return MAPSQ_OK;
  ctx->h_pinned[32] = 0;
  MQ_CUDA(cudaMemsetAsync(ctx->d_status, 0, sizeof(uint32_t), ctx->stream));
  if (st & 2u) return set_error(ctx, MAPSQ_ERR_TIMEOUT, "a bounded device wait gave up (status 0x%x)", st);
  if (st & kStatusBounds) return set_error(ctx, MAPSQ_ERR_CUDA, "a device bounds check failed (status 0x%x)", st);
  return set_error(ctx, MAPSQ_ERR_CUDA, "device status 0x%x (hash table full or index out of range)", st);
}

int checked_sync(Ctx* ctx) {
#ifdef MAPSQ_CHECKED
  MQ_CUDA(cudaMemcpyAsync(ctx->h_pinned + 32, ctx->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
  MQ_CUDA(cudaStreamSynchronize(ctx->stream));
  return check_status(ctx);
#else
  (void)ctx;
  return MAPSQ_OK;
#endif
}

}  // namespace mapsq

using namespace mapsq;

extern "C" {

const char* mapsq_strerror(int status) {
  switch (status) {
    case MAPSQ_OK: return "ok";
    case MAPSQ_ERR_INVALID: return "invalid argument";
    case MAPSQ_ERR_UNSUPPORTED: return "unsupported";
    case MAPSQ_ERR_OOM: return "out of device memory";
    case MAPSQ_ERR_BUDGET: return "memory budget exceeded";
    case MAPSQ_ERR_CUDA: return "CUDA error";
    case MAPSQ_ERR_TIMEOUT: return "device wait timed out";
    case MAPSQ_ERR_BUSY: return "busy";
    case MAPSQ_ERR_NOT_FOUND: return "not found";
    default: return "unknown status";
  }
}

const char* mapsq_last_error(const mapsq_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

const char* mapsq_build_info(void) {
#ifdef MAPSQ_CHECKED
  return "sm_103a checked";
#else
  return "sm_103a";
#endif
}

int mapsq_create(mapsq_ctx** out, int device, const mapsq_allocator* allocator, void* cuda_stream,
                 uint64_t mem_budget_bytes) {
  if (!out) return MAPSQ_ERR_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return MAPSQ_ERR_INVALID;
  }
  if (allocator && (!allocator->alloc || !allocator->free)) return MAPSQ_ERR_INVALID;
  Ctx* ctx = new (std::nothrow) Ctx();
  if (!ctx) return MAPSQ_ERR_OOM;
  ctx->device = device;
  ctx->budget = mem_budget_bytes;
  int rc = MAPSQ_OK;
  auto fail = [&](int code) {
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    if (ctx->h_mapped) cudaFreeHost(ctx->h_mapped);
    delete ctx;
    return code;
  };
  if (cudaSetDevice(device) != cudaSuccess) return fail(MAPSQ_ERR_CUDA);
  if (cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) != cudaSuccess) return fail(MAPSQ_ERR_CUDA);
  ctx->stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : ctx->own_stream;
  if (allocator) {
    ctx->has_allocator = true;
    ctx->allocator = *allocator;
  } else {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&ctx->pool, &props) != cudaSuccess) return fail(MAPSQ_ERR_CUDA);
    uint64_t keep = UINT64_MAX;  // keep freed blocks cached in the pool
    cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  if (cudaMallocHost(&ctx->h_pinned, kPinnedWords * sizeof(uint64_t)) != cudaSuccess) return fail(MAPSQ_ERR_CUDA);
  memset(ctx->h_pinned, 0, kPinnedWords * sizeof(uint64_t));
  if (cudaHostAlloc(&ctx->h_mapped, kMappedWords * sizeof(uint64_t), cudaHostAllocMapped) != cudaSuccess)
    return fail(MAPSQ_ERR_CUDA);
  memset(ctx->h_mapped, 0, kMappedWords * sizeof(uint64_t));
  void* dm = nullptr;
  if (cudaHostGetDevicePointer(&dm, ctx->h_mapped, 0) != cudaSuccess) return fail(MAPSQ_ERR_CUDA);
  ctx->d_mapped = static_cast<uint64_t*>(dm);
  void* st = nullptr;
  rc = dev_alloc(ctx, 256, &st);
  if (rc != MAPSQ_OK) return fail(rc);
  ctx->d_status = static_cast<uint32_t*>(st);
  if (cudaMemsetAsync(ctx->d_status, 0, 256, ctx->stream) != cudaSuccess) return fail(MAPSQ_ERR_CUDA);
  *out = ctx;
  return MAPSQ_OK;
}

int mapsq_destroy(mapsq_ctx* ctx) {
  if (!ctx) return MAPSQ_OK;
  server_shutdown(ctx);
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto& r : ctx->pending) {
    cudaEventDestroy(r.start);
    cudaEventDestroy(r.stop);
  }
  for (auto e : ctx->free_events) cudaEventDestroy(e);
  while (!ctx->live_tables.empty()) table_release(ctx, ctx->live_tables.back());
  for (void* p : ctx->chunk_cache) dev_free(ctx, p, Scratch::kChunk);
  ctx->chunk_cache.clear();
  store_release(ctx);
  dict_release(ctx);
  dev_free(ctx, ctx->d_status, 256);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
  if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
  if (ctx->h_mapped) cudaFreeHost(ctx->h_mapped);
  for (int s = 0; s < Ctx::kStageSlots; ++s) {
    if (ctx->h_stage[s]) cudaFreeHost(ctx->h_stage[s]);
    if (ctx->stage_done[s]) cudaEventDestroy(ctx->stage_done[s]);
  }
  if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
  delete ctx;
  return MAPSQ_OK;
}

int mapsq_set_stream(mapsq_ctx* ctx, void* cuda_stream) {
  if (!ctx) return MAPSQ_ERR_INVALID;
  if (ctx->server) return set_error(ctx, MAPSQ_ERR_BUSY, "the serving loop is running");
  // memory released to the context in the old stream's order (cached scratch) must be idle first
  MQ_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : ctx->own_stream;
  return MAPSQ_OK;
}

int mapsq_load_triples(mapsq_ctx* ctx, const uint32_t* s, const uint32_t* p, const uint32_t* o, uint64_t n,
                       int ptrs_on_device) {
  if (!ctx) return MAPSQ_ERR_INVALID;
  if (ctx->server) return set_error(ctx, MAPSQ_ERR_BUSY, "the serving loop is running");
  if (n && (!s || !p || !o)) return set_error(ctx, MAPSQ_ERR_INVALID, "NULL triple column");
  if (n >= (uint64_t(1) << 32)) return set_error(ctx, MAPSQ_ERR_INVALID, "at most 2^32-1 triples");
  MQ_CUDA(cudaSetDevice(ctx->device));
  return store_build(ctx, s, p, o, n, ptrs_on_device);
}

int mapsq_store_info(mapsq_ctx* ctx, uint64_t* n_triples, uint32_t* n_predicates) {
  if (!ctx) return MAPSQ_ERR_INVALID;
  std::lock_guard<std::recursive_mutex> cl(ctx->mu);
  if (n_triples) *n_triples = ctx->store.n;
  if (n_predicates) *n_predicates = uint32_t(ctx->store.pred_id.size());
  return MAPSQ_OK;
}

int mapsq_scan_pattern(mapsq_ctx* ctx, const mapsq_pattern* tp, mapsq_table** out) {
  if (!ctx || !tp || !out) return ctx ? set_error(ctx, MAPSQ_ERR_INVALID, "NULL argument") : MAPSQ_ERR_INVALID;
  if (ctx->server) return set_error(ctx, MAPSQ_ERR_BUSY, "the serving loop is running");
  MQ_CUDA(cudaSetDevice(ctx->device));
  MQ_TRY(validate_pattern(ctx, *tp));
  if (!ctx->store.loaded) return set_error(ctx, MAPSQ_ERR_INVALID, "no triple store loaded");
  PatternRange r;
  MQ_TRY(scan_ranges(ctx, tp, 1, &r));
  TableImpl* t = nullptr;
  MQ_TRY(scan_emit(ctx, *tp, r, &t));
  *out = &t->pub;
  return MAPSQ_OK;
}

int mapsq_join(mapsq_ctx* ctx, const mapsq_table* left, const mapsq_table* right, mapsq_table** out,
               const mapsq_join_opts* opts) {
  if (!ctx || !left || !right || !out)
    return ctx ? set_error(ctx, MAPSQ_ERR_INVALID, "NULL argument") : MAPSQ_ERR_INVALID;
  if (ctx->server) return set_error(ctx, MAPSQ_ERR_BUSY, "the serving loop is running");
  MQ_CUDA(cudaSetDevice(ctx->device));
  TableImpl* t = nullptr;
  MQ_TRY(join_tables(ctx, left, right, opts, &t));
  *out = &t->pub;
  return MAPSQ_OK;
}

int mapsq_join_to_host(mapsq_ctx* ctx, const mapsq_table* left, const mapsq_table* right,
                       const mapsq_join_opts* opts, uint32_t* const* host_cols, uint64_t capacity_rows,
                       uint64_t* out_rows, mapsq_table* out, uint32_t* slices) {
  if (!ctx || !left || !right || !out_rows)
    return ctx ? set_error(ctx, MAPSQ_ERR_INVALID, "NULL argument") : MAPSQ_ERR_INVALID;
  if (ctx->server) return set_error(ctx, MAPSQ_ERR_BUSY, "the serving loop is running");
  MQ_CUDA(cudaSetDevice(ctx->device));
  return join_to_host(ctx, left, right, opts, host_cols, capacity_rows, out_rows, out, slices);
}

int mapsq_join_batch(mapsq_ctx* ctx, uint32_t k, const mapsq_table* const* left, const mapsq_table* const* right,
                     mapsq_table** out, const mapsq_join_opts* opts) {
  if (!ctx || (k && (!left || !right || !out)))
    return ctx ? set_error(ctx, MAPSQ_ERR_INVALID, "NULL argument") : MAPSQ_ERR_INVALID;
  if (ctx->server) return set_error(ctx, MAPSQ_ERR_BUSY, "the serving loop is running");
  MQ_CUDA(cudaSetDevice(ctx->device));
  std::vector<TableImpl*> t(k, nullptr);
  MQ_TRY(join_batch(ctx, k, left, right, opts, t.data()));
  for (uint32_t j = 0; j < k; ++j) out[j] = &t[j]->pub;
  return MAPSQ_OK;
}

int mapsq_table_from_columns(mapsq_ctx* ctx, uint64_t nrows, uint32_t ncols, const int32_t* var,
                             const uint32_t* const* cols, int on_device, mapsq_table** out) {
  if (!ctx || !out || (ncols && (!var || !cols)))
    return ctx ? set_error(ctx, MAPSQ_ERR_INVALID, "NULL argument") : MAPSQ_ERR_INVALID;
  if (ctx->server) return set_error(ctx, MAPSQ_ERR_BUSY, "the serving loop is running");
  if (ncols > MAPSQ_MAX_VARS) return set_error(ctx, MAPSQ_ERR_INVALID, "more than 16 columns");
  if (ncols == 0 && nrows > 1) return set_error(ctx, MAPSQ_ERR_INVALID, "a 0-column table has 0 or 1 rows");
  uint32_t seen = 0;
  for (uint32_t c = 0; c < ncols; ++c) {
    if (var[c] < 0 || var[c] >= MAPSQ_MAX_VARS) return set_error(ctx, MAPSQ_ERR_INVALID, "variable id %d", var[c]);
    if (seen & (1u << var[c])) return set_error(ctx, MAPSQ_ERR_INVALID, "variable %d twice", var[c]);
    seen |= 1u << var[c];
    if (nrows && !cols[c]) return set_error(ctx, MAPSQ_ERR_INVALID, "NULL column %u", c);
  }
  MQ_CUDA(cudaSetDevice(ctx->device));
  TableImpl* t = nullptr;
  MQ_TRY(table_alloc(ctx, nrows, ncols, var, &t));
  for (uint32_t c = 0; c < ncols && nrows; ++c) {
    cudaError_t e;
    if (on_device) {
      int rc = copy_u32(ctx, t->pub.col[c], cols[c], nrows);
      if (rc != MAPSQ_OK) {
        table_release(ctx, t);
        return rc;
      }
      continue;
    }
    e = cudaMemcpyAsync(t->pub.col[c], cols[c], nrows * sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) {
      table_release(ctx, t);
      return cuda_fail(ctx, e, "cudaMemcpyAsync", __FILE__, __LINE__);
    }
  }
  // host sources are borrowed for the call only
  if (!on_device) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
      table_release(ctx, t);
      return cuda_fail(ctx, e, "cudaStreamSynchronize", __FILE__, __LINE__);
    }
  }
  *out = &t->pub;
  return MAPSQ_OK;
}

int mapsq_table_to_host(mapsq_ctx* ctx, const mapsq_table* t, uint32_t* const* host_cols) {
  if (!ctx || !t || (t->ncols && !host_cols))
    return ctx ? set_error(ctx, MAPSQ_ERR_INVALID, "NULL argument") : MAPSQ_ERR_INVALID;
  std::lock_guard<std::recursive_mutex> cl(ctx->mu);
  MQ_CUDA(cudaSetDevice(ctx->device));
  for (uint32_t c = 0; c < t->ncols && t->nrows; ++c) {
    if (!host_cols[c]) return set_error(ctx, MAPSQ_ERR_INVALID, "NULL host column %u", c);
    MQ_CUDA(cudaMemcpyAsync(host_cols[c], t->col[c], t->nrows * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                            ctx->stream));
  }
  MQ_CUDA(cudaStreamSynchronize(ctx->stream));
  return MAPSQ_OK;
}

void mapsq_table_free(mapsq_ctx* ctx, mapsq_table* t) {
  if (!ctx || !t) return;
  std::lock_guard<std::recursive_mutex> cl(ctx->mu);
  TableImpl* impl = reinterpret_cast<TableImpl*>(t);
  table_release(ctx, impl);
}

int mapsq_sync(mapsq_ctx* ctx) {
  if (!ctx) return MAPSQ_ERR_INVALID;
  std::lock_guard<std::recursive_mutex> cl(ctx->mu);
  MQ_CUDA(cudaSetDevice(ctx->device));
  return read_words(ctx, nullptr, 0, nullptr);  // every queued operation has run once it returns
}

int mapsq_set_wait_limit(mapsq_ctx* ctx, uint32_t spins) {
  if (!ctx) return MAPSQ_ERR_INVALID;
  if (spins == 0) return set_error(ctx, MAPSQ_ERR_INVALID, "a wait limit of 0 polls");
  std::lock_guard<std::recursive_mutex> cl(ctx->mu);
  ctx->wait_spins = spins;
  return MAPSQ_OK;
}

int mapsq_selftest_wait(mapsq_ctx* ctx, uint32_t spins) {
  if (!ctx) return MAPSQ_ERR_INVALID;
  if (spins == 0) return set_error(ctx, MAPSQ_ERR_INVALID, "a wait limit of 0 polls");
  if (ctx->server) return set_error(ctx, MAPSQ_ERR_BUSY, "the serving loop is running");
  MQ_CUDA(cudaSetDevice(ctx->device));
  constexpr uint64_t n = 4 * 4096;  // four look-back tiles
  int rc = MAPSQ_OK;
  {
    Scratch scratch(ctx);
    uint32_t* in = nullptr;
    uint64_t* out = nullptr;
    MQ_TRY(scratch.get(n, &in));
    MQ_TRY(scratch.get(n + 1, &out));
    MQ_CUDA(cudaMemsetAsync(in, 0, n * sizeof(uint32_t), ctx->stream));
    const uint32_t saved = ctx->wait_spins;
    ctx->wait_spins = spins;
    rc = prefix_sum_withheld(ctx, in, out, n);
    ctx->wait_spins = saved;
  }
  MQ_TRY(rc);
  MQ_CUDA(cudaMemcpyAsync(ctx->h_pinned + 32, ctx->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
  MQ_CUDA(cudaStreamSynchronize(ctx->stream));
  return check_status(ctx);
}

int mapsq_memory_in_use(mapsq_ctx* ctx, uint64_t* bytes, uint64_t* peak_bytes) {
  if (!ctx) return MAPSQ_ERR_INVALID;
  std::lock_guard<std::recursive_mutex> cl(ctx->mu);
  if (bytes) *bytes = ctx->in_use;
  if (peak_bytes) *peak_bytes = ctx->peak;
  return MAPSQ_OK;
}

int mapsq_set_profiling(mapsq_ctx* ctx, int enable) {
  if (!ctx) return MAPSQ_ERR_INVALID;
  std::lock_guard<std::recursive_mutex> cl(ctx->mu);
  if (!enable) MQ_TRY(drain_profile(ctx));
  ctx->profiling = enable != 0;
  return MAPSQ_OK;
}

int mapsq_kernel_stats(mapsq_ctx* ctx, mapsq_kernel_stat* out, uint32_t cap, uint32_t* n) {
  if (!ctx || !n || (cap && !out)) return MAPSQ_ERR_INVALID;
  std::lock_guard<std::recursive_mutex> cl(ctx->mu);
  MQ_TRY(drain_profile(ctx));
  uint32_t k = 0;
  for (int i = 0; i < K_COUNT_KERNELS; ++i) {
    if (!ctx->totals[i].launches) continue;
    if (k < cap) {
      memset(&out[k], 0, sizeof(mapsq_kernel_stat));
      strncpy(out[k].name, kKernelNames[i], sizeof(out[k].name) - 1);
      out[k].launches = ctx->totals[i].launches;
      out[k].device_ms = ctx->totals[i].ms;
      out[k].alg_bytes = ctx->totals[i].bytes;
    }
    ++k;
  }
  *n = k;
  return MAPSQ_OK;
}

int mapsq_launch_count(mapsq_ctx* ctx, uint64_t* launches) {
  if (!ctx || !launches) return MAPSQ_ERR_INVALID;
  std::lock_guard<std::recursive_mutex> cl(ctx->mu);
  *launches = ctx->launches;
  return MAPSQ_OK;
}

int mapsq_profile_only(mapsq_ctx* ctx, const char* name) {
  if (!ctx) return MAPSQ_ERR_INVALID;
  std::lock_guard<std::recursive_mutex> cl(ctx->mu);
  if (!name) {
    ctx->profile_only = -1;
    return MAPSQ_OK;
  }
  for (int i = 0; i < K_COUNT_KERNELS; ++i)
    if (strcmp(name, kKernelNames[i]) == 0) {
      ctx->profile_only = i;
      return MAPSQ_OK;
    }
  return set_error(ctx, MAPSQ_ERR_INVALID, "unknown kernel kind %s", name);
}

int mapsq_reset_stats(mapsq_ctx* ctx) {
  if (!ctx) return MAPSQ_ERR_INVALID;
  std::lock_guard<std::recursive_mutex> cl(ctx->mu);
  MQ_TRY(drain_profile(ctx));
  for (auto& t : ctx->totals) t = KernelTotals{};
  return MAPSQ_OK;
}

}  // extern "C"
