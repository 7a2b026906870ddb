// The SELECT clause of a query over BGP solutions (Section 1: query Q selects
// ?person from the solutions of its two patterns): projection onto chosen
// variables, optionally DISTINCT, and decoding of term ids back to strings
// through a device-resident dictionary.
//
// Projection keeps every row (SPARQL's default bag semantics) and is a column
// gather.  DISTINCT inserts every row's index into an open-addressing table
// of 2^m row ids (at least twice the rows) keyed by a hash of the row's
// values: the first row to claim a slot owns it, a later row reaching an owned
// slot compares its values with the owner's and is a duplicate when they are
// equal; the kept rows are then compacted in row order by a prefix sum.
// Decoding looks each id's string up in the dictionary (offsets and bytes),
// sizes the output with a prefix sum of the lengths and copies the bytes.
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace mapsq {

namespace {

constexpr uint32_t kEmptyRow = 0xffffffffu;
constexpr int kSelThreads = 256;

struct ColSet {
  const uint32_t* src[MAPSQ_MAX_VARS];
  uint32_t* dst[MAPSQ_MAX_VARS];
  int n;
};

unsigned grid_for(uint64_t n) { return unsigned(std::min<uint64_t>(ceil_div(std::max<uint64_t>(n, 1), kSelThreads), 152ull * 16)); }

__global__ void gather_columns_kernel(ColSet cs, uint64_t n) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
    for (int c = 0; c < cs.n; ++c) cs.dst[c][i] = __ldg(cs.src[c] + i);
}

// 64-bit hash of a row's values (each value mixed in turn with a multiply and
// a xor-shift, then MurmurHash3's finaliser).
__device__ __forceinline__ uint64_t row_hash(const ColSet& cs, uint64_t i) {
  uint64_t h = 0x9e3779b97f4a7c15ull;
  for (int c = 0; c < cs.n; ++c) {
    h = (h ^ __ldg(cs.src[c] + i)) * 0xff51afd7ed558ccdull;
    h ^= h >> 29;
  }
  h ^= h >> 33;
  h *= 0xc4ceb9fe1a85ec53ull;
  h ^= h >> 33;
  return h;
}

__device__ __forceinline__ bool rows_equal(const ColSet& cs, uint64_t a, uint64_t b) {
  for (int c = 0; c < cs.n; ++c)
    if (__ldg(cs.src[c] + a) != __ldg(cs.src[c] + b)) return false;
  return true;
}

// keep[i] = 1 if row i owns the slot of its values, 0 if an equal row does.
__global__ void distinct_kernel(ColSet cs, uint64_t n, uint32_t* __restrict__ table, uint32_t mask,
                                uint32_t* __restrict__ keep, uint32_t* __restrict__ status) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    uint32_t slot = uint32_t(row_hash(cs, i)) & mask;
    uint32_t k = 0;
    bool done = false;
    for (uint32_t probes = 0; probes <= mask && !done; ++probes) {
      uint32_t owner = table[slot];
      if (owner == kEmptyRow) {
        owner = atomicCAS(table + slot, kEmptyRow, uint32_t(i));
        if (owner == kEmptyRow) {
          k = 1;
          done = true;
          break;
        }
      }
      if (rows_equal(cs, owner, i)) {
        done = true;
        break;
      }
      slot = (slot + 1) & mask;
    }
    if (!done) atomicOr(status, 1u);  // the table was full: cannot happen at half load
    keep[i] = k;
  }
}

// Kept rows to their place: pos[i] = number of kept rows before row i.
__global__ void compact_kernel(ColSet cs, uint64_t n, const uint32_t* __restrict__ keep,
                               const uint64_t* __restrict__ pos) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
    if (keep[i]) {
      const uint64_t o = pos[i];
      for (int c = 0; c < cs.n; ++c) cs.dst[c][o] = __ldg(cs.src[c] + i);
    }
}

// Length of each row's string; an id without a term sets bit 1 of the status word.
__global__ void decode_len_kernel(const uint32_t* __restrict__ ids, uint64_t n, const uint64_t* __restrict__ off,
                                  uint32_t n_terms, uint32_t* __restrict__ len, uint32_t* __restrict__ status) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t id = __ldg(ids + i);
    if (id >= n_terms) {
      atomicOr(status, 1u);
      len[i] = 0;
    } else {
      len[i] = uint32_t(__ldg(off + id + 1) - __ldg(off + id));
    }
  }
}

__global__ void decode_copy_kernel(const uint32_t* __restrict__ ids, uint64_t n, const uint64_t* __restrict__ off,
                                   uint32_t n_terms, const char* __restrict__ bytes, const uint64_t* __restrict__ pos,
                                   char* __restrict__ out) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t id = __ldg(ids + i);
    if (id >= n_terms) continue;
    const uint64_t a = __ldg(off + id), b = __ldg(off + id + 1);
    char* dst = out + pos[i];
    for (uint64_t q = a; q < b; ++q) dst[q - a] = bytes[q];
  }
}

int check_device_table(Ctx* ctx, const mapsq_table* t) {
  if (t->ncols > MAPSQ_MAX_VARS) return set_error(ctx, MAPSQ_ERR_INVALID, "table with %u columns", t->ncols);
  if (t->ncols && t->nrows && !t->on_device) return set_error(ctx, MAPSQ_ERR_INVALID, "columns must be on the device");
  for (uint32_t c = 0; c < t->ncols; ++c)
    if (t->nrows && (!t->col[c] || (reinterpret_cast<uintptr_t>(t->col[c]) & 3)))
      return set_error(ctx, MAPSQ_ERR_INVALID, "column %u is NULL or not 4-byte aligned", c);
  return MAPSQ_OK;
}

// Status word after a synchronising read: 0 or an error of this call.
int take_status(Ctx* ctx, const uint32_t* d_word, const char* what) {
  uint32_t st = 0;
  MQ_CUDA(cudaMemcpyAsync(ctx->h_pinned + 40, d_word, sizeof st, cudaMemcpyDeviceToHost, ctx->stream));
  MQ_CUDA(cudaStreamSynchronize(ctx->stream));
  memcpy(&st, ctx->h_pinned + 40, sizeof st);
  return st ? set_error(ctx, MAPSQ_ERR_INVALID, "%s", what) : MAPSQ_OK;
}

}  // namespace

int project_table(Ctx* ctx, const mapsq_table* t, uint32_t nvars, const int32_t* vars, uint32_t flags,
                  TableImpl** out) {
  if (flags & ~uint32_t(MAPSQ_DISTINCT)) return set_error(ctx, MAPSQ_ERR_INVALID, "unknown flags 0x%x", flags);
  if (nvars == 0 || nvars > MAPSQ_MAX_VARS || !vars)
    return set_error(ctx, MAPSQ_ERR_INVALID, "select %u variables", nvars);
  MQ_TRY(check_device_table(ctx, t));
  ColSet src{};
  src.n = int(nvars);
  for (uint32_t v = 0; v < nvars; ++v) {
    int found = -1;
    for (uint32_t c = 0; c < t->ncols; ++c)
      if (t->var[c] == vars[v]) found = int(c);
    if (found < 0) return set_error(ctx, MAPSQ_ERR_INVALID, "variable %d is not a column of the table", vars[v]);
    for (uint32_t w = 0; w < v; ++w)
      if (vars[w] == vars[v]) return set_error(ctx, MAPSQ_ERR_INVALID, "variable %d selected twice", vars[v]);
    src.src[v] = t->col[found];
  }
  const uint64_t n = t->nrows;
  if (!(flags & MAPSQ_DISTINCT) || n <= 1) {
    TableImpl* r = nullptr;
    MQ_TRY(table_alloc(ctx, n, nvars, vars, &r));
    ColSet cs = src;
    for (uint32_t v = 0; v < nvars; ++v) cs.dst[v] = r->pub.col[v];
    if (n) {
      gather_columns_kernel<<<grid_for(n), kSelThreads, 0, ctx->stream>>>(cs, n);
      ++ctx->launches;
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) {
        table_release(ctx, r);
        return cuda_fail(ctx, e, "gather_columns_kernel", __FILE__, __LINE__);
      }
    }
    *out = r;
    return MAPSQ_OK;
  }
  if (n > (uint64_t(1) << 31))
    return set_error(ctx, MAPSQ_ERR_UNSUPPORTED, "DISTINCT over %llu rows (at most 2^31)", (unsigned long long)n);
  uint64_t m = 1;
  while (m < 2 * n) m <<= 1;
  Scratch scratch(ctx);
  uint32_t *table = nullptr, *keep = nullptr, *status = nullptr;
  uint64_t* pos = nullptr;
  MQ_TRY(scratch.get(m, &table));
  MQ_TRY(scratch.get(n, &keep));
  MQ_TRY(scratch.get(n + 1, &pos));
  MQ_TRY(scratch.get(1, &status));
  MQ_CUDA(cudaMemsetAsync(table, 0xff, m * 4, ctx->stream));
  MQ_CUDA(cudaMemsetAsync(status, 0, 4, ctx->stream));
  distinct_kernel<<<grid_for(n), kSelThreads, 0, ctx->stream>>>(src, n, table, uint32_t(m - 1), keep, status);
  ++ctx->launches;
  MQ_CUDA(cudaGetLastError());
  MQ_TRY(prefix_sum_u32_u64(ctx, keep, pos, n));
  uint64_t kept = 0;
  MQ_TRY(read_u64(ctx, pos + n, &kept, 1));
  MQ_TRY(take_status(ctx, status, "DISTINCT table full"));
  TableImpl* r = nullptr;
  MQ_TRY(table_alloc(ctx, kept, nvars, vars, &r));
  ColSet cs = src;
  for (uint32_t v = 0; v < nvars; ++v) cs.dst[v] = r->pub.col[v];
  if (kept) {
    compact_kernel<<<grid_for(n), kSelThreads, 0, ctx->stream>>>(cs, n, keep, pos);
    ++ctx->launches;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      table_release(ctx, r);
      return cuda_fail(ctx, e, "compact_kernel", __FILE__, __LINE__);
    }
  }
  *out = r;
  return MAPSQ_OK;
}

}  // namespace mapsq

using namespace mapsq;

extern "C" {

int mapsq_project(mapsq_ctx* ctx, const mapsq_table* t, uint32_t nvars, const int32_t* vars, uint32_t flags,
                  mapsq_table** out) {
  if (!ctx || !t || !out) return ctx ? set_error(ctx, MAPSQ_ERR_INVALID, "NULL argument") : MAPSQ_ERR_INVALID;
  if (ctx->server) return set_error(ctx, MAPSQ_ERR_BUSY, "the serving loop is running");
  MQ_CUDA(cudaSetDevice(ctx->device));
  TableImpl* r = nullptr;
  MQ_TRY(project_table(ctx, t, nvars, vars, flags, &r));
  *out = &r->pub;
  return MAPSQ_OK;
}

int mapsq_query_select(mapsq_ctx* ctx, const mapsq_pattern* bgp, uint32_t n, uint32_t nvars, const int32_t* vars,
                       uint32_t flags, mapsq_table** out) {
  if (!ctx || !out) return ctx ? set_error(ctx, MAPSQ_ERR_INVALID, "NULL argument") : MAPSQ_ERR_INVALID;
  mapsq_table* all = nullptr;
  MQ_TRY(mapsq_query(ctx, bgp, n, &all));
  TableImpl* r = nullptr;
  const int rc = project_table(ctx, all, nvars, vars, flags, &r);
  table_release(ctx, reinterpret_cast<TableImpl*>(all));
  if (rc != MAPSQ_OK) return rc;
  *out = &r->pub;
  return MAPSQ_OK;
}

int mapsq_dict_load(mapsq_ctx* ctx, const uint64_t* offsets, const char* bytes, uint32_t n_terms) {
  if (!ctx || !offsets || (!bytes && offsets[n_terms]))
    return ctx ? set_error(ctx, MAPSQ_ERR_INVALID, "NULL argument") : MAPSQ_ERR_INVALID;
  if (ctx->server) return set_error(ctx, MAPSQ_ERR_BUSY, "the serving loop is running");
  for (uint32_t i = 0; i < n_terms; ++i)
    if (offsets[i + 1] < offsets[i]) return set_error(ctx, MAPSQ_ERR_INVALID, "dictionary offsets decrease at %u", i);
  if (offsets[0] != 0) return set_error(ctx, MAPSQ_ERR_INVALID, "dictionary offsets do not start at 0");
  MQ_CUDA(cudaSetDevice(ctx->device));
  const uint64_t nbytes = offsets[n_terms];
  void *d_off = nullptr, *d_bytes = nullptr;
  MQ_TRY(dev_alloc(ctx, (uint64_t(n_terms) + 1) * 8, &d_off));
  const int rc = dev_alloc(ctx, std::max<uint64_t>(nbytes, 1), &d_bytes);
  if (rc != MAPSQ_OK) {
    dev_free(ctx, d_off, (uint64_t(n_terms) + 1) * 8);
    return rc;
  }
  cudaError_t e = cudaMemcpyAsync(d_off, offsets, (uint64_t(n_terms) + 1) * 8, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess && nbytes) e = cudaMemcpyAsync(d_bytes, bytes, nbytes, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);  // pageable sources: wait before they go away
  if (e != cudaSuccess) {
    dev_free(ctx, d_off, (uint64_t(n_terms) + 1) * 8);
    dev_free(ctx, d_bytes, std::max<uint64_t>(nbytes, 1));
    return cuda_fail(ctx, e, "dictionary upload", __FILE__, __LINE__);
  }
  dict_release(ctx);
  ctx->dict_off = static_cast<uint64_t*>(d_off);
  ctx->dict_bytes = static_cast<char*>(d_bytes);
  ctx->dict_terms = n_terms;
  ctx->dict_nbytes = nbytes;
  return MAPSQ_OK;
}

int mapsq_decode(mapsq_ctx* ctx, const mapsq_table* t, uint32_t col, uint64_t* offsets, char* bytes, uint64_t cap,
                 uint64_t* nbytes) {
  if (!ctx || !t || !offsets || !nbytes)
    return ctx ? set_error(ctx, MAPSQ_ERR_INVALID, "NULL argument") : MAPSQ_ERR_INVALID;
  if (!ctx->dict_off) return set_error(ctx, MAPSQ_ERR_INVALID, "no dictionary loaded");
  if (col >= t->ncols) return set_error(ctx, MAPSQ_ERR_INVALID, "column %u of a %u-column table", col, t->ncols);
  MQ_TRY(check_device_table(ctx, t));
  MQ_CUDA(cudaSetDevice(ctx->device));
  const uint64_t n = t->nrows;
  if (n == 0) {
    offsets[0] = 0;
    *nbytes = 0;
    return MAPSQ_OK;
  }
  Scratch scratch(ctx);
  uint32_t *len = nullptr, *status = nullptr;
  uint64_t* pos = nullptr;
  MQ_TRY(scratch.get(n, &len));
  MQ_TRY(scratch.get(n + 1, &pos));
  MQ_TRY(scratch.get(1, &status));
  MQ_CUDA(cudaMemsetAsync(status, 0, 4, ctx->stream));
  decode_len_kernel<<<grid_for(n), kSelThreads, 0, ctx->stream>>>(t->col[col], n, ctx->dict_off, ctx->dict_terms,
                                                                   len, status);
  ++ctx->launches;
  MQ_CUDA(cudaGetLastError());
  MQ_TRY(prefix_sum_u32_u64(ctx, len, pos, n));
  MQ_CUDA(cudaMemcpyAsync(offsets, pos, (n + 1) * 8, cudaMemcpyDeviceToHost, ctx->stream));
  MQ_TRY(take_status(ctx, status, "a term id has no entry in the dictionary"));
  const uint64_t total = offsets[n];
  *nbytes = total;
  if (!bytes || total > cap || total == 0) return MAPSQ_OK;
  char* d_out = nullptr;
  MQ_TRY(scratch.get(total, &d_out));
  decode_copy_kernel<<<grid_for(n), kSelThreads, 0, ctx->stream>>>(t->col[col], n, ctx->dict_off, ctx->dict_terms,
                                                                    ctx->dict_bytes, pos, d_out);
  ++ctx->launches;
  MQ_CUDA(cudaGetLastError());
  MQ_CUDA(cudaMemcpyAsync(bytes, d_out, total, cudaMemcpyDeviceToHost, ctx->stream));
  MQ_CUDA(cudaStreamSynchronize(ctx->stream));
  return MAPSQ_OK;
}

}  // extern "C"
