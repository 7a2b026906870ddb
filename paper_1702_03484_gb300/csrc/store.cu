// Device-resident triple store: dedup + per-predicate SO and OS orders.
//
// The paper matches each triple pattern with a CPU engine used as a black box
// (Section 2).  Here the graph lives in HBM as two sorted copies of its
// triples, (p, s, o) and (p, o, s), so that a pattern with a constant predicate
// and a constant subject or object is a binary search plus a contiguous slice.
// Sorting is a stable LSD radix sort over 8-bit digits of the three uint32
// columns; a pass whose digit is the same for every row is skipped.
#include <algorithm>

#include "internal.cuh"

namespace mapsq {

namespace {

constexpr int kRadixThreads = 256;
constexpr int kRadixIters = 16;
constexpr int kRadixTile = kRadixThreads * kRadixIters;
constexpr int kDigits = 256;

struct Cols3 {
  uint32_t* c[3];
};

__global__ void radix_histogram_kernel(const uint32_t* __restrict__ key, uint64_t n, int shift,
                                       uint32_t* __restrict__ hist, uint32_t ntiles) {
  __shared__ uint32_t h[kDigits];
  h[threadIdx.x] = 0;
  __syncthreads();
  uint64_t base = uint64_t(blockIdx.x) * kRadixTile;
  for (int it = 0; it < kRadixIters; ++it) {
    uint64_t i = base + uint64_t(it) * kRadixThreads + threadIdx.x;
    if (i < n) {
      uint32_t d = (key[i] >> shift) & 0xffu;
      // warp-aggregated increment: one shared atomic per distinct digit in the warp
      unsigned active = __activemask();
      unsigned peers = __match_any_sync(active, d);
      int leader = __ffs(peers) - 1;
      if ((threadIdx.x & 31) == leader) atomicAdd(&h[d], __popc(peers));
    }
  }
  __syncthreads();
  hist[uint64_t(threadIdx.x) * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void digit_totals_kernel(const uint32_t* __restrict__ offs, uint32_t ntiles, uint64_t n,
                                    uint64_t* __restrict__ totals) {
  int d = threadIdx.x;
  uint64_t a = offs[uint64_t(d) * ntiles];
  uint64_t b = d + 1 < kDigits ? offs[uint64_t(d + 1) * ntiles] : n;
  totals[d] = b - a;
}

// Stable scatter of one LSD pass: within a tile, rows keep their order per digit.
__global__ void radix_scatter_kernel(Cols3 src, Cols3 dst, int key_col, int shift, uint64_t n,
                                     const uint32_t* __restrict__ offs, uint32_t ntiles) {
  __shared__ uint32_t run[kDigits];
  __shared__ uint32_t wcnt[kRadixThreads / 32][kDigits];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  run[tid] = offs[uint64_t(tid) * ntiles + blockIdx.x];
  const unsigned lt_mask = (1u << lane) - 1u;
  uint64_t base = uint64_t(blockIdx.x) * kRadixTile;
  for (int it = 0; it < kRadixIters; ++it) {
#pragma unroll
    for (int w = 0; w < kRadixThreads / 32; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    uint64_t i = base + uint64_t(it) * kRadixThreads + tid;
    bool valid = i < n;
    uint32_t v0 = 0, v1 = 0, v2 = 0, d = kDigits;
    if (valid) {
      v0 = src.c[0][i];
      v1 = src.c[1][i];
      v2 = src.c[2][i];
      uint32_t k = key_col == 0 ? v0 : key_col == 1 ? v1 : v2;
      d = (k >> shift) & 0xffu;
    }
    unsigned peers = __match_any_sync(0xffffffffu, d);
    uint32_t rank = __popc(peers & lt_mask);
    if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t acc = run[tid];
#pragma unroll
      for (int w = 0; w < kRadixThreads / 32; ++w) {
        uint32_t c = wcnt[w][tid];
        wcnt[w][tid] = acc;
        acc += c;
      }
      run[tid] = acc;
    }
    __syncthreads();
    if (valid) {
      uint32_t pos = wcnt[warp][d] + rank;
      dst.c[0][pos] = v0;
      dst.c[1][pos] = v1;
      dst.c[2][pos] = v2;
    }
    __syncthreads();
  }
}

// keep[i] = 1 if triple i differs from triple i-1 (rows sorted, so equal triples are adjacent)
__global__ void dedup_flags_kernel(Cols3 t, uint64_t n, uint32_t* __restrict__ keep) {
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
    uint32_t k = 1;
    if (i > 0)
      k = (t.c[0][i] != t.c[0][i - 1]) | (t.c[1][i] != t.c[1][i - 1]) | (t.c[2][i] != t.c[2][i - 1]);
    keep[i] = k;
  }
}

__global__ void compact3_kernel(Cols3 src, Cols3 dst, uint64_t n, const uint32_t* __restrict__ keep,
                                const uint32_t* __restrict__ pos) {
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
    if (keep[i]) {
      uint32_t q = pos[i];
      dst.c[0][q] = src.c[0][i];
      dst.c[1][q] = src.c[1][i];
      dst.c[2][q] = src.c[2][i];
    }
  }
}

__global__ void pred_head_flags_kernel(const uint32_t* __restrict__ p, uint64_t n, uint32_t* __restrict__ head) {
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x)
    head[i] = (i == 0 || p[i] != p[i - 1]) ? 1u : 0u;
}

__global__ void pred_heads_kernel(const uint32_t* __restrict__ p, uint64_t n, const uint32_t* __restrict__ head,
                                  const uint32_t* __restrict__ pos, uint32_t* __restrict__ ids,
                                  uint64_t* __restrict__ begin) {
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x)
    if (head[i]) {
      ids[pos[i]] = p[i];
      begin[pos[i]] = i;
    }
}

unsigned grid_for(uint64_t n) { return unsigned(std::max<uint64_t>(1, std::min<uint64_t>(ceil_div(n, 256), 152ull * 32))); }

// LSD radix sort of three columns by the key columns listed least significant
// first.  Ping-pongs between ``a`` and ``b``; returns in *in_b whether the sorted
// rows ended in ``b``.
int radix_sort3(Ctx* ctx, Cols3 a, Cols3 b, uint64_t n, const int* key_cols, int nkeys, bool* in_b) {
  *in_b = false;
  if (n <= 1) return MAPSQ_OK;
  uint32_t ntiles = uint32_t(ceil_div(n, kRadixTile));
  Scratch scratch(ctx);
  uint32_t *hist = nullptr, *offs = nullptr;
  uint64_t* totals = nullptr;
  MQ_TRY(scratch.get(size_t(kDigits) * ntiles, &hist));
  MQ_TRY(scratch.get(size_t(kDigits) * ntiles + 1, &offs));
  MQ_TRY(scratch.get(kDigits, &totals));
  std::vector<uint64_t> host_tot(kDigits);
  uint64_t* pinned = nullptr;
  MQ_CUDA(cudaMallocHost(&pinned, kDigits * sizeof(uint64_t)));
  Cols3 cur = a, oth = b;
  bool cur_is_b = false;
  int rc = MAPSQ_OK;
  for (int k = 0; k < nkeys && rc == MAPSQ_OK; ++k) {
    for (int shift = 0; shift < 32; shift += 8) {
      int rec = prof_begin(ctx, K_STORE_HIST);
      radix_histogram_kernel<<<ntiles, kRadixThreads, 0, ctx->stream>>>(cur.c[key_cols[k]], n, shift, hist, ntiles);
      ++ctx->launches;
      prof_end(ctx, rec, double(n) * 4);
      if ((rc = prefix_sum_u32_u32(ctx, hist, offs, size_t(kDigits) * ntiles)) != MAPSQ_OK) break;
      digit_totals_kernel<<<1, kDigits, 0, ctx->stream>>>(offs, ntiles, n, totals);
      ++ctx->launches;
      cudaError_t e = cudaMemcpyAsync(pinned, totals, kDigits * sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) {
        rc = cuda_fail(ctx, e, "radix digit totals", __FILE__, __LINE__);
        break;
      }
      bool trivial = false;
      for (int d = 0; d < kDigits; ++d) trivial |= pinned[d] == n;
      if (trivial) continue;  // every row has the same digit: the pass keeps the order
      rec = prof_begin(ctx, K_STORE_SCATTER);
      radix_scatter_kernel<<<ntiles, kRadixThreads, 0, ctx->stream>>>(cur, oth, key_cols[k], shift, n, offs, ntiles);
      ++ctx->launches;
      prof_end(ctx, rec, double(n) * 24);
      e = cudaGetLastError();
      if (e != cudaSuccess) {
        rc = cuda_fail(ctx, e, "radix_scatter_kernel", __FILE__, __LINE__);
        break;
      }
      std::swap(cur, oth);
      cur_is_b = !cur_is_b;
    }
  }
  cudaStreamSynchronize(ctx->stream);
  cudaFreeHost(pinned);
  *in_b = cur_is_b;
  return rc;
}

}  // namespace

void store_release(Ctx* ctx) {
  Store& st = ctx->store;
  shared_release(ctx, st.shared);  // scan results that alias the store keep it alive
  st = Store{};
}

int store_build(Ctx* ctx, const uint32_t* s, const uint32_t* p, const uint32_t* o, uint64_t n, int on_device) {
  store_release(ctx);
  Store& st = ctx->store;
  Scratch scratch(ctx);
  Cols3 a{}, b{};
  uint64_t cap = std::max<uint64_t>(n, 1);
  for (int c = 0; c < 3; ++c) {
    MQ_TRY(scratch.get(cap, &a.c[c]));
    MQ_TRY(scratch.get(cap, &b.c[c]));
  }
  const uint32_t* in[3] = {s, p, o};
  for (int c = 0; c < 3 && n; ++c) {
    if (on_device) {
      MQ_TRY(copy_u32(ctx, a.c[c], in[c], n));
    } else {
      MQ_CUDA(cudaMemcpyAsync(a.c[c], in[c], n * sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream));
    }
  }
  // (p, s, o) order: least significant key first
  const int so_keys[3] = {2, 0, 1};
  bool in_b = false;
  MQ_TRY(radix_sort3(ctx, a, b, n, so_keys, 3, &in_b));
  Cols3 sorted = in_b ? b : a, other = in_b ? a : b;

  // dedup: RDF graphs are sets
  uint32_t *keep = nullptr, *pos = nullptr;
  MQ_TRY(scratch.get(cap, &keep));
  MQ_TRY(scratch.get(cap + 1, &pos));
  uint64_t m = 0;
  if (n) {
    int rec = prof_begin(ctx, K_STORE_DEDUP);
    dedup_flags_kernel<<<grid_for(n), 256, 0, ctx->stream>>>(sorted, n, keep);
    ++ctx->launches;
    prof_end(ctx, rec, double(n) * 16);
    MQ_TRY(prefix_sum_u32_u32(ctx, keep, pos, n));
    rec = prof_begin(ctx, K_STORE_DEDUP);
    compact3_kernel<<<grid_for(n), 256, 0, ctx->stream>>>(sorted, other, n, keep, pos);
    ++ctx->launches;
    prof_end(ctx, rec, double(n) * 32);
    MQ_CUDA(cudaGetLastError());
    uint32_t m32 = 0;
    MQ_CUDA(cudaMemcpyAsync(ctx->h_pinned, pos + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
    MQ_CUDA(cudaStreamSynchronize(ctx->stream));
    memcpy(&m32, ctx->h_pinned, sizeof(uint32_t));
    m = m32;
  }
  Cols3 dd = other;  // deduped (p, s, o)-sorted triples, m rows

  // predicate segments
  std::vector<uint32_t> pid;
  std::vector<uint64_t> pbeg;
  if (m) {
    uint32_t* head = keep;  // reuse
    int rec = prof_begin(ctx, K_PRED_HEADS);
    pred_head_flags_kernel<<<grid_for(m), 256, 0, ctx->stream>>>(dd.c[1], m, head);
    ++ctx->launches;
    prof_end(ctx, rec, double(m) * 8);
    MQ_TRY(prefix_sum_u32_u32(ctx, head, pos, m));
    uint32_t nh = 0;
    MQ_CUDA(cudaMemcpyAsync(ctx->h_pinned, pos + m, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
    MQ_CUDA(cudaStreamSynchronize(ctx->stream));
    memcpy(&nh, ctx->h_pinned, sizeof(uint32_t));
    uint32_t* ids = nullptr;
    uint64_t* beg = nullptr;
    MQ_TRY(scratch.get(nh, &ids));
    MQ_TRY(scratch.get(nh, &beg));
    pred_heads_kernel<<<grid_for(m), 256, 0, ctx->stream>>>(dd.c[1], m, head, pos, ids, beg);
    ++ctx->launches;
    MQ_CUDA(cudaGetLastError());
    pid.resize(nh);
    pbeg.resize(nh + 1);
    MQ_CUDA(cudaMemcpyAsync(pid.data(), ids, nh * sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
    MQ_CUDA(cudaMemcpyAsync(pbeg.data(), beg, nh * sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream));
    MQ_CUDA(cudaStreamSynchronize(ctx->stream));
    pbeg[nh] = m;
  } else {
    pbeg.assign(1, 0);
  }

  // the store block: so_s, so_o, os_o, os_s
  uint64_t stride = (std::max<uint64_t>(m, 1) + 63) & ~uint64_t(63);
  size_t bytes = size_t(stride) * 4 * sizeof(uint32_t);
  void* blk = nullptr;
  MQ_TRY(dev_alloc(ctx, bytes, &blk));
  uint32_t* base = static_cast<uint32_t*>(blk);
  st.shared = new SharedBlock{blk, bytes, 1};
  st.so_s = base;
  st.so_o = base + stride;
  st.os_o = base + 2 * stride;
  st.os_s = base + 3 * stride;
  MQ_TRY(copy_u32(ctx, st.so_s, dd.c[0], m));
  MQ_TRY(copy_u32(ctx, st.so_o, dd.c[2], m));

  // (p, o, s) order of the deduped triples, sorted from the (p, s, o) copy
  Cols3 x = dd, y = sorted;
  const int os_keys[3] = {0, 2, 1};
  MQ_TRY(radix_sort3(ctx, x, y, m, os_keys, 3, &in_b));
  Cols3 os = in_b ? y : x;
  MQ_TRY(copy_u32(ctx, st.os_o, os.c[2], m));
  MQ_TRY(copy_u32(ctx, st.os_s, os.c[0], m));
  MQ_CUDA(cudaStreamSynchronize(ctx->stream));
  st.n = m;
  st.pred_id = std::move(pid);
  st.pred_begin = std::move(pbeg);
  st.loaded = true;
  return MAPSQ_OK;
}

}  // namespace mapsq
