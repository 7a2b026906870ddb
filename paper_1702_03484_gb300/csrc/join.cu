// MapSQ's MapReduce-based join (Algorithm 1) as a hash shuffle plus a
// count / prefix-sum / write reduce.
//
// Map: every row of both tables is mapped to its key, the shared variables
// packed into 64 bits (one variable: the id; two: smaller variable id in the
// high word), and keeps its other columns as its value (by row index).
// Shuffle: the smaller table (the build side) is partitioned by key through an
// open-addressing hash table: one insert pass gives each row its key group and
// its rank inside the group (warp-aggregated atomics), a prefix sum over the
// groups' sizes gives each group's start, and a scatter pass writes the build
// side's value columns grouped by key.  Reduce: every row of the other table
// (the probe side) looks its key up and counts its matches (the size of its
// LEFT x RIGHT cross product); an exclusive prefix sum of the counts gives each
// probe row its output range; the write pass then emits every LEFT x RIGHT pair
// exactly once, partitioned by output position so that skewed keys are spread
// over all SMs, with 16-byte streaming stores into each output column.
//
// Output layout (Table 1(c)): shared variables in ascending id, then the left
// table's other columns, then the right table's.  No shared variable: the cross
// product, one key group holding every row.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "internal.cuh"
#include "lookback.cuh"

namespace mapsq {

namespace {

constexpr uint64_t kEmptyKey = ~0ull;
constexpr int kWriteThreads = 256;
constexpr int kWriteGroups = 4;                                     // 4-row groups per thread per tile
constexpr int kWriteTile = kWriteThreads * kWriteGroups * 4;        // output rows per tile
constexpr int kOffCache = 2048;                                     // offsets cached in shared memory

struct __align__(16) Slot {
  uint64_t key;
  uint32_t cnt;
  uint32_t beg;
};

struct KeyCols {
  const uint32_t* c0;  // variable with the smaller id (high word when two)
  const uint32_t* c1;  // nullptr for a single-variable key
};

__device__ __forceinline__ uint64_t load_key(const KeyCols& k, uint64_t i) {
  uint64_t a = k.c0[i];
  return k.c1 ? (a << 32) | k.c1[i] : a;
}

// MurmurHash3's 64-bit finaliser (Appleby), a bijective mix of the key bits.
__device__ __forceinline__ uint64_t mix_key(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

// Home slot in [0, M): multiply-shift range reduction of the mixed key.
__device__ __forceinline__ uint32_t home_slot(uint64_t key, uint32_t M) {
  return uint32_t(((mix_key(key) >> 32) * uint64_t(M)) >> 32);
}

__global__ void hash_init_kernel(Slot* __restrict__ tab, uint32_t* __restrict__ cnt, uint64_t nslots) {
  for (uint64_t j = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < nslots; j += uint64_t(gridDim.x) * blockDim.x) {
    tab[j] = Slot{kEmptyKey, 0u, 0u};
    cnt[j] = 0u;
  }
}

// Insert every build row's key; slot_of[i] = its group's slot, rank_of[i] = its
// rank inside the group.  The key equal to the empty marker lives in slot M.
__global__ void hash_insert_kernel(KeyCols bk, uint64_t nb, Slot* __restrict__ tab, uint32_t* __restrict__ cnt,
                                   uint32_t M, uint32_t* __restrict__ slot_of, uint32_t* __restrict__ rank_of,
                                   uint32_t* __restrict__ status) {
  const unsigned lane = threadIdx.x & 31;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t base = uint64_t(blockIdx.x) * blockDim.x; base < nb; base += stride) {
    uint64_t i = base + threadIdx.x;
    bool valid = i < nb;
    uint32_t s = 0xffffffffu;
    if (valid) {
      uint64_t key = load_key(bk, i);
      if (key == kEmptyKey) {
        s = M;
      } else {
        uint32_t h = home_slot(key, M);
        for (uint32_t probe = 0; probe < M; ++probe) {
          uint64_t k = *reinterpret_cast<volatile uint64_t*>(&tab[h].key);
          if (k == key) { s = h; break; }
          if (k == kEmptyKey) {
            unsigned long long prev = atomicCAS(reinterpret_cast<unsigned long long*>(&tab[h].key),
                                                (unsigned long long)kEmptyKey, (unsigned long long)key);
            if (prev == kEmptyKey || prev == key) { s = h; break; }
          }
          h = h + 1 == M ? 0 : h + 1;
        }
        if (s == 0xffffffffu) atomicOr(status, 1u);  // table full: the host retries larger
      }
    }
    // warp-aggregated group ranks: one atomic per distinct slot in the warp
    unsigned peers = __match_any_sync(0xffffffffu, s);
    int leader = __ffs(peers) - 1;
    uint32_t base_rank = 0;
    if (lane == unsigned(leader) && valid && s != 0xffffffffu) base_rank = atomicAdd(&cnt[s], __popc(peers));
    base_rank = __shfl_sync(0xffffffffu, base_rank, leader);
    if (valid) {
      slot_of[i] = s;
      rank_of[i] = base_rank + __popc(peers & ((1u << lane) - 1u));
    }
  }
}

__global__ void hash_finalize_kernel(Slot* __restrict__ tab, const uint32_t* __restrict__ cnt,
                                     const uint32_t* __restrict__ beg, uint64_t nslots) {
  for (uint64_t j = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < nslots; j += uint64_t(gridDim.x) * blockDim.x) {
    uint32_t c = cnt[j];
    if (c) {
      tab[j].cnt = c;
      tab[j].beg = beg[j];
    }
  }
}

struct ValueCols {
  const uint32_t* src[MAPSQ_MAX_VARS];
  uint32_t* dst[MAPSQ_MAX_VARS];
  int n;
};

// Group the build side's value columns by key: row i goes to beg[slot] + rank.
__global__ void hash_scatter_kernel(ValueCols v, uint64_t nb, const uint32_t* __restrict__ slot_of,
                                    const uint32_t* __restrict__ rank_of, const uint32_t* __restrict__ beg) {
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nb; i += uint64_t(gridDim.x) * blockDim.x) {
    uint32_t pos = beg[slot_of[i]] + rank_of[i];
    for (int c = 0; c < v.n; ++c) v.dst[c][pos] = v.src[c][i];
  }
}

// Count pass fused with the prefix sum: each probe row looks its key up, records
// the start of its key group in pbeg and contributes its match count to a
// single-pass scan that writes the probe rows' output offsets.
struct ProbeCounts {
  KeyCols pk;
  const Slot* tab;
  uint32_t M;
  uint32_t* pbeg;
  __device__ __forceinline__ uint32_t operator()(uint64_t i) const {
    uint64_t key = load_key(pk, i);
    uint32_t c = 0, b = 0;
    if (key == kEmptyKey) {
      Slot sl = tab[M];
      c = sl.cnt;
      b = sl.beg;
    } else {
      uint32_t h = home_slot(key, M);
      for (uint32_t probe = 0; probe < M; ++probe) {
        Slot sl = tab[h];
        if (sl.key == key) {
          c = sl.cnt;
          b = sl.beg;
          break;
        }
        if (sl.key == kEmptyKey) break;
        h = h + 1 == M ? 0 : h + 1;
      }
    }
    pbeg[i] = b;
    return c;
  }
};

__global__ void __launch_bounds__(kLbThreads) probe_count_kernel(KeyCols pk, uint64_t np, const Slot* __restrict__ tab,
                                                                 uint32_t M, uint32_t* __restrict__ pbeg,
                                                                 uint64_t* __restrict__ off, uint64_t* scratch,
                                                                 uint32_t* err) {
  ProbeCounts pc{pk, tab, M, pbeg};
  lookback_scan_tile<uint64_t>(pc, np, off, scratch, err);
}

struct WriteParams {
  const uint64_t* off;   // exclusive prefix sums of the probe counts (np + 1)
  const uint32_t* pbeg;  // group start per probe row
  uint64_t np, nb, T;
  const uint32_t* src[MAPSQ_MAX_VARS];
  uint32_t* out[MAPSQ_MAX_VARS];
  uint32_t from_build;   // bit c: column c comes from the grouped build side
  int ncols;
  int cross;             // 1: cross product (no key), offsets implicit
};

__device__ __forceinline__ uint64_t upper_bound_u64(const uint64_t* a, uint64_t lo, uint64_t hi, uint64_t v) {
  while (lo < hi) {
    uint64_t mid = lo + (hi - lo) / 2;
    if (a[mid] <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Write pass: CTA tiles of kWriteTile output rows; each thread writes 4-row
// groups of every output column with one 16-byte streaming store.
__global__ void __launch_bounds__(kWriteThreads) join_write_kernel(WriteParams p) {
  __shared__ uint64_t s_off[kOffCache + 1];
  __shared__ uint64_t s_ilo, s_ihi;
  const uint64_t ntiles = (p.T + kWriteTile - 1) / kWriteTile;
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint64_t t0 = tile * kWriteTile;
    const uint64_t t1 = min(t0 + uint64_t(kWriteTile), p.T);
    bool cached = false;
    uint64_t ilo = 0, ihi = 0;
    if (!p.cross) {
      if (threadIdx.x == 0) {
        // probe rows whose output range meets [t0, t1)
        uint64_t a = upper_bound_u64(p.off, 0, p.np + 1, t0) - 1;
        uint64_t b = upper_bound_u64(p.off, a, p.np + 1, t1 - 1) - 1;
        s_ilo = a;
        s_ihi = b;
      }
      __syncthreads();
      ilo = s_ilo;
      ihi = s_ihi;
      cached = ihi - ilo + 2 <= kOffCache + 1;
      if (cached)
        for (uint64_t k = threadIdx.x; k < ihi - ilo + 2; k += blockDim.x) s_off[k] = p.off[ilo + k];
      __syncthreads();
    }
    for (int g = 0; g < kWriteGroups; ++g) {
      const uint64_t r0 = t0 + 4ull * (threadIdx.x + uint64_t(g) * kWriteThreads);
      if (r0 >= t1) break;
      const int nr = int(min(uint64_t(4), t1 - r0));
      uint64_t pi[4];
      uint64_t bi[4];
      if (p.cross) {
        uint64_t i = r0 / p.nb, j = r0 - i * p.nb;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          pi[k] = i;
          bi[k] = j;
          if (++j == p.nb) { j = 0; ++i; }
        }
      } else {
        uint64_t i;
        if (cached) {
          i = ilo + upper_bound_u64(s_off, 0, ihi - ilo + 2, r0) - 1;
        } else {
          i = upper_bound_u64(p.off, ilo, ihi + 2, r0) - 1;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint64_t r = r0 + k;
          if (k < nr) {
            // next probe row with a match: a binary search, since rows without
            // matches can sit between two output rows
            if (cached) {
              if (s_off[i + 1 - ilo] <= r) i = ilo + upper_bound_u64(s_off, i + 1 - ilo, ihi - ilo + 2, r) - 1;
              bi[k] = p.pbeg[i] + (r - s_off[i - ilo]);
            } else {
              if (p.off[i + 1] <= r) i = upper_bound_u64(p.off, i + 1, ihi + 2, r) - 1;
              bi[k] = p.pbeg[i] + (r - p.off[i]);
            }
          } else {
            bi[k] = 0;
          }
          pi[k] = i;
        }
      }
      for (int c = 0; c < p.ncols; ++c) {
        const uint32_t* src = p.src[c];
        const bool fb = (p.from_build >> c) & 1u;
        uint32_t v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = k < nr ? __ldg(src + (fb ? bi[k] : pi[k])) : 0u;
        uint32_t* dst = p.out[c] + r0;
        if (nr == 4) {
          __stcs(reinterpret_cast<uint4*>(dst), make_uint4(v[0], v[1], v[2], v[3]));
        } else {
          for (int k = 0; k < nr; ++k) __stcs(dst + k, v[k]);
        }
      }
    }
    __syncthreads();
  }
}

unsigned grid_for(uint64_t n, uint64_t cap = 152ull * 16) {
  return unsigned(std::max<uint64_t>(1, std::min<uint64_t>(ceil_div(n, 256), cap)));
}

struct Layout {
  int nkey = 0;
  int lkey[2] = {-1, -1}, rkey[2] = {-1, -1};
  int ncols = 0;
  int32_t var[MAPSQ_MAX_VARS];
  int side[MAPSQ_MAX_VARS];  // 0: left, 1: right
  int col[MAPSQ_MAX_VARS];
};

int make_layout(Ctx* ctx, const mapsq_table* L, const mapsq_table* R, Layout* lay) {
  int32_t shared[MAPSQ_MAX_VARS];
  int ns = 0;
  for (uint32_t a = 0; a < L->ncols; ++a)
    for (uint32_t b = 0; b < R->ncols; ++b)
      if (L->var[a] == R->var[b]) shared[ns++] = L->var[a];
  if (ns > 2)
    return set_error(ctx, MAPSQ_ERR_UNSUPPORTED, "join on %d shared variables (at most 2 are supported)", ns);
  std::sort(shared, shared + ns);
  lay->nkey = ns;
  auto find = [](const mapsq_table* t, int32_t v) {
    for (uint32_t c = 0; c < t->ncols; ++c)
      if (t->var[c] == v) return int(c);
    return -1;
  };
  int n = 0;
  for (int k = 0; k < ns; ++k) {
    lay->lkey[k] = find(L, shared[k]);
    lay->rkey[k] = find(R, shared[k]);
    lay->var[n] = shared[k];
    lay->side[n] = 0;
    lay->col[n] = lay->lkey[k];
    ++n;
  }
  auto is_shared = [&](int32_t v) { return std::find(shared, shared + ns, v) != shared + ns; };
  for (uint32_t c = 0; c < L->ncols; ++c)
    if (!is_shared(L->var[c])) { lay->var[n] = L->var[c]; lay->side[n] = 0; lay->col[n] = int(c); ++n; }
  for (uint32_t c = 0; c < R->ncols; ++c)
    if (!is_shared(R->var[c])) { lay->var[n] = R->var[c]; lay->side[n] = 1; lay->col[n] = int(c); ++n; }
  if (n > MAPSQ_MAX_VARS) return set_error(ctx, MAPSQ_ERR_INVALID, "join result would have %d columns", n);
  lay->ncols = n;
  return MAPSQ_OK;
}

int check_table(Ctx* ctx, const mapsq_table* t, const char* which) {
  if (t->ncols > MAPSQ_MAX_VARS) return set_error(ctx, MAPSQ_ERR_INVALID, "%s table: %u columns", which, t->ncols);
  if (t->ncols == 0 && t->nrows > 1)
    return set_error(ctx, MAPSQ_ERR_INVALID, "%s table: 0 columns and %llu rows", which, (unsigned long long)t->nrows);
  uint32_t seen = 0;
  for (uint32_t c = 0; c < t->ncols; ++c) {
    if (t->var[c] < 0 || t->var[c] >= MAPSQ_MAX_VARS)
      return set_error(ctx, MAPSQ_ERR_INVALID, "%s table: variable id %d", which, t->var[c]);
    if (seen & (1u << t->var[c])) return set_error(ctx, MAPSQ_ERR_INVALID, "%s table: variable %d twice", which, t->var[c]);
    seen |= 1u << t->var[c];
    if (t->nrows && (!t->col[c] || (reinterpret_cast<uintptr_t>(t->col[c]) & 15)))
      return set_error(ctx, MAPSQ_ERR_INVALID, "%s table: column %u is NULL or not 16-byte aligned", which, c);
  }
  if (t->ncols && t->nrows && !t->on_device)
    return set_error(ctx, MAPSQ_ERR_INVALID, "%s table: columns must be on the device", which);
  return MAPSQ_OK;
}

}  // namespace

int join_tables(Ctx* ctx, const mapsq_table* L, const mapsq_table* R, const mapsq_join_opts* opts,
                TableImpl** out) {
  (void)opts;
  MQ_TRY(check_table(ctx, L, "left"));
  MQ_TRY(check_table(ctx, R, "right"));
  Layout lay;
  MQ_TRY(make_layout(ctx, L, R, &lay));
  // build on the smaller side, probe with the larger
  const bool build_left = L->nrows < R->nrows;
  const mapsq_table* B = build_left ? L : R;
  const mapsq_table* P = build_left ? R : L;
  const int bside = build_left ? 0 : 1;
  const int* bkey = build_left ? lay.lkey : lay.rkey;
  const int* pkey = build_left ? lay.rkey : lay.lkey;
  const uint64_t nb = B->nrows, np = P->nrows;

  if (nb >= (uint64_t(1) << 31))
    return set_error(ctx, MAPSQ_ERR_UNSUPPORTED, "build side of %llu rows (at most 2^31-1)", (unsigned long long)nb);

  Scratch scratch(ctx);
  uint64_t T = 0;
  uint64_t* off = nullptr;
  uint32_t* pbeg = nullptr;
  uint32_t* grouped[MAPSQ_MAX_VARS] = {};
  const bool cross = lay.nkey == 0;

  if (nb == 0 || np == 0) {
    T = 0;
  } else if (cross) {
    if (np > UINT64_MAX / nb) return set_error(ctx, MAPSQ_ERR_BUDGET, "cross product overflows 64 bits");
    T = np * nb;
  } else {
    KeyCols bk{B->col[bkey[0]], lay.nkey == 2 ? B->col[bkey[1]] : nullptr};
    KeyCols pk{P->col[pkey[0]], lay.nkey == 2 ? P->col[pkey[1]] : nullptr};
    uint64_t M = std::max<uint64_t>(1024, 2 * nb);
    if (M >= 0xffffffffull) M = 0xfffffffeull;
    Slot* tab = nullptr;
    uint32_t *cnt = nullptr, *beg = nullptr, *slot_of = nullptr, *rank_of = nullptr;
    MQ_TRY(scratch.get(M + 1, &tab));
    MQ_TRY(scratch.get(M + 2, &cnt));
    MQ_TRY(scratch.get(M + 2, &beg));
    MQ_TRY(scratch.get(nb, &slot_of));
    MQ_TRY(scratch.get(nb, &rank_of));
    hash_init_kernel<<<grid_for(M + 1, 152ull * 32), 256, 0, ctx->stream>>>(tab, cnt, M + 1);
    ++ctx->launches;
    int rec = prof_begin(ctx, K_HASH_INSERT);
    hash_insert_kernel<<<grid_for(nb, 152ull * 32), 256, 0, ctx->stream>>>(bk, nb, tab, cnt, uint32_t(M), slot_of,
                                                                            rank_of, ctx->d_status);
    ++ctx->launches;
    prof_end(ctx, rec, 4.0 * lay.nkey * nb);
    MQ_CUDA(cudaGetLastError());
    MQ_TRY(prefix_sum_u32_u32(ctx, cnt, beg, M + 1));
    hash_finalize_kernel<<<grid_for(M + 1, 152ull * 32), 256, 0, ctx->stream>>>(tab, cnt, beg, M + 1);
    ++ctx->launches;
    // group the build side's value columns
    ValueCols vc{};
    for (int c = 0; c < lay.ncols; ++c) {
      if (lay.side[c] != bside) continue;
      MQ_TRY(scratch.get(nb, &grouped[c]));
      vc.src[vc.n] = B->col[lay.col[c]];
      vc.dst[vc.n] = grouped[c];
      ++vc.n;
    }
    if (vc.n) {
      rec = prof_begin(ctx, K_HASH_SCATTER);
      hash_scatter_kernel<<<grid_for(nb, 152ull * 32), 256, 0, ctx->stream>>>(vc, nb, slot_of, rank_of, beg);
      ++ctx->launches;
      prof_end(ctx, rec, 4.0 * vc.n * nb);
      MQ_CUDA(cudaGetLastError());
    }
    // count pass fused with the prefix sum of the counts
    uint64_t* lb = nullptr;
    MQ_TRY(scratch.get(np, &pbeg));
    MQ_TRY(scratch.get(np + 1, &off));
    MQ_TRY(scratch.get(lookback_scratch_words(np), &lb));
    MQ_CUDA(cudaMemsetAsync(lb, 0, lookback_scratch_words(np) * sizeof(uint64_t), ctx->stream));
    rec = prof_begin(ctx, K_PROBE_COUNT);
    probe_count_kernel<<<unsigned(ceil_div(np, kLbTile)), kLbThreads, 0, ctx->stream>>>(pk, np, tab, uint32_t(M), pbeg,
                                                                                        off, lb, ctx->d_status);
    ++ctx->launches;
    prof_end(ctx, rec, 4.0 * lay.nkey * np);
    MQ_CUDA(cudaGetLastError());
    // also reports a full hash table (impossible with M >= 2 nb) through the status word
    MQ_TRY(read_u64(ctx, off + np, &T, 1));
  }

  TableImpl* t = nullptr;
  if (lay.ncols == 0) {
    MQ_TRY(table_alloc(ctx, T, 0, lay.var, &t));
    *out = t;
    return MAPSQ_OK;
  }
  MQ_TRY(table_alloc(ctx, T, uint32_t(lay.ncols), lay.var, &t));
  if (T) {
    WriteParams wp{};
    wp.off = off;
    wp.pbeg = pbeg;
    wp.np = np;
    wp.nb = nb;
    wp.T = T;
    wp.ncols = lay.ncols;
    wp.cross = cross ? 1 : 0;
    double in_bytes = 0;
    for (int c = 0; c < lay.ncols; ++c) {
      const bool fb = lay.side[c] == bside && c >= lay.nkey;
      wp.out[c] = t->pub.col[c];
      if (fb) {
        wp.src[c] = cross ? B->col[lay.col[c]] : grouped[c];
        wp.from_build |= 1u << c;
        in_bytes += 4.0 * nb;
      } else {
        // key columns and the probe side's own columns come from the probe row
        int pc = c < lay.nkey ? pkey[c] : lay.col[c];
        wp.src[c] = P->col[pc];
        if (c >= lay.nkey) in_bytes += 4.0 * np;
      }
    }
    uint64_t ntiles = ceil_div(T, kWriteTile);
    unsigned grid = unsigned(std::min<uint64_t>(ntiles, 152ull * 8));
    int rec = prof_begin(ctx, cross ? K_CROSS_WRITE : K_JOIN_WRITE);
    join_write_kernel<<<grid, kWriteThreads, 0, ctx->stream>>>(wp);
    ++ctx->launches;
    prof_end(ctx, rec, 4.0 * double(T) * lay.ncols + in_bytes);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      table_release(ctx, t);
      return cuda_fail(ctx, e, "join_write_kernel", __FILE__, __LINE__);
    }
  }
  *out = t;
  return MAPSQ_OK;
}

// ---------------------------------------------------------------------------
// Join without any allocation, for callers that cannot call cudaMalloc.
//
// Some callers have no way to allocate device memory: code running inside a
// host that owns all device memory and hands out only fixed buffers, code on a
// path where an allocation could block or fail (a latency-critical loop, a
// process past its memory quota), or code whose allocator the library cannot
// reach.  mapsq_join_noalloc serves them: the caller passes the inputs and the
// output buffers, and every intermediate of the hash join lives in one
// file-scope device array of fixed size, kNoAllocScratchBytes, which each GPU
// that loads this library holds until the process exits.
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
constexpr uint64_t kNoAllocMaxBuild = uint64_t(1) << 18;  // rows of the smaller input
constexpr uint64_t kNoAllocMaxProbe = uint64_t(1) << 20;  // rows of the larger input
constexpr int kNoAllocMaxDevices = 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device.  The symbol's name
// is only a host-side stand-in: the address must come from cudaGetSymbolAddress,
// taken once per device with that device current.
int noalloc_scratch(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return MAPSQ_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MAPSQ_ERR_CUDA;
    g_noalloc_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_noalloc_addr[dev]);
  return MAPSQ_OK;
}

struct SlotCounts {
  const uint32_t* cnt;
  __device__ __forceinline__ uint32_t operator()(uint64_t i) const { return cnt[i]; }
};

// Prefix sum of the hash slots' group sizes (group starts), scratch passed in.
__global__ void __launch_bounds__(kLbThreads) noalloc_slot_prefix_kernel(const uint32_t* __restrict__ cnt, uint64_t n,
                                                                         uint32_t* __restrict__ beg, uint64_t* lb,
                                                                         uint32_t* err) {
  SlotCounts v{cnt};
  lookback_scan_tile<uint32_t>(v, n, beg, lb, err);
}

// Bump carving of the scratch array, 256-byte aligned regions.
struct Carve {
  unsigned char* base;
  size_t used = 0;
  template <class T>
  T* take(uint64_t count) {
    T* p = reinterpret_cast<T*>(base + used);
    used += (size_t(count) * sizeof(T) + 255) & ~size_t(255);
    return p;
  }
};

}  // namespace

}  // namespace mapsq

using namespace mapsq;

extern "C" int mapsq_join_noalloc(const mapsq_table* left, const mapsq_table* right, uint32_t* const* out_cols,
                                  uint64_t out_capacity_rows, mapsq_table* out, uint64_t* out_rows,
                                  void* cuda_stream) {
  if (!left || !right || !out || !out_rows) return MAPSQ_ERR_INVALID;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  MQ_TRY(check_table(nullptr, left, "left"));
  MQ_TRY(check_table(nullptr, right, "right"));
  Layout lay;
  MQ_TRY(make_layout(nullptr, left, right, &lay));
  const bool build_left = left->nrows < right->nrows;
  const mapsq_table* B = build_left ? left : right;
  const mapsq_table* P = build_left ? right : left;
  const int bside = build_left ? 0 : 1;
  const int* bkey = build_left ? lay.lkey : lay.rkey;
  const int* pkey = build_left ? lay.rkey : lay.lkey;
  const uint64_t nb = B->nrows, np = P->nrows;
  if (nb > kNoAllocMaxBuild || np > kNoAllocMaxProbe) return MAPSQ_ERR_INVALID;  // beyond the scratch array
  if (lay.ncols && !out_cols) return MAPSQ_ERR_INVALID;
  for (int c = 0; c < lay.ncols; ++c)
    if (!out_cols[c] || (reinterpret_cast<uintptr_t>(out_cols[c]) & 15)) return MAPSQ_ERR_INVALID;

  unsigned char* base = nullptr;
  MQ_TRY(noalloc_scratch(&base));
  Carve cv{base};
  uint32_t* status = cv.take<uint32_t>(64);
  const bool cross = lay.nkey == 0;
  uint64_t T = 0;
  uint64_t* off = nullptr;
  uint32_t* pbeg = nullptr;
  uint32_t* grouped[MAPSQ_MAX_VARS] = {};
  if (nb == 0 || np == 0) {
    T = 0;
  } else if (cross) {
    T = np * nb;  // both below 2^20: no overflow
  } else {
    KeyCols bk{B->col[bkey[0]], lay.nkey == 2 ? B->col[bkey[1]] : nullptr};
    KeyCols pk{P->col[pkey[0]], lay.nkey == 2 ? P->col[pkey[1]] : nullptr};
    const uint64_t M = std::max<uint64_t>(1024, 2 * nb);
    Slot* tab = cv.take<Slot>(M + 1);
    uint32_t* cnt = cv.take<uint32_t>(M + 2);
    uint32_t* beg = cv.take<uint32_t>(M + 2);
    uint32_t* slot_of = cv.take<uint32_t>(nb);
    uint32_t* rank_of = cv.take<uint32_t>(nb);
    ValueCols vc{};
    for (int c = 0; c < lay.ncols; ++c) {
      if (lay.side[c] != bside) continue;
      grouped[c] = cv.take<uint32_t>(nb);
      vc.src[vc.n] = B->col[lay.col[c]];
      vc.dst[vc.n] = grouped[c];
      ++vc.n;
    }
    pbeg = cv.take<uint32_t>(np);
    off = cv.take<uint64_t>(np + 1);
    uint64_t* lb_slots = cv.take<uint64_t>(lookback_scratch_words(M + 1));
    uint64_t* lb_probe = cv.take<uint64_t>(lookback_scratch_words(np));
    if (cv.used > kNoAllocScratchBytes) return MAPSQ_ERR_INVALID;
    // every call starts from cleared state: the array keeps the previous call's contents
    if (cudaMemsetAsync(status, 0, 64 * sizeof(uint32_t), stream) != cudaSuccess ||
        cudaMemsetAsync(lb_slots, 0, lookback_scratch_words(M + 1) * sizeof(uint64_t), stream) != cudaSuccess ||
        cudaMemsetAsync(lb_probe, 0, lookback_scratch_words(np) * sizeof(uint64_t), stream) != cudaSuccess)
      return MAPSQ_ERR_CUDA;
    hash_init_kernel<<<grid_for(M + 1, 152ull * 32), 256, 0, stream>>>(tab, cnt, M + 1);
    hash_insert_kernel<<<grid_for(nb, 152ull * 32), 256, 0, stream>>>(bk, nb, tab, cnt, uint32_t(M), slot_of, rank_of,
                                                                      status);
    noalloc_slot_prefix_kernel<<<unsigned(ceil_div(M + 1, kLbTile)), kLbThreads, 0, stream>>>(cnt, M + 1, beg,
                                                                                              lb_slots, status);
    hash_finalize_kernel<<<grid_for(M + 1, 152ull * 32), 256, 0, stream>>>(tab, cnt, beg, M + 1);
    if (vc.n) hash_scatter_kernel<<<grid_for(nb, 152ull * 32), 256, 0, stream>>>(vc, nb, slot_of, rank_of, beg);
    probe_count_kernel<<<unsigned(ceil_div(np, kLbTile)), kLbThreads, 0, stream>>>(pk, np, tab, uint32_t(M), pbeg, off,
                                                                                   lb_probe, status);
    if (cudaGetLastError() != cudaSuccess) return MAPSQ_ERR_CUDA;
    uint64_t host[2] = {0, 0};
    if (cudaMemcpyAsync(&host[0], off + np, sizeof(uint64_t), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaMemcpyAsync(&host[1], status, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
      return MAPSQ_ERR_CUDA;
    if (host[1] & 2u) return MAPSQ_ERR_TIMEOUT;
    if (host[1]) return MAPSQ_ERR_CUDA;
    T = host[0];
  }
  *out_rows = T;
  if (T > out_capacity_rows) return MAPSQ_ERR_BUDGET;
  memset(out, 0, sizeof(*out));
  out->nrows = T;
  out->ncols = uint32_t(lay.ncols);
  out->on_device = 1;
  for (int c = 0; c < MAPSQ_MAX_VARS; ++c) out->var[c] = c < lay.ncols ? lay.var[c] : -1;
  for (int c = 0; c < lay.ncols; ++c) out->col[c] = out_cols[c];
  if (T && lay.ncols) {
    WriteParams wp{};
    wp.off = off;
    wp.pbeg = pbeg;
    wp.np = np;
    wp.nb = nb;
    wp.T = T;
    wp.ncols = lay.ncols;
    wp.cross = cross ? 1 : 0;
    for (int c = 0; c < lay.ncols; ++c) {
      const bool fb = lay.side[c] == bside && c >= lay.nkey;
      wp.out[c] = out_cols[c];
      if (fb) {
        wp.src[c] = cross ? B->col[lay.col[c]] : grouped[c];
        wp.from_build |= 1u << c;
      } else {
        wp.src[c] = P->col[c < lay.nkey ? pkey[c] : lay.col[c]];
      }
    }
    unsigned grid = unsigned(std::min<uint64_t>(ceil_div(T, kWriteTile), 152ull * 8));
    join_write_kernel<<<grid, kWriteThreads, 0, stream>>>(wp);
    if (cudaGetLastError() != cudaSuccess) return MAPSQ_ERR_CUDA;
  }
  return MAPSQ_OK;
}
