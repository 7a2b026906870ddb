// MapSQ's MapReduce-based join (Algorithm 1) as a hash shuffle plus a
// count / prefix-sum / write reduce.
//
// Map: every row of both tables is mapped to its key, the shared variables
// packed into 64 bits (one variable: the id; two: smaller variable id in the
// high word), and keeps its other columns as its value (by row index).
// Shuffle: the smaller table (the build side) is partitioned by key through an
// open-addressing hash table sized from a HyperLogLog estimate of its distinct
// keys: one insert pass gives each row its key group and its rank inside the
// group (warp-aggregated atomics), a prefix sum over the groups' sizes gives
// each group's start, and a scatter pass writes the build side's value columns
// grouped by key, row-major.  Reduce: every row of the other table (the probe
// side) looks its key up and counts its matches (the size of its LEFT x RIGHT
// cross product) inside a single-pass look-back prefix sum that gives each probe
// row its output range; a partition pass finds, for every output tile, the
// probe rows that feed it; the write pass then emits every LEFT x RIGHT pair
// exactly once, partitioned by output position so that skewed keys are spread
// over all SMs, with 16-byte streaming stores into each output column.
//
// Output layout (Table 1(c)): shared variables in ascending id, then the left
// table's other columns, then the right table's.  No shared variable: the cross
// product, one key group holding every row.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "internal.cuh"
#include "lookback.cuh"

namespace mapsq {

namespace {

constexpr uint64_t kEmptyKey = ~0ull;
constexpr uint32_t kNoSlot = 0xffffffffu;
constexpr int kThreads = 256;                                        // threads per CTA of the probe and write passes
constexpr int kProbeTile = 2048;                                     // probe rows per count tile
constexpr int kProbeItems = kProbeTile / kThreads;                   // probe rows per thread
constexpr int kWriteRows = 16;                                       // output rows per thread per write tile
constexpr int kWriteTile = kThreads * kWriteRows;                    // output rows per write tile
constexpr int kStageRows = 1800;                                     // probe rows staged per write tile (48 KB of static shared memory in all)
constexpr int kMapWords = kWriteTile + kWriteTile / 32;              // row map, padded one word per 32
constexpr int kHllBits = 12;
constexpr int kHllRegs = 1 << kHllBits;
constexpr uint64_t kHllMinBuild = uint64_t(1) << 16;                 // smaller build sides size the table by rows

// Open-addressing table of the build side's distinct keys: ``keys`` holds M
// 64-bit keys in buckets of 4 (one 32-byte sector), probed bucket after bucket
// from the key's home bucket; ``group`` holds, per slot, the key group's size
// and its first row in the grouped build values.  The all-ones key marks an
// empty slot; the one real key equal to it uses the extra group entry M.
constexpr int kBucket = 4;

struct HashTable {
  uint64_t* keys;  // M entries, M a multiple of kBucket
  uint2* group;    // M + 1 entries: {count, begin}
  uint32_t M;
};

struct KeyCols {
  const uint32_t* c0;  // variable with the smaller id (high word when two)
  const uint32_t* c1;  // nullptr for a single-variable key
};

// Key columns are streamed once per pass: evict-first loads keep the hash table
// resident in L2.
__device__ __forceinline__ uint64_t load_key(const KeyCols& k, uint64_t i) {
  uint64_t a = __ldcs(k.c0 + i);
  return k.c1 ? (a << 32) | __ldcs(k.c1 + i) : a;
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

// Home bucket in [0, M / kBucket): Fibonacci (multiplicative) hashing of the
// key, folded to 32 bits, then multiply-shift range reduction.
__device__ __forceinline__ uint32_t home_bucket(uint64_t key, uint32_t M) {
  const uint32_t h = uint32_t((key * 0x9e3779b97f4a7c15ull) >> 32) ^ uint32_t(key >> 29);
  return uint32_t((uint64_t(h * 0x85ebca6bu) * uint64_t(M / kBucket)) >> 32);
}

// Slot of ``key`` in the table, or kNoSlot, starting from its home bucket
// whose keys are already loaded (k01 = slots 0-1, k23 = slots 2-3).
__device__ __forceinline__ uint32_t find_slot(const HashTable& t, uint64_t key, uint32_t b, ulonglong2 k01,
                                              ulonglong2 k23) {
  if (key == kEmptyKey) return t.M;
  const uint32_t nbk = t.M / kBucket;
  for (uint32_t it = 0; it < nbk; ++it) {
    // first slot of the bucket holding the key or empty decides
    const uint32_t hit = uint32_t(k01.x == key) | uint32_t(k01.y == key) << 1 | uint32_t(k23.x == key) << 2 |
                         uint32_t(k23.y == key) << 3;
    const uint32_t emp = uint32_t(k01.x == kEmptyKey) | uint32_t(k01.y == kEmptyKey) << 1 |
                         uint32_t(k23.x == kEmptyKey) << 2 | uint32_t(k23.y == kEmptyKey) << 3;
    if (hit | emp) {
      const int j = __ffs(hit | emp) - 1;
      return (hit >> j) & 1u ? b * kBucket + j : kNoSlot;
    }
    b = b + 1 == nbk ? 0 : b + 1;
    const ulonglong2* p = reinterpret_cast<const ulonglong2*>(t.keys + uint64_t(b) * kBucket);
    k01 = __ldg(p);
    k23 = __ldg(p + 1);
  }
  return kNoSlot;
}

__device__ __forceinline__ void load_bucket(const HashTable& t, uint64_t key, uint32_t* b, ulonglong2* k01,
                                            ulonglong2* k23) {
  *b = home_bucket(key, t.M);
  const ulonglong2* p = reinterpret_cast<const ulonglong2*>(t.keys + uint64_t(*b) * kBucket);
  *k01 = __ldg(p);
  *k23 = __ldg(p + 1);
}

// HyperLogLog sketch of the build keys (Flajolet, Fusy, Gandouet, Meunier,
// 2007): 2^12 registers hold the largest leading-zero count + 1 seen among the
// hashes routed to them.  The input is salted so the hash is independent of the
// table's.
__global__ void hll_kernel(KeyCols k, uint64_t n, uint32_t* __restrict__ regs) {
  __shared__ uint32_t s[kHllRegs];
  for (int j = threadIdx.x; j < kHllRegs; j += blockDim.x) s[j] = 0;
  __syncthreads();
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
    uint64_t h = mix_key(load_key(k, i) ^ 0x9e3779b97f4a7c15ull);
    uint32_t idx = uint32_t(h >> (64 - kHllBits));
    uint64_t w = (h << kHllBits) | (1ull << (kHllBits - 1));
    atomicMax(&s[idx], uint32_t(__clzll(w) + 1));
  }
  __syncthreads();
  for (int j = threadIdx.x; j < kHllRegs; j += blockDim.x)
    if (s[j]) atomicMax(&regs[j], s[j]);
}

double hll_estimate(const uint32_t* regs) {
  const double m = kHllRegs;
  double sum = 0.0;
  int zeros = 0;
  for (int j = 0; j < kHllRegs; ++j) {
    sum += std::ldexp(1.0, -int(regs[j]));
    zeros += regs[j] == 0;
  }
  double e = (0.7213 / (1.0 + 1.079 / m)) * m * m / sum;
  if (e <= 2.5 * m && zeros > 0) e = m * std::log(m / zeros);  // small-range correction (linear counting)
  return e;
}

// Insert every build row's key; slot_of[i] = its group's slot, rank_of[i] = its
// rank inside the group, counted in the group table.
__global__ void hash_insert_kernel(KeyCols bk, uint64_t nb, HashTable t, uint32_t* __restrict__ slot_of,
                                   uint32_t* __restrict__ rank_of, uint32_t* __restrict__ status) {
  const unsigned lane = threadIdx.x & 31;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  const uint32_t nbk = t.M / kBucket;
  for (uint64_t base = uint64_t(blockIdx.x) * blockDim.x; base < nb; base += stride) {
    uint64_t i = base + threadIdx.x;
    bool valid = i < nb;
    uint32_t s = kNoSlot;
    if (valid) {
      const uint64_t key = load_key(bk, i);
      if (key == kEmptyKey) {
        s = t.M;
      } else {
        uint32_t b = home_bucket(key, t.M);
        for (uint32_t it = 0; it < nbk && s == kNoSlot; ++it) {
          uint64_t* bkt = t.keys + uint64_t(b) * kBucket;
          const ulonglong2 k01 = __ldcg(reinterpret_cast<const ulonglong2*>(bkt));
          const ulonglong2 k23 = __ldcg(reinterpret_cast<const ulonglong2*>(bkt) + 1);
          const uint64_t k[4] = {k01.x, k01.y, k23.x, k23.y};
#pragma unroll
          for (int j = 0; j < kBucket; ++j) {
            if (s != kNoSlot) break;
            if (k[j] == key) {
              s = b * kBucket + j;
            } else if (k[j] == kEmptyKey) {
              const unsigned long long prev = atomicCAS(reinterpret_cast<unsigned long long*>(bkt + j),
                                                        (unsigned long long)kEmptyKey, (unsigned long long)key);
              if (prev == kEmptyKey || prev == key) s = b * kBucket + j;
            }
          }
          b = b + 1 == nbk ? 0 : b + 1;
        }
        if (s == kNoSlot) atomicOr(status, 1u);  // table full: the host rebuilds it larger
      }
    }
    // warp-aggregated group ranks: one atomic per distinct slot in the warp
    unsigned peers = __match_any_sync(0xffffffffu, s);
    int leader = __ffs(peers) - 1;
    uint32_t base_rank = 0;
    if (lane == unsigned(leader) && valid && s != kNoSlot) base_rank = atomicAdd(&t.group[s].x, __popc(peers));
    base_rank = __shfl_sync(0xffffffffu, base_rank, leader);
    if (valid) {
      slot_of[i] = s;
      rank_of[i] = base_rank + __popc(peers & ((1u << lane) - 1u));
    }
  }
}

// Group starts: exclusive prefix sum of the groups' sizes, written next to
// them (look-back scan over the M + 1 group entries).
struct GroupCounts {
  const uint2* group;
  __device__ __forceinline__ void fill(uint64_t base, uint64_t n, uint64_t* s) const {
#pragma unroll 4
    for (int k = 0; k < kLbItems; ++k) {
      const int local = k * kLbThreads + threadIdx.x;
      const uint64_t row = base + local;
      s[lb_pad(local)] = row < n ? uint64_t(group[row].x) : 0ull;
    }
  }
};

struct GroupStarts {
  uint2* group;
  __device__ __forceinline__ void store(uint64_t row, uint64_t v) const {
    if (group[row].x) group[row].y = uint32_t(v);
  }
  __device__ __forceinline__ void total(uint64_t) const {}
};

__global__ void __launch_bounds__(kLbThreads) slot_prefix_kernel(uint2* __restrict__ group, uint64_t n, uint64_t* lb,
                                                                 uint32_t* err) {
  GroupCounts c{group};
  GroupStarts s{group};
  lookback_scan_tile(c, n, s, lb, err);
}

struct BuildValues {
  const uint32_t* src[MAPSQ_MAX_VARS];
  int n;
};

constexpr int kScatterRows = 4;  // build rows per thread, loads issued together

// Group the build side's value columns by key, row-major: row i's values go to
// grouped[(begin of its group + rank) * n + j].
__global__ void hash_scatter_kernel(BuildValues v, uint64_t nb, const uint32_t* __restrict__ slot_of,
                                    const uint32_t* __restrict__ rank_of, const uint2* __restrict__ group,
                                    uint32_t* __restrict__ grouped) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x * kScatterRows;
  for (uint64_t base = uint64_t(blockIdx.x) * blockDim.x * kScatterRows + threadIdx.x; base < nb; base += stride) {
    uint32_t s[kScatterRows], rk[kScatterRows], beg[kScatterRows];
#pragma unroll
    for (int k = 0; k < kScatterRows; ++k) {
      const uint64_t i = base + uint64_t(k) * blockDim.x;
      s[k] = i < nb ? __ldcs(slot_of + i) : kNoSlot;
      rk[k] = i < nb ? __ldcs(rank_of + i) : 0u;
    }
#pragma unroll
    for (int k = 0; k < kScatterRows; ++k) beg[k] = s[k] != kNoSlot ? group[s[k]].y : 0u;
    for (int c = 0; c < v.n; ++c) {
      uint32_t x[kScatterRows];
#pragma unroll
      for (int k = 0; k < kScatterRows; ++k) {
        const uint64_t i = base + uint64_t(k) * blockDim.x;
        x[k] = s[k] != kNoSlot ? __ldcs(v.src[c] + i) : 0u;
      }
#pragma unroll
      for (int k = 0; k < kScatterRows; ++k)
        if (s[k] != kNoSlot) grouped[uint64_t(beg[k] + rk[k]) * uint32_t(v.n) + c] = x[k];
    }
  }
}

// Probes ``kProbeItems`` rows per thread, four lookups in flight at a time:
// out_cnt[k] / out_beg[k] = match count and group start of row
// base + k * kThreads + threadIdx.x (0 past np).
__device__ __forceinline__ void probe_rows(const KeyCols& pk, uint64_t np, const HashTable& t, uint64_t base,
                                           uint32_t* out_cnt, uint32_t* out_beg) {
  constexpr int H = 4;
#pragma unroll
  for (int h0 = 0; h0 < kProbeItems; h0 += H) {
    uint64_t key[H];
    uint32_t b[H], s[H];
    ulonglong2 k01[H], k23[H];
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const uint64_t row = base + uint64_t(h0 + k) * kThreads + threadIdx.x;
      key[k] = row < np ? load_key(pk, row) : kEmptyKey;
    }
#pragma unroll
    for (int k = 0; k < H; ++k)
      if (key[k] != kEmptyKey) load_bucket(t, key[k], &b[k], &k01[k], &k23[k]);
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const uint64_t row = base + uint64_t(h0 + k) * kThreads + threadIdx.x;
      s[k] = row < np ? find_slot(t, key[k], b[k], k01[k], k23[k]) : kNoSlot;
    }
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const uint2 g = s[k] != kNoSlot ? t.group[s[k]] : make_uint2(0u, 0u);
      out_cnt[h0 + k] = g.x;
      out_beg[h0 + k] = g.y;
    }
  }
}

// Count pass, tile-local: every probe row's match count and group start, the
// exclusive prefix sums of the counts inside its tile of kProbeTile rows, and
// the tile's total.  Output offsets are tile_base[row / kProbeTile] +
// local[row] once the tile totals are scanned; no CTA waits for another.
template <class OffT>
__global__ void __launch_bounds__(kThreads, 4) probe_count_kernel(KeyCols pk, uint64_t np, HashTable t,
                                                                  OffT* __restrict__ local,
                                                                  uint32_t* __restrict__ pbeg,
                                                                  uint64_t* __restrict__ tile_total,
                                                                  uint32_t* __restrict__ status) {
  __shared__ uint32_t s_cnt[kProbeTile + kProbeTile / 32];
  __shared__ uint64_t s_warp[kThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t base = uint64_t(blockIdx.x) * kProbeTile;
  auto pad = [](int i) { return i + (i >> 5); };
  {
    uint32_t cnt[kProbeItems], beg[kProbeItems];
    probe_rows(pk, np, t, base, cnt, beg);
#pragma unroll
    for (int k = 0; k < kProbeItems; ++k) {
      const int loc = k * kThreads + tid;
      if (base + loc < np) __stcs(pbeg + base + loc, beg[k]);
      s_cnt[pad(loc)] = cnt[k];
    }
  }
  __syncthreads();
  // block scan: each thread owns kProbeItems consecutive rows
  uint32_t v[kProbeItems];
  uint64_t sum = 0;
#pragma unroll
  for (int k = 0; k < kProbeItems; ++k) {
    v[k] = s_cnt[pad(tid * kProbeItems + k)];
    sum += v[k];
  }
  uint64_t inc = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint64_t x = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += x;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  uint64_t run = inc - sum, tile_sum = 0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) {
    const uint64_t x = s_warp[w];
    if (w < warp) run += x;
    tile_sum += x;
  }
  // local offsets, written back in row order through shared memory, half a tile at a time
  __syncthreads();
  uint64_t* s_off = reinterpret_cast<uint64_t*>(s_cnt);
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    if ((tid * kProbeItems) / (kProbeTile / 2) == half) {
#pragma unroll
      for (int k = 0; k < kProbeItems; ++k) {
        s_off[(tid * kProbeItems + k) % (kProbeTile / 2)] = run;
        run += v[k];
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kProbeItems / 2; ++k) {
      const int loc = half * (kProbeTile / 2) + k * kThreads + tid;
      const uint64_t row = base + loc;
      if (row < np) __stcs(local + row, OffT(s_off[loc - half * (kProbeTile / 2)]));
    }
    __syncthreads();
  }
  if (tid == 0) {
    tile_total[blockIdx.x] = tile_sum;
    if (sizeof(OffT) < 8 && tile_sum > 0xffffffffull) atomicOr(status, 4u);  // needs 64-bit local offsets
  }
}

// Exclusive scan of the count tiles' totals by one CTA: tile_base[t], and the
// join's row count in tile_base[ntiles].
__global__ void __launch_bounds__(1024) tile_scan_kernel(const uint64_t* __restrict__ tile_total, uint64_t ntiles,
                                                        uint64_t* __restrict__ tile_base) {
  __shared__ uint64_t s_warp[32];
  __shared__ uint64_t s_carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (uint64_t b = 0; b < ntiles; b += blockDim.x) {
    const uint64_t i = b + threadIdx.x;
    const uint64_t v = i < ntiles ? tile_total[i] : 0ull;
    uint64_t inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      uint64_t x = __shfl_up_sync(0xffffffffu, inc, d);
      if (lane >= d) inc += x;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    uint64_t before = s_carry, chunk = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) {
      if (w < warp) before += s_warp[w];
      chunk += s_warp[w];
    }
    if (i < ntiles) tile_base[i] = before + inc - v;
    __syncthreads();
    if (threadIdx.x == 0) s_carry += chunk;
    __syncthreads();
  }
  if (threadIdx.x == 0) tile_base[ntiles] = s_carry;
}

// Output offset of probe row i (i == np gives the row count).
template <class OffT>
struct Offsets {
  const OffT* local;
  const uint64_t* tile_base;
  uint64_t np, T;
  __device__ __forceinline__ uint64_t at(uint64_t i) const {
    return i < np ? tile_base[i / kProbeTile] + uint64_t(local[i]) : T;
  }
  // the probe row whose output range holds output row v, searched in [lo, hi)
  __device__ __forceinline__ uint64_t row_of(uint64_t v, uint64_t lo, uint64_t hi) const {
    while (lo < hi) {
      uint64_t mid = lo + (hi - lo) / 2;
      if (at(mid) <= v) lo = mid + 1; else hi = mid;
    }
    return lo - 1;
  }
};

template <class T>
__device__ __forceinline__ uint64_t upper_bound_t(const T* a, uint64_t lo, uint64_t hi, uint64_t v) {
  while (lo < hi) {
    uint64_t mid = lo + (hi - lo) / 2;
    if (uint64_t(a[mid]) <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Merge-path partition of the output: part[t] = the probe row whose output
// range holds output row min(t * kWriteTile, T - 1), for t in [0, ntiles]:
// first the count tile (search over tile bases), then the row inside it.
template <class OffT>
__global__ void write_partition_kernel(Offsets<OffT> off, uint64_t count_tiles, uint64_t ntiles,
                                       uint64_t* __restrict__ part) {
  for (uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t <= ntiles; t += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t v = min(t * uint64_t(kWriteTile), off.T - 1);
    const uint64_t ct = upper_bound_t(off.tile_base, 0, count_tiles + 1, v) - 1;
    const uint64_t lo = ct * kProbeTile, hi = min(lo + kProbeTile, off.np);
    part[t] = lo + upper_bound_t(off.local + lo, 0, hi - lo, v - off.tile_base[ct]) - 1;
  }
}

template <class OffT>
struct WriteParams {
  Offsets<OffT> off;
  const uint64_t* part;  // probe row of each output tile's first row (ntiles + 1)
  const uint32_t* pbeg;  // group start of each probe row
  uint64_t np, nb, T;
  const uint32_t* src[MAPSQ_MAX_VARS];
  uint32_t* out[MAPSQ_MAX_VARS];
  uint32_t from_build;   // bit c: column c comes from the build side
  uint32_t bstride;      // words between consecutive build rows in src (row-major grouped values)
  int ncols;
};

__device__ __forceinline__ uint32_t upper_bound_u32(const uint32_t* a, uint32_t lo, uint32_t hi, uint32_t v) {
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (a[mid] <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Write pass: CTA tiles of kWriteTile output rows.  (1) The probe rows feeding
// the tile get their output offsets (relative to the tile) and group starts
// staged in shared memory.  (2) Every thread maps 16 consecutive output rows to
// (probe row, build row) with one 32-bit search and a short walk, into shared
// memory.  (3) Every thread takes 16 rows striped over the block (a row per
// lane), reads their map entries once, and for every column issues the 16
// gathers before the 16 coalesced streaming stores.
template <class OffT>
__global__ void __launch_bounds__(kThreads, 4) join_write_kernel(WriteParams<OffT> p) {
  __shared__ uint32_t s_rel[kStageRows + 1];
  __shared__ uint32_t s_beg[kStageRows];
  __shared__ uint32_t s_pk[kMapWords];  // probe row of each output row (relative to the tile's first)
  __shared__ uint32_t s_bk[kMapWords];  // build row of each output row
  // row q lives at q + q / 32: conflict-free both for the 16 consecutive rows a
  // thread maps and for the rows striped over the block that it gathers
  auto mi = [](uint32_t q) { return q + (q >> 5); };
  __shared__ uint32_t s_skip;
  const uint64_t ntiles = (p.T + kWriteTile - 1) / kWriteTile;
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint64_t t0 = tile * kWriteTile;
    const uint32_t n = uint32_t(min(uint64_t(kWriteTile), p.T - t0));
    const uint64_t ilo = p.part[tile];
    const uint64_t nst = p.part[tile + 1] - ilo + 1;  // probe rows ilo .. part[tile + 1] can feed this tile
    const uint32_t q0 = threadIdx.x * kWriteRows;
    if (nst <= kStageRows) {
      const uint32_t ns = uint32_t(nst);
      for (uint32_t k = threadIdx.x; k <= ns; k += kThreads) {
        const uint64_t v = p.off.at(ilo + k);
        s_rel[k] = v <= t0 ? 0u : uint32_t(min(v - t0, uint64_t(kWriteTile)));
      }
      for (uint32_t k = threadIdx.x; k < ns; k += kThreads) s_beg[k] = p.pbeg[ilo + k];
      if (threadIdx.x == 0) s_skip = uint32_t(t0 - p.off.at(ilo));  // rows of probe row ilo before this tile
      __syncthreads();
      if (q0 < n) {
        uint32_t k = upper_bound_u32(s_rel, 0, ns + 1, q0) - 1;
        const uint32_t skip = s_skip;
#pragma unroll 4
        for (int j = 0; j < kWriteRows; ++j) {
          const uint32_t q = q0 + j;
          if (q >= n) break;
          if (s_rel[k + 1] <= q) {
            ++k;
            if (s_rel[k + 1] <= q) k = upper_bound_u32(s_rel, k + 1, ns + 1, q) - 1;
          }
          s_pk[mi(q)] = k;
          s_bk[mi(q)] = s_beg[k] + (q - s_rel[k]) + (k == 0 ? skip : 0u);
        }
      }
    } else if (q0 < n) {
      // more probe rows than the stage holds (rows with few matches): global search
      const uint64_t hi = ilo + nst + 1;
      uint64_t i = p.off.row_of(t0 + q0, ilo, hi);
      for (int j = 0; j < kWriteRows; ++j) {
        const uint32_t q = q0 + j;
        if (q >= n) break;
        const uint64_t r = t0 + q;
        if (p.off.at(i + 1) <= r) i = p.off.row_of(r, i + 1, hi);
        s_pk[mi(q)] = uint32_t(i - ilo);
        s_bk[mi(q)] = p.pbeg[i] + uint32_t(r - p.off.at(i));
      }
    }
    __syncthreads();
    uint32_t pk[kWriteRows], bk[kWriteRows];
#pragma unroll
    for (int j = 0; j < kWriteRows; ++j) {
      const uint32_t q = uint32_t(j) * kThreads + threadIdx.x;
      pk[j] = q < n ? s_pk[mi(q)] : 0u;
      bk[j] = q < n ? s_bk[mi(q)] : 0u;
    }
    for (int c = 0; c < p.ncols; ++c) {
      const bool fb = (p.from_build >> c) & 1u;
      const uint32_t* src = fb ? p.src[c] : p.src[c] + ilo;
      const uint32_t st = fb ? p.bstride : 1u;
      uint32_t* dst = p.out[c] + t0;
      uint32_t x[kWriteRows];
#pragma unroll
      for (int j = 0; j < kWriteRows; ++j) {
        const uint32_t q = uint32_t(j) * kThreads + threadIdx.x;
        x[j] = q < n ? __ldg(src + uint64_t(fb ? bk[j] : pk[j]) * st) : 0u;
      }
#pragma unroll
      for (int j = 0; j < kWriteRows; ++j) {
        const uint32_t q = uint32_t(j) * kThreads + threadIdx.x;
        if (q < n) __stcs(dst + q, x[j]);
      }
    }
    __syncthreads();
  }
}

struct CrossParams {
  uint64_t np, nb, T;
  const uint32_t* src[MAPSQ_MAX_VARS];
  uint32_t* out[MAPSQ_MAX_VARS];
  uint32_t from_build;   // bit c: column c comes from the smaller table
  int ncols;
};

// Cross product (no shared variable): output row r pairs probe row r / nb with
// build row r % nb.
__global__ void __launch_bounds__(kThreads) cross_write_kernel(CrossParams p) {
  const uint64_t ngroups = (p.T + 3) / 4;
  for (uint64_t g = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < ngroups; g += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t r0 = 4 * g;
    const int nr = int(min(uint64_t(4), p.T - r0));
    uint64_t pi[4], bi[4];
    uint64_t i = r0 / p.nb, j = r0 - i * p.nb;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      pi[k] = i;
      bi[k] = j;
      if (++j == p.nb) { j = 0; ++i; }
    }
    for (int c = 0; c < p.ncols; ++c) {
      const bool fb = (p.from_build >> c) & 1u;
      uint32_t v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = k < nr ? __ldg(p.src[c] + (fb ? bi[k] : pi[k])) : 0u;
      if (nr == 4) {
        __stcs(reinterpret_cast<uint4*>(p.out[c] + r0), make_uint4(v[0], v[1], v[2], v[3]));
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (k < nr) __stcs(p.out[c] + r0 + k, v[k]);
      }
    }
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

// One join, split in two halves so that the caller can allocate the output once
// its size is known: count() runs the map, shuffle and count passes and sets T;
// write() runs the partition and write passes.  Device memory comes from
// ``Mem`` (the context's allocator, or a fixed array carved by the caller), and
// ``host`` is a host buffer of at least kHllRegs / 2 + 2 words for read-backs.
template <class Mem>
struct HashJoin {
  Ctx* ctx;               // NULL without a context (no profiling, no launch count)
  cudaStream_t stream;
  uint32_t* status;       // device status word
  Mem* mem;
  uint64_t* host;
  Layout lay;
  const mapsq_table *L = nullptr, *R = nullptr, *B = nullptr, *P = nullptr;
  int bside = 1;
  const int *bkey = nullptr, *pkey = nullptr;
  uint64_t nb = 0, np = 0, T = 0;
  bool cross = false, off32 = true;
  KeyCols bk{}, pk{};
  HashTable table{};
  uint64_t M = 0;
  uint32_t* grouped = nullptr;
  uint32_t nbv = 0;       // build value columns (row-major stride of ``grouped``)
  uint64_t nt = 0;                 // count tiles
  void* local = nullptr;           // tile-local output offsets of the probe rows (u32 or u64)
  uint32_t* pbeg = nullptr;        // group start of each probe row
  uint64_t* tile_base = nullptr;   // nt + 1

  int fail(int code, const char* what) { return ctx ? set_error(ctx, code, "%s", what) : code; }
  int cuda(cudaError_t e, const char* what) {
    return e == cudaSuccess ? MAPSQ_OK : (ctx ? cuda_fail(ctx, e, what, __FILE__, __LINE__) : MAPSQ_ERR_CUDA);
  }
  void launched() {
    if (ctx) ++ctx->launches;
  }
  int rec(int kid) { return ctx ? prof_begin(ctx, kid) : -1; }
  void done(int r, double bytes) {
    if (ctx) prof_end(ctx, r, bytes);
  }

  int prepare(const mapsq_table* left, const mapsq_table* right) {
    L = left;
    R = right;
    MQ_TRY(check_table(ctx, L, "left"));
    MQ_TRY(check_table(ctx, R, "right"));
    MQ_TRY(make_layout(ctx, L, R, &lay));
    const bool build_left = L->nrows < R->nrows;  // build on the smaller side
    B = build_left ? L : R;
    P = build_left ? R : L;
    bside = build_left ? 0 : 1;
    bkey = build_left ? lay.lkey : lay.rkey;
    pkey = build_left ? lay.rkey : lay.lkey;
    nb = B->nrows;
    np = P->nrows;
    cross = lay.nkey == 0;
    if (nb >= (uint64_t(1) << 31)) return fail(MAPSQ_ERR_UNSUPPORTED, "build side of 2^31 rows or more");
    if (!cross) {
      bk = KeyCols{B->col[bkey[0]], lay.nkey == 2 ? B->col[bkey[1]] : nullptr};
      pk = KeyCols{P->col[pkey[0]], lay.nkey == 2 ? P->col[pkey[1]] : nullptr};
    }
    return MAPSQ_OK;
  }

  // Reads ``count`` 64-bit words and then the status word, synchronising the stream.
  int readback(const void* dptr, int count) {
    host[count] = 0;  // the status word fills only its low half
    MQ_TRY(cuda(cudaMemcpyAsync(host, dptr, sizeof(uint64_t) * count, cudaMemcpyDeviceToHost, stream), "readback"));
    MQ_TRY(cuda(cudaMemcpyAsync(host + count, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream), "status"));
    MQ_TRY(cuda(cudaStreamSynchronize(stream), "cudaStreamSynchronize"));
    return MAPSQ_OK;
  }

  int build_table() {
    uint32_t *slot_of = nullptr, *rank_of = nullptr;
    uint64_t* lb = nullptr;
    MQ_TRY(mem->get(M, &table.keys));
    MQ_TRY(mem->get(M + 1, &table.group));
    table.M = uint32_t(M);
    MQ_TRY(mem->get(nb, &slot_of));
    MQ_TRY(mem->get(nb, &rank_of));
    MQ_TRY(mem->get(lookback_scratch_words(M + 1), &lb));
    MQ_TRY(cuda(cudaMemsetAsync(lb, 0, lookback_scratch_words(M + 1) * sizeof(uint64_t), stream), "memset"));
    MQ_TRY(cuda(cudaMemsetAsync(table.keys, 0xff, M * sizeof(uint64_t), stream), "memset"));  // all empty
    MQ_TRY(cuda(cudaMemsetAsync(table.group, 0, (M + 1) * sizeof(uint2), stream), "memset"));
    int r = rec(K_HASH_INSERT);
    hash_insert_kernel<<<grid_for(nb, 152ull * 32), 256, 0, stream>>>(bk, nb, table, slot_of, rank_of, status);
    launched();
    done(r, 4.0 * lay.nkey * nb);
    r = rec(K_PREFIX_SUM);
    slot_prefix_kernel<<<unsigned(ceil_div(M + 1, kLbTile)), kLbThreads, 0, stream>>>(table.group, M + 1, lb, status);
    launched();
    done(r, 8.0 * (M + 1));
    BuildValues bv{};
    for (int c = lay.nkey; c < lay.ncols; ++c)
      if (lay.side[c] == bside) bv.src[bv.n++] = B->col[lay.col[c]];
    nbv = uint32_t(bv.n);
    if (nbv) {
      MQ_TRY(mem->get(nb * nbv, &grouped));
      r = rec(K_HASH_SCATTER);
      hash_scatter_kernel<<<grid_for(ceil_div(nb, kScatterRows), 152ull * 16), 256, 0, stream>>>(
          bv, nb, slot_of, rank_of, table.group, grouped);
      launched();
      done(r, 4.0 * nbv * nb);
    }
    return cuda(cudaGetLastError(), "hash build kernels");
  }

  template <class OffT>
  int probe() {
    OffT* loc = nullptr;
    uint64_t* tot = nullptr;
    nt = ceil_div(np, kProbeTile);
    MQ_TRY(mem->get(np, &loc));
    if (!pbeg) MQ_TRY(mem->get(np, &pbeg));
    MQ_TRY(mem->get(nt, &tot));
    MQ_TRY(mem->get(nt + 1, &tile_base));
    int r = rec(K_PROBE_COUNT);
    probe_count_kernel<OffT><<<unsigned(nt), kThreads, 0, stream>>>(pk, np, table, loc, pbeg, tot, status);
    launched();
    done(r, 4.0 * lay.nkey * np);
    tile_scan_kernel<<<1, 1024, 0, stream>>>(tot, nt, tile_base);
    launched();
    local = loc;
    return cuda(cudaGetLastError(), "probe_count_kernel");
  }

  int count() {
    T = 0;
    if (nb == 0 || np == 0) return MAPSQ_OK;
    if (cross) {
      if (np > UINT64_MAX / nb) return fail(MAPSQ_ERR_BUDGET, "cross product overflows 64 bits");
      T = np * nb;
      return MAPSQ_OK;
    }
    MQ_TRY(cuda(cudaMemsetAsync(status, 0, sizeof(uint32_t), stream), "memset"));
    M = std::max<uint64_t>(1024, 2 * nb);
    if (nb >= kHllMinBuild) {
      // size the table from the distinct keys: load factor about 0.6
      uint32_t* regs = nullptr;
      MQ_TRY(mem->get(kHllRegs, &regs));
      MQ_TRY(cuda(cudaMemsetAsync(regs, 0, kHllRegs * sizeof(uint32_t), stream), "memset"));
      int r = rec(K_HLL);
      hll_kernel<<<grid_for(nb / 4, 152ull * 8), 256, 0, stream>>>(bk, nb, regs);
      launched();
      done(r, 4.0 * lay.nkey * nb);
      MQ_TRY(readback(regs, kHllRegs / 2));
      double est = hll_estimate(reinterpret_cast<const uint32_t*>(host));
      M = std::min<uint64_t>(M, std::max<uint64_t>(1024, uint64_t(1.6 * est) + 1024));
    }
    if (M >= 0xfffffff0ull) M = 0xfffffff0ull;
    M = (M + kBucket - 1) / kBucket * kBucket;
    for (int attempt = 0;; ++attempt) {
      MQ_TRY(build_table());
      if (off32) {
        MQ_TRY(probe<uint32_t>());
      } else {
        MQ_TRY(probe<uint64_t>());
      }
      MQ_TRY(readback(tile_base + nt, 1));
      const uint32_t st = uint32_t(host[1]);
      if (st & 1u) {
        // a distinct-key estimate far too low: rebuild at two slots per build row
        if (attempt > 0 || M >= 2 * nb) return fail(MAPSQ_ERR_CUDA, "hash table full");
        M = (std::max<uint64_t>(1024, 2 * nb) + kBucket - 1) / kBucket * kBucket;
        MQ_TRY(cuda(cudaMemsetAsync(status, 0, sizeof(uint32_t), stream), "memset"));
        continue;
      }
      if (st & 2u) return fail(MAPSQ_ERR_TIMEOUT, "a prefix-sum look-back wait gave up");
      if (st & 4u) {
        // a count tile's total needs 64-bit local offsets: count again with them
        if (!off32) return fail(MAPSQ_ERR_CUDA, "device status word set");
        off32 = false;
        MQ_TRY(cuda(cudaMemsetAsync(status, 0, sizeof(uint32_t), stream), "memset"));
        MQ_TRY(probe<uint64_t>());
        MQ_TRY(readback(tile_base + nt, 1));
        if (host[1]) return fail(MAPSQ_ERR_CUDA, "device status word set");
      } else if (st) {
        return fail(MAPSQ_ERR_CUDA, "device status word set");
      }
      T = host[0];
      return MAPSQ_OK;
    }
  }

  template <class OffT>
  int write_hash(uint32_t* const* out_cols) {
    WriteParams<OffT> wp{};
    wp.off = Offsets<OffT>{static_cast<const OffT*>(local), tile_base, np, T};
    wp.pbeg = pbeg;
    wp.np = np;
    wp.nb = nb;
    wp.T = T;
    wp.ncols = lay.ncols;
    wp.bstride = nbv;
    const uint64_t ntiles = ceil_div(T, kWriteTile);
    uint64_t* part = nullptr;
    MQ_TRY(mem->get(ntiles + 1, &part));
    int r = rec(K_PARTITION);
    write_partition_kernel<OffT><<<grid_for(ntiles + 1, 152ull * 8), 256, 0, stream>>>(wp.off, nt, ntiles, part);
    launched();
    done(r, 8.0 * (ntiles + 1));
    wp.part = part;
    double in_bytes = 0;
    uint32_t j = 0;
    for (int c = 0; c < lay.ncols; ++c) {
      const bool fb = lay.side[c] == bside && c >= lay.nkey;
      wp.out[c] = out_cols[c];
      if (fb) {
        wp.src[c] = grouped + j++;
        wp.from_build |= 1u << c;
        in_bytes += 4.0 * nb;
      } else {
        // key columns and the probe side's own columns come from the probe row
        wp.src[c] = P->col[c < lay.nkey ? pkey[c] : lay.col[c]];
        if (c >= lay.nkey) in_bytes += 4.0 * np;
      }
    }
    unsigned grid = unsigned(std::min<uint64_t>(ntiles, 152ull * 8));
    r = rec(K_JOIN_WRITE);
    join_write_kernel<OffT><<<grid, kThreads, 0, stream>>>(wp);
    launched();
    done(r, 4.0 * double(T) * lay.ncols + in_bytes);
    return cuda(cudaGetLastError(), "join_write_kernel");
  }

  int write_cross(uint32_t* const* out_cols) {
    CrossParams cp{};
    cp.np = np;
    cp.nb = nb;
    cp.T = T;
    cp.ncols = lay.ncols;
    double in_bytes = 0;
    for (int c = 0; c < lay.ncols; ++c) {
      const bool fb = lay.side[c] == bside;
      cp.out[c] = out_cols[c];
      cp.src[c] = (fb ? B : P)->col[lay.col[c]];
      if (fb) cp.from_build |= 1u << c;
      in_bytes += 4.0 * (fb ? nb : np);
    }
    int r = rec(K_CROSS_WRITE);
    cross_write_kernel<<<grid_for(ceil_div(T, 4), 152ull * 8), kThreads, 0, stream>>>(cp);
    launched();
    done(r, 4.0 * double(T) * lay.ncols + in_bytes);
    return cuda(cudaGetLastError(), "cross_write_kernel");
  }

  int write(uint32_t* const* out_cols) {
    if (T == 0 || lay.ncols == 0) return MAPSQ_OK;
    if (cross) return write_cross(out_cols);
    return off32 ? write_hash<uint32_t>(out_cols) : write_hash<uint64_t>(out_cols);
  }
};

}  // namespace

int join_tables(Ctx* ctx, const mapsq_table* L, const mapsq_table* R, const mapsq_join_opts* opts,
                TableImpl** out) {
  (void)opts;
  Scratch scratch(ctx);
  HashJoin<Scratch> j{ctx, ctx->stream, ctx->d_status, &scratch, ctx->h_pinned + 64};
  MQ_TRY(j.prepare(L, R));
  MQ_TRY(j.count());
  TableImpl* t = nullptr;
  MQ_TRY(table_alloc(ctx, j.T, uint32_t(j.lay.ncols), j.lay.var, &t));
  int rc = j.write(t->pub.col);
  if (rc != MAPSQ_OK) {
    table_release(ctx, t);
    return rc;
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

// Bump carving of the scratch array into 256-byte aligned regions; refuses to
// run past its end.
struct Carve {
  unsigned char* base;
  size_t used = 0;
  template <class T>
  int get(size_t count, T** out) {
    size_t bytes = (std::max<size_t>(count * sizeof(T), 16) + 255) & ~size_t(255);
    if (used + bytes > kNoAllocScratchBytes) return MAPSQ_ERR_INVALID;
    *out = reinterpret_cast<T*>(base + used);
    used += bytes;
    return MAPSQ_OK;
  }
};

}  // namespace

}  // namespace mapsq

using namespace mapsq;

extern "C" int mapsq_join_noalloc(const mapsq_table* left, const mapsq_table* right, uint32_t* const* out_cols,
                                  uint64_t out_capacity_rows, mapsq_table* out, uint64_t* out_rows,
                                  void* cuda_stream) {
  if (!left || !right || !out || !out_rows) return MAPSQ_ERR_INVALID;
  unsigned char* base = nullptr;
  MQ_TRY(noalloc_scratch(&base));
  Carve carve{base};
  uint32_t* status = nullptr;
  MQ_TRY(carve.get(64, &status));
  uint64_t host[kHllRegs / 2 + 8];
  HashJoin<Carve> j{nullptr, static_cast<cudaStream_t>(cuda_stream), status, &carve, host};
  MQ_TRY(j.prepare(left, right));
  if (j.nb > kNoAllocMaxBuild || j.np > kNoAllocMaxProbe) return MAPSQ_ERR_INVALID;  // beyond the scratch array
  const int ncols = j.lay.ncols;
  if (ncols && !out_cols) return MAPSQ_ERR_INVALID;
  for (int c = 0; c < ncols; ++c)
    if (!out_cols[c] || (reinterpret_cast<uintptr_t>(out_cols[c]) & 15)) return MAPSQ_ERR_INVALID;
  MQ_TRY(j.count());
  *out_rows = j.T;
  if (j.T > out_capacity_rows) return MAPSQ_ERR_BUDGET;
  memset(out, 0, sizeof(*out));
  out->nrows = j.T;
  out->ncols = uint32_t(ncols);
  out->on_device = 1;
  for (int c = 0; c < MAPSQ_MAX_VARS; ++c) out->var[c] = c < ncols ? j.lay.var[c] : -1;
  for (int c = 0; c < ncols; ++c) out->col[c] = out_cols[c];
  return j.write(out_cols);
}
