// MapSQ's MapReduce-based join (Algorithm 1) as a hash shuffle plus a
// count / prefix-sum / write reduce, for a batch of independent joins at once.
//
// Map: every row of both tables is mapped to its key, the shared variables
// packed into 64 bits (one variable: the id; two: smaller variable id in the
// high word), and keeps its other columns as its value (by row index).
// Shuffle: the smaller table (the build side) is partitioned by key through an
// open-addressing hash table sized from a HyperLogLog estimate of its distinct
// keys: one insert pass gives each row its key group and its rank inside the
// group (warp-aggregated atomics), a prefix sum over the groups' sizes gives
// each group's start, and a scatter pass writes the build side's value columns
// grouped by key, row-major.  When one table is already sorted on its (single)
// key column (a run of the triple store) and large against the other, it is
// itself the grouping (Algorithm 1's Sort step done by the store's order): no
// table is built and each row of the other side searches it for its key's run
// (the sorted join; the crossover is measured by the autotuner).  Reduce:
// every row of the other table (the probe side) looks its key up and counts
// its matches (the size of its LEFT x RIGHT cross product); tile-local prefix
// sums and a scan of the tile totals give every probe row its output range; a
// partition step finds, for every output tile, the probe rows that feed it;
// the write pass then emits every LEFT x RIGHT pair exactly once, partitioned
// by output position so that skewed keys are spread over all SMs.
//
// Batching: every phase is one launch for all the joins of a batch.  Its work
// items (a join and a tile of that join) are numbered across the batch; a CTA
// finds its join by a binary search of the per-join item offsets.  The write
// phase is a persistent kernel that takes items from a device work counter.
// A batch synchronises once, to size its outputs (twice when large build sides
// need a distinct-key estimate).  A single join is a batch of one; a join whose
// probe side is one tile gets its offsets and partition from its count kernel.
//
// Output layout (Table 1(c)): shared variables in ascending id, then the left
// table's other columns, then the right table's.  No shared variable: the cross
// product, one key group holding every row.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>

#include "internal.cuh"
#include "lookback.cuh"
#include "search.cuh"

namespace mapsq {

namespace {

constexpr uint64_t kEmptyKey = ~0ull;
constexpr uint32_t kNoSlot = 0xffffffffu;
constexpr int kThreads = 256;                          // threads per CTA
constexpr int kRowTile = 2048;                         // rows per work item (build, slots, probe)
constexpr int kRowItems = kRowTile / kThreads;         // rows per thread
constexpr int kWriteRows = 16;                         // output rows per thread per write tile
constexpr int kWriteTile = kThreads * kWriteRows;      // output rows per write tile
constexpr int kStageRows = 1800;                       // probe rows per stage chunk
constexpr int kWriteBlocks = 4;                        // write CTAs per SM (register budget)
constexpr int kStageChunks = 4;                        // stage chunks at most per write tile
constexpr int kProbeIn = 1;                            // probe rows in flight per thread (registers go to occupancy)
constexpr int kProbeBlocks = 8;                        // probe CTAs per SM (32 registers)
constexpr int kDenseBlocks = 8;                        // dense write CTAs per SM (32 registers)
constexpr int kFusedBlocks = 8;                        // one-pass dense join CTAs per SM (32 registers)
constexpr int kFusedProbeIn = 1;                       // its lookups in flight per thread (registers go to occupancy)
constexpr uint64_t kFusedMinProbe = uint64_t(1) << 20;  // probe sides from which a dense join may take one pass
constexpr int kEarlyTiles = 64;                        // joins of up to this many write tiles are partitioned by the count scan
constexpr int kMapWords = kWriteTile + kWriteTile / 32;  // row map, padded one word per 32
constexpr int kWriteSmem = int(sizeof(uint32_t)) * (2 * kStageRows + 1 + 2 * kMapWords);  // write kernel's dynamic shared memory
constexpr int kHllBits = 12;
constexpr int kHllRegs = 1 << kHllBits;
constexpr uint64_t kHllMinBuild = uint64_t(1) << 16;   // smaller build sides size the table by rows
constexpr int kHllSpan = 4;                            // row tiles per sketch CTA (one flush per 8K rows)
constexpr int kBucket = 4;
constexpr int kPhases = 11;
constexpr int kDenseUnroll = 4;                        // probe rows of a thread unrolled in the dense write
constexpr uint32_t kDenseMax = 16;                     // default crossover of the mean matches per probe row
constexpr uint64_t kDenseCap = 64;                     // no dense write when a probe row has more matches
constexpr int kSamples = 2048;                         // sorted key column samples per count CTA (8 KB)
constexpr int kSortedThreads = 1024;                   // threads of the sorted count (two rows each)
constexpr int kSortedItems = kRowTile / kSortedThreads;
constexpr int kSearchWays = 4;                         // sorted count: pivots per search round + 1
constexpr uint64_t kKaryMaxItems = 152;                // sorted count launches of up to this many CTAs search K-ary
constexpr uint32_t kSortedRatio = 4;                   // default: sorted side at least this many times the other's rows

constexpr int kRegionBits = 8;
constexpr int kRegions = 1 << kRegionBits;             // build partitions, by the top bits of the home bucket
constexpr int kHllWords = kHllRegs + kRegions;         // a sketch's registers, then its region histogram
constexpr int kPartThreads = 256;                      // threads of the partition kernel (one per region)
constexpr int kPartItems = 16;
constexpr int kPartRows = kPartThreads * kPartItems;   // build rows per partition CTA

enum Phase { PH_HLL = 0, PH_INSERT, PH_SLOTS, PH_SCATTER, PH_COUNT, PH_PART, PH_WRITE, PH_CROSS, PH_SORTED, PH_DENSE,
             PH_REGION };

// Open-addressing table of the build side's distinct keys: ``keys`` holds M
// 64-bit keys in buckets of 4 (one 32-byte sector, read by one 32-byte load),
// probed bucket after bucket
// from the key's home bucket; ``group`` holds, per slot, the key group's size
// and its first row inside its tile of kRowTile slots (the tile's start is
// slot_base[slot / kRowTile]).  The all-ones key marks an empty slot; the one
// real key equal to it uses the extra group entry M.
struct HashTable {
  uint64_t* keys;  // M entries, M a multiple of kBucket
  uint2* group;    // M + 1 entries: {count, begin within the slot tile}
  uint64_t* slot_base;
  uint32_t M;
};

struct KeyCols {
  const uint32_t* c0;  // variable with the smaller id (high word when two)
  const uint32_t* c1;  // nullptr for a single-variable key
};

// Everything one join of a batch needs on the device.
struct JoinDesc {
  KeyCols bk, pk;                 // build and probe keys
  uint64_t nb, np;                // build and probe rows
  HashTable t;
  uint32_t* hll;                  // kHllRegs registers and kRegions region counts, or NULL
  uint32_t* slot_of;              // nb: slot of each build row
  uint32_t* rank_of;              // nb: rank inside its group
  uint64_t* slot_total;           // per slot tile: sum of its group sizes
  const uint32_t* bsrc[MAPSQ_MAX_VARS];  // build value columns
  int nbv;                        // their number (row-major stride of ``grouped``)
  uint32_t* grouped;              // nb * nbv: build values grouped by key
  uint32_t* local;                // np: output offset of each probe row inside its tile
  uint32_t* nzmask;               // np / 32 + 1: bit i % 32 of word i / 32 set when probe row i has a match
  uint32_t* pbeg;                 // np: group start of each probe row
  uint64_t* tile_total;           // per probe tile: its output rows
  uint64_t* tile_base;            // per probe tile + 1: output offset of the tile (last = T)
  uint64_t T;                     // output rows (set after the count phase)
  uint64_t* part;                 // output tiles + 1: first probe row of each output tile
  const uint32_t* src[MAPSQ_MAX_VARS];  // output column c: probe column, or build values + j
  uint32_t* out[MAPSQ_MAX_VARS];
  uint32_t from_build;            // bit c: column c comes from the build side
  int ncols;
  int cross;                      // no shared variable: output row r pairs probe row r / nb with build row r % nb
  int hash;                       // shared variables and both sides non-empty: the hash path runs
  int sorted;                     // the build side is sorted on its (one) key column: groups are its runs
  uint32_t bstride;               // words between a build row's values: nbv (grouped) or 1 (columns)
  uint32_t* check;                // status word of the checked build's bounds checks
};

// Item offsets of one phase: join j owns items [first[j], first[j + 1]).
__device__ __forceinline__ uint32_t item_join(const uint64_t* first, uint32_t k, uint64_t item) {
  uint32_t lo = 0, hi = k;  // last j with first[j] <= item
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (first[mid] <= item) lo = mid; else hi = mid;
  }
  return lo;
}

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
__device__ __forceinline__ uint32_t home_x(uint64_t key) {
  const uint32_t h = uint32_t((key * 0x9e3779b97f4a7c15ull) >> 32) ^ uint32_t(key >> 29);
  return h * 0x85ebca6bu;
}

__device__ __forceinline__ uint32_t home_bucket(uint64_t key, uint32_t M) {
  return uint32_t((uint64_t(home_x(key)) * uint64_t(M / kBucket)) >> 32);
}

// Region of a key: the top bits of the same 32-bit value, so that the regions
// cut the table into consecutive runs of home buckets whatever its size.
__device__ __forceinline__ uint32_t home_region(uint64_t key) { return home_x(key) >> (32 - kRegionBits); }

__device__ __forceinline__ uint64_t* bucket_keys(const HashTable& t, uint32_t b) {
  return t.keys + uint64_t(b) * kBucket;
}

// Group entry {count, begin within the slot tile} of slot s.
__device__ __forceinline__ uint2* group_of(const HashTable& t, uint32_t s) { return t.group + s; }

// Four 64-bit words in one 32-byte load (``p`` 32-byte aligned): the keys of a
// bucket, or four grouped build rows of two values.  Read-only through the
// non-coherent path (probes, writes), or at L2 (inserts, whose buckets other
// threads fill meanwhile).
__device__ __forceinline__ void ld_u64x4_nc(const uint64_t* p, ulonglong2* k01, ulonglong2* k23) {
  asm volatile("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];"
               : "=l"(k01->x), "=l"(k01->y), "=l"(k23->x), "=l"(k23->y)
               : "l"(p));
}

__device__ __forceinline__ void ld_u64x4_cg(const uint64_t* p, ulonglong2* k01, ulonglong2* k23) {
  asm volatile("ld.global.cg.v4.u64 {%0, %1, %2, %3}, [%4];"
               : "=l"(k01->x), "=l"(k01->y), "=l"(k23->x), "=l"(k23->y)
               : "l"(p)
               : "memory");
}

__device__ __forceinline__ void load_bucket(const HashTable& t, uint64_t key, uint32_t* b, ulonglong2* k01,
                                            ulonglong2* k23) {
  *b = home_bucket(key, t.M);
  ld_u64x4_nc(bucket_keys(t, *b), k01, k23);
}

// Slot of ``key`` in the table, or kNoSlot, starting from its home bucket
// whose keys are already loaded (k01 = slots 0-1, k23 = slots 2-3).
__device__ __forceinline__ uint32_t find_slot(const HashTable& t, uint64_t key, uint32_t b, ulonglong2 k01,
                                              ulonglong2 k23) {
  if (key == kEmptyKey) return t.M;
  const uint32_t nbk = t.M / kBucket;
  for (uint32_t it = 0; it < nbk; ++it) {
    // the first slot of the bucket holding the key or empty decides
    const uint32_t hit = uint32_t(k01.x == key) | uint32_t(k01.y == key) << 1 | uint32_t(k23.x == key) << 2 |
                         uint32_t(k23.y == key) << 3;
    const uint32_t emp = uint32_t(k01.x == kEmptyKey) | uint32_t(k01.y == kEmptyKey) << 1 |
                         uint32_t(k23.x == kEmptyKey) << 2 | uint32_t(k23.y == kEmptyKey) << 3;
    if (hit | emp) {
      const int j = __ffs(hit | emp) - 1;
      return (hit >> j) & 1u ? b * kBucket + j : kNoSlot;
    }
    b = b + 1 == nbk ? 0 : b + 1;
    ld_u64x4_nc(bucket_keys(t, b), &k01, &k23);
  }
  return kNoSlot;
}

// Group start (over the whole build side) of slot s.
__device__ __forceinline__ uint32_t group_begin(const HashTable& t, uint32_t s, uint32_t local_begin) {
  return local_begin + uint32_t(t.slot_base[s / kRowTile]);
}

// Block-wide exclusive scan of one value per thread (row order = thread order
// of ``vals`` laid out kRowItems consecutive rows per thread); returns the
// thread's exclusive prefix and the block total.
template <int NT>
__device__ __forceinline__ uint64_t block_scan_n(uint64_t sum, uint64_t* s_warp, uint64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t inc = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t x = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += x;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  uint64_t before = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) {
    const uint64_t x = s_warp[w];
    if (w < warp) before += x;
    tot += x;
  }
  *total = tot;
  return before + inc - sum;
}

__device__ __forceinline__ uint64_t block_scan(uint64_t sum, uint64_t* s_warp, uint64_t* total) {
  return block_scan_n<kThreads>(sum, s_warp, total);
}

// ------------------------------------------------------------------ phases

// HyperLogLog sketch of the build keys (Flajolet, Fusy, Gandouet, Meunier,
// 2007): 2^12 registers hold the largest leading-zero count + 1 seen among the
// hashes routed to them.  The input is salted so the hash is independent of the
// table's.  The same pass counts the rows of each region (home_region), the
// histogram of the build side's partition.
__global__ void __launch_bounds__(kThreads) hll_kernel(const JoinDesc* __restrict__ jd, const uint64_t* first,
                                                      uint32_t k) {
  constexpr int kHists = kThreads / 32;
  __shared__ uint32_t s[kHllRegs];
  __shared__ uint32_t s_hists[kHists * kRegions];  // one region histogram per warp
  uint32_t* s_hist = s_hists + (threadIdx.x >> 5) * kRegions;
  const uint32_t j = item_join(first, k, blockIdx.x);
  const JoinDesc& d = jd[j];
  const uint64_t base = (blockIdx.x - first[j]) * uint64_t(kRowTile) * kHllSpan;
  for (int r = threadIdx.x; r < kHllRegs; r += kThreads) s[r] = 0;
  for (int r = threadIdx.x; r < kHists * kRegions; r += kThreads) s_hists[r] = 0;
  __syncthreads();
#pragma unroll 8
  for (int it = 0; it < kRowItems * kHllSpan; ++it) {
    const uint64_t i = base + uint64_t(it) * kThreads + threadIdx.x;
    if (i < d.nb) {
      const uint64_t key = load_key(d.bk, i);
      const uint64_t h = mix_key(key ^ 0x9e3779b97f4a7c15ull);
      const uint64_t w = (h << kHllBits) | (1ull << (kHllBits - 1));
      const uint32_t reg = uint32_t(h >> (64 - kHllBits)), rho = uint32_t(__clzll(w) + 1);
      if (s[reg] < rho) atomicMax(&s[reg], rho);  // most rows cannot raise their register
      atomicAdd(&s_hist[home_region(key)], 1u);
    }
  }
  __syncthreads();
  // a register already at least this high in global memory stays so (the
  // maximum only grows): most flushes of a large build side end at the read
  for (int r = threadIdx.x; r < kHllRegs; r += kThreads)
    if (s[r] && s[r] > __ldcg(d.hll + r)) atomicMax(&d.hll[r], s[r]);
  for (int r = threadIdx.x; r < kRegions; r += kThreads) {
    uint32_t c = 0;
#pragma unroll
    for (int h = 0; h < kHists; ++h) c += s_hists[h * kRegions + r];
    if (c) atomicAdd(&d.hll[kHllRegs + r], c);
  }
}

// Partition of a large build side by region, so that the insert and the
// scatter that follow touch the hash table and the grouped values one run of
// consecutive slots at a time (L2-resident) instead of all over.  A CTA takes
// kPartRows rows: it ranks every row inside its region (shared-memory
// atomics: the order inside a region is free), reserves each region's run in
// the output with one atomic per region, notes for every position of its
// region-ordered buffer the distance to that position's output row, then
// moves the rows column by column through shared memory so that each region's
// rows leave as one contiguous run.
struct PartDesc {
  const uint32_t* src[MAPSQ_MAX_VARS];  // build columns: the key column(s), then the value columns
  uint32_t* dst[MAPSQ_MAX_VARS];        // their partitioned copies
  uint32_t* cursor;                     // kRegions: next free row of each region (starts at its offset)
  uint64_t n;
  int nkey, ncols;
  uint32_t* check;                      // status word of the checked build's bounds checks
};

static_assert(kPartThreads == kRegions, "one thread per region in the region scan");

__global__ void __launch_bounds__(kPartThreads, 4) partition_kernel(const PartDesc* __restrict__ pd,
                                                                    const uint64_t* first, uint32_t k) {
  __shared__ __align__(16) uint32_t s_buf[kPartRows];  // one column's values, in region order
  __shared__ uint32_t s_delta[kPartRows];              // global row of position q, minus q (mod 2^32)
  __shared__ uint32_t s_cnt[kRegions], s_dr[kRegions], s_wsum[kRegions / 32];
  const uint32_t j = item_join(first, k, blockIdx.x);
  const PartDesc& p = pd[j];
  const uint64_t base = (blockIdx.x - first[j]) * uint64_t(kPartRows);
  const uint32_t n = uint32_t(min(uint64_t(kPartRows), p.n - base));
  const unsigned lane = threadIdx.x & 31, tid = threadIdx.x;
  s_cnt[tid] = 0;
  __syncthreads();
  uint32_t pos[kPartItems];  // region << 24 | rank inside the region, then the position in s_buf
#pragma unroll
  for (int h = 0; h < kPartItems; h += 8) {
    uint32_t hi[8], lo[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint32_t i = uint32_t(h + q) * kPartThreads + tid;
      hi[q] = i < n ? __ldg(p.src[0] + base + i) : 0u;
      lo[q] = i < n && p.nkey == 2 ? __ldg(p.src[1] + base + i) : 0u;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint32_t i = uint32_t(h + q) * kPartThreads + tid;
      if (i < n) {
        const uint64_t key = p.nkey == 2 ? (uint64_t(hi[q]) << 32) | lo[q] : uint64_t(hi[q]);
        const uint32_t reg = home_region(key);
        pos[h + q] = (reg << 24) | atomicAdd(&s_cnt[reg], 1u);
      } else {
        pos[h + q] = ~0u;
      }
    }
  }
  __syncthreads();
  // exclusive scan of the region counts; each region's run in the output
  const uint32_t v = s_cnt[tid];
  uint32_t inc = v;
#pragma unroll
  for (int dd = 1; dd < 32; dd <<= 1) {
    const uint32_t x = __shfl_up_sync(0xffffffffu, inc, dd);
    if (lane >= unsigned(dd)) inc += x;
  }
  if (lane == 31) s_wsum[tid >> 5] = inc;
  __syncthreads();
  uint32_t before = 0;
  for (uint32_t w = 0; w < (tid >> 5); ++w) before += s_wsum[w];
  const uint32_t lo_r = before + inc - v;
  const uint32_t gb = v ? atomicAdd(p.cursor + tid, v) : 0u;
  __syncthreads();  // every thread has read s_cnt
  s_cnt[tid] = lo_r;
  s_dr[tid] = gb - lo_r;
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kPartItems; ++it)
    if (pos[it] != ~0u) {
      const uint32_t reg = pos[it] >> 24;
      pos[it] = s_cnt[reg] + (pos[it] & 0xffffffu);
      s_delta[pos[it]] = s_dr[reg];
    }
  for (int c = 0; c < p.ncols; ++c) {
#pragma unroll
    for (int it = 0; it < kPartItems; ++it)
      if (pos[it] != ~0u) s_buf[pos[it]] = __ldcs(p.src[c] + base + uint32_t(it) * kPartThreads + tid);
    __syncthreads();
    for (uint32_t q = tid; q < n; q += kPartThreads) {
      const uint64_t at = uint32_t(s_delta[q] + q);
      if (MQ_IN_BOUNDS(at < p.n, p.check)) __stcg(p.dst[c] + at, s_buf[q]);
    }
    __syncthreads();
  }
}

double hll_estimate(const uint32_t* regs) {
  // 2^-r for every register value (at most 64 - kHllBits + 1): a table, since
  // a batch sizes up to hundreds of tables one after another on the host
  static const std::array<double, 65> inv = [] {
    std::array<double, 65> a{};
    for (int r = 0; r <= 64; ++r) a[r] = std::ldexp(1.0, -r);
    return a;
  }();
  const double m = kHllRegs;
  double sum = 0.0;
  int zeros = 0;
  for (int j = 0; j < kHllRegs; ++j) {
    const uint32_t r = regs[j] < 64u ? regs[j] : 64u;
    sum += inv[r];
    zeros += r == 0;
  }
  double e = (0.7213 / (1.0 + 1.079 / m)) * m * m / sum;
  if (e <= 2.5 * m && zeros > 0) e = m * std::log(m / zeros);  // small-range correction (linear counting)
  return e;
}

// Insert every build row's key; slot_of[i] = its group's slot, rank_of[i] = its
// rank inside the group, counted in the group table (warp-aggregated).
__global__ void __launch_bounds__(kThreads, 8) hash_insert_kernel(const JoinDesc* __restrict__ jd, const uint64_t* first,
                                                              uint32_t k, uint32_t* __restrict__ status) {
  const uint32_t j = item_join(first, k, blockIdx.x);
  const JoinDesc& d = jd[j];
  const HashTable t = d.t;
  const uint64_t base = (blockIdx.x - first[j]) * kRowTile;
  const unsigned lane = threadIdx.x & 31;
  const uint32_t nbk = t.M / kBucket;
  for (int it = 0; it < kRowItems; ++it) {
    const uint64_t i = base + uint64_t(it) * kThreads + threadIdx.x;
    const bool valid = i < d.nb;
    uint32_t s = kNoSlot;
    if (valid) {
      const uint64_t key = load_key(d.bk, i);
      if (key == kEmptyKey) {
        s = t.M;
      } else {
        uint32_t b = home_bucket(key, t.M);
        for (uint32_t n = 0; n < nbk && s == kNoSlot; ++n) {
          uint64_t* bkt = bucket_keys(t, b);
          ulonglong2 k01, k23;
          ld_u64x4_cg(bkt, &k01, &k23);
          const uint64_t kk[4] = {k01.x, k01.y, k23.x, k23.y};
#pragma unroll
          for (int q = 0; q < kBucket; ++q) {
            if (s != kNoSlot) break;
            if (kk[q] == key) {
              s = b * kBucket + q;
            } else if (kk[q] == kEmptyKey) {
              const unsigned long long prev = atomicCAS(reinterpret_cast<unsigned long long*>(bkt + q),
                                                        (unsigned long long)kEmptyKey, (unsigned long long)key);
              if (prev == kEmptyKey || prev == key) s = b * kBucket + q;
            }
          }
          b = b + 1 == nbk ? 0 : b + 1;
        }
        if (s == kNoSlot) atomicOr(status, 1u);  // table full: the host rebuilds it larger
      }
    }
    const unsigned peers = __match_any_sync(0xffffffffu, s);
    const int leader = __ffs(peers) - 1;
    uint32_t base_rank = 0;
    if (lane == unsigned(leader) && valid && s != kNoSlot) base_rank = atomicAdd(&group_of(t, s)->x, __popc(peers));
    base_rank = __shfl_sync(0xffffffffu, base_rank, leader);
    if (valid) {
      d.slot_of[i] = s;
      d.rank_of[i] = base_rank + __popc(peers & ((1u << lane) - 1u));
    }
  }
}

// The join's largest match count of a probe row (atomic maximum over warps).
template <int N>
__device__ __forceinline__ void join_max_count(const uint32_t (&v)[N], uint64_t* out) {
  uint32_t m = 0;
#pragma unroll
  for (int q = 0; q < N; ++q) m = max(m, v[q]);
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0 && m) atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)m);
}

// A join whose probe side is one tile needs no tile scan: the count kernel
// writes its tile offsets, its row count and, for a small output, its write
// partition, searching the tile's offsets where the block still holds them in
// shared memory (s_off[pad(i)] = output offset of probe row i).  The whole
// block calls this after the offsets are in place.
__device__ __forceinline__ void single_tile_finish(const JoinDesc& d, uint64_t tile_sum, uint64_t* total,
                                                   const uint32_t* s_off) {
  if (threadIdx.x == 0) {
    d.tile_base[0] = 0;
    d.tile_base[1] = tile_sum;
    *total = tile_sum;
  }
  const uint64_t ntw = (tile_sum + kWriteTile - 1) / kWriteTile;
  if (tile_sum && ntw <= kEarlyTiles && threadIdx.x <= ntw) {
    const uint32_t v = uint32_t(min(uint64_t(threadIdx.x) * kWriteTile, tile_sum - 1));
    uint32_t lo = 0, hi = uint32_t(d.np);  // last probe row whose offset is <= v
    while (lo < hi) {
      const uint32_t m = (lo + hi) >> 1;
      if (s_off[m + (m >> 5)] <= v) lo = m + 1; else hi = m;
    }
    d.part[threadIdx.x] = lo - 1;
  }
}

// Slot tiles: the group starts inside each tile of kRowTile slots (written into
// group[].y) and the tile's total; per join, the largest group (groups[j])
// and the number of groups (groups[k + j]).
__global__ void __launch_bounds__(kThreads) slot_scan_kernel(const JoinDesc* __restrict__ jd, const uint64_t* first,
                                                            uint32_t k, uint64_t* __restrict__ groups) {
  __shared__ uint64_t s_warp[kThreads / 32];
  const uint32_t j = item_join(first, k, blockIdx.x);
  const JoinDesc& d = jd[j];
  const uint64_t base = (blockIdx.x - first[j]) * kRowTile, n = uint64_t(d.t.M) + 1;
  uint32_t c[kRowItems];
  uint64_t sum = 0;
  uint32_t most = 0, nonzero = 0;
#pragma unroll
  for (int it = 0; it < kRowItems; ++it) {
    const uint64_t s = base + uint64_t(threadIdx.x) * kRowItems + it;
    c[it] = s < n ? group_of(d.t, uint32_t(s))->x : 0u;
    sum += c[it];
    most = max(most, c[it]);
    nonzero += c[it] != 0;
  }
  __shared__ uint32_t s_most[kThreads / 32], s_nonzero[kThreads / 32];
  most = __reduce_max_sync(0xffffffffu, most);
  nonzero = __reduce_add_sync(0xffffffffu, nonzero);
  if ((threadIdx.x & 31) == 0) {
    s_most[threadIdx.x >> 5] = most;
    s_nonzero[threadIdx.x >> 5] = nonzero;
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // one atomic of each kind per CTA
    for (int w = 1; w < kThreads / 32; ++w) {
      most = max(most, s_most[w]);
      nonzero += s_nonzero[w];
    }
    if (most) atomicMax(reinterpret_cast<unsigned long long*>(groups + j), (unsigned long long)most);
    if (nonzero) atomicAdd(reinterpret_cast<unsigned long long*>(groups + k + j), (unsigned long long)nonzero);
  }
  uint64_t total;
  uint64_t run = block_scan(sum, s_warp, &total);
#pragma unroll
  for (int it = 0; it < kRowItems; ++it) {
    const uint64_t s = base + uint64_t(threadIdx.x) * kRowItems + it;
    if (s < n && c[it]) group_of(d.t, uint32_t(s))->y = uint32_t(run);
    run += c[it];
  }
  if (threadIdx.x == 0) d.slot_total[blockIdx.x - first[j]] = total;
}

template <class T>
__device__ __forceinline__ uint64_t upper_bound_t(const T* a, uint64_t lo, uint64_t hi, uint64_t v) {
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo) / 2;
    if (uint64_t(a[mid]) <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// The probe row whose output range holds output row v (given the tile offsets).
__device__ __forceinline__ uint64_t part_row(const JoinDesc& d, uint64_t v) {
  const uint64_t nt = (d.np + kRowTile - 1) / kRowTile;
  const uint64_t ct = upper_bound_t(d.tile_base, 0, nt + 1, v) - 1;
  const uint64_t lo = ct * kRowTile, hi = min(lo + kRowTile, d.np);
  return lo + upper_bound_t(d.local + lo, 0, hi - lo, v - d.tile_base[ct]) - 1;
}

// Exclusive scans of per-tile totals, one CTA per join: slot tile starts
// (which = 0) or probe tile output offsets with the join's row count last
// (which = 1).
__global__ void __launch_bounds__(1024) tiles_scan_kernel(JoinDesc* __restrict__ jd, uint32_t k, int which,
                                                         uint64_t* __restrict__ totals_out) {
  __shared__ uint64_t s_warp[32];
  __shared__ uint64_t s_carry;
  JoinDesc& d = jd[blockIdx.x];
  if (!d.hash && !(d.sorted && which == 1)) {
    if (which == 1 && threadIdx.x == 0) totals_out[blockIdx.x] = d.cross ? d.np * d.nb : 0;
    return;
  }
  const uint64_t n = which == 0 ? (uint64_t(d.t.M) + kRowTile) / kRowTile : (d.np + kRowTile - 1) / kRowTile;
  const uint64_t* tot = which == 0 ? d.slot_total : d.tile_total;
  uint64_t* out = which == 0 ? d.t.slot_base : d.tile_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (uint64_t b = 0; b < n; b += blockDim.x) {
    const uint64_t i = b + threadIdx.x;
    const uint64_t v = i < n ? tot[i] : 0ull;
    uint64_t inc = v;
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
      const uint64_t x = __shfl_up_sync(0xffffffffu, inc, dd);
      if (lane >= dd) inc += x;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    uint64_t before = s_carry, chunk = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) {
      if (w < warp) before += s_warp[w];
      chunk += s_warp[w];
    }
    if (i < n) out[i] = before + inc - v;
    __syncthreads();
    if (threadIdx.x == 0) s_carry += chunk;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[n] = s_carry;
    if (which == 1) totals_out[blockIdx.x] = s_carry;
  }
  // a join of few write tiles gets its output partition here (saves a launch)
  if (which == 1) {
    __syncthreads();  // the tile offsets above are visible to the whole block
    const uint64_t T = s_carry, ntiles = (T + kWriteTile - 1) / kWriteTile;
    if (T && ntiles <= kEarlyTiles && threadIdx.x <= ntiles)
      d.part[threadIdx.x] = part_row(d, min(uint64_t(threadIdx.x) * kWriteTile, T - 1));
  }
}

// Group the build side's value columns by key, row-major: row i's values go to
// grouped[(start of its group + rank) * nbv + c].
__global__ void __launch_bounds__(kThreads) hash_scatter_kernel(const JoinDesc* __restrict__ jd, const uint64_t* first,
                                                               uint32_t k) {
  const uint32_t j = item_join(first, k, blockIdx.x);
  const JoinDesc& d = jd[j];
  const uint64_t base = (blockIdx.x - first[j]) * kRowTile;
  const int nbv = d.nbv;
#pragma unroll 1
  for (int h0 = 0; h0 < kRowItems; h0 += 4) {
    uint32_t s[4], pos[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint64_t i = base + uint64_t(h0 + q) * kThreads + threadIdx.x;
      s[q] = i < d.nb ? __ldcs(d.slot_of + i) : kNoSlot;
      pos[q] = i < d.nb ? __ldcs(d.rank_of + i) : 0u;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (s[q] != kNoSlot) pos[q] += group_begin(d.t, s[q], group_of(d.t, s[q])->y);
    if (nbv == 2) {
      // a row's two values in one 8-byte store
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint64_t i = base + uint64_t(h0 + q) * kThreads + threadIdx.x;
        if (s[q] != kNoSlot && MQ_IN_BOUNDS(pos[q] < d.nb, d.check))
          reinterpret_cast<uint2*>(d.grouped)[pos[q]] = make_uint2(__ldcs(d.bsrc[0] + i), __ldcs(d.bsrc[1] + i));
      }
      continue;
    }
    for (int c = 0; c < nbv; ++c) {
      uint32_t x[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint64_t i = base + uint64_t(h0 + q) * kThreads + threadIdx.x;
        x[q] = s[q] != kNoSlot ? __ldcs(d.bsrc[c] + i) : 0u;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (s[q] != kNoSlot && MQ_IN_BOUNDS(pos[q] < d.nb, d.check)) d.grouped[uint64_t(pos[q]) * uint32_t(nbv) + c] = x[q];
    }
  }
}


// Count phase, tile-local: every probe row's match count and group start
// (kProbeIn lookups in flight per thread), the match bitmask, the exclusive
// prefix sums of the counts inside its tile of kRowTile rows (``local``), and
// the tile's total.  No CTA waits for another; the tile totals are scanned
// afterwards (or, for a one-tile probe side, finished here).
__global__ void __launch_bounds__(kThreads, kProbeBlocks) probe_count_kernel(const JoinDesc* __restrict__ jd,
                                                                  const uint64_t* first, uint32_t k,
                                                                  uint32_t* __restrict__ status,
                                                                  uint64_t* __restrict__ totals) {
  __shared__ uint32_t s_cnt[kRowTile + kRowTile / 32];
  __shared__ uint64_t s_warp[kThreads / 32];
  const uint32_t jj = item_join(first, k, blockIdx.x);
  const JoinDesc& d = jd[jj];
  const HashTable t = d.t;
  const uint64_t tile = blockIdx.x - first[jj];
  const uint64_t base = tile * kRowTile;
  const uint64_t np = d.np;
  auto pad = [](int i) { return i + (i >> 5); };
  // keys loaded as they are needed: the registers go to more CTAs per SM
#pragma unroll
  for (int h0 = 0; h0 < kRowItems; h0 += kProbeIn) {
    uint64_t key[kProbeIn];
    uint32_t b[kProbeIn], s[kProbeIn];
    ulonglong2 k01[kProbeIn], k23[kProbeIn];
#pragma unroll
    for (int q = 0; q < kProbeIn; ++q) {
      const uint64_t row = base + uint64_t(h0 + q) * kThreads + threadIdx.x;
      key[q] = row < np ? load_key(d.pk, row) : kEmptyKey;
    }
#pragma unroll
    for (int q = 0; q < kProbeIn; ++q)
      if (key[q] != kEmptyKey) load_bucket(t, key[q], &b[q], &k01[q], &k23[q]);
#pragma unroll
    for (int q = 0; q < kProbeIn; ++q) {
      const uint64_t row = base + uint64_t(h0 + q) * kThreads + threadIdx.x;
      s[q] = row < np ? find_slot(t, key[q], b[q], k01[q], k23[q]) : kNoSlot;
    }
#pragma unroll
    for (int q = 0; q < kProbeIn; ++q) {
      const int loc = (h0 + q) * kThreads + threadIdx.x;
      const uint64_t row = base + loc;
      const uint2 g = s[q] != kNoSlot ? *group_of(t, s[q]) : make_uint2(0u, 0u);
      const uint32_t gbeg = g.x ? group_begin(t, s[q], g.y) : 0u;
      if (row < np) __stcs(d.pbeg + row, gbeg);
      s_cnt[pad(loc)] = MQ_IN_BOUNDS(uint64_t(gbeg) + g.x <= d.nb, d.check) ? g.x : 0u;
      const unsigned nz = __ballot_sync(0xffffffffu, g.x != 0);  // the warp's 32 consecutive rows
      if ((threadIdx.x & 31) == 0 && row < np) d.nzmask[row >> 5] = nz;
    }
  }
  __syncthreads();
  uint32_t v[kRowItems];
  uint64_t sum = 0;
#pragma unroll
  for (int q = 0; q < kRowItems; ++q) {
    v[q] = s_cnt[pad(threadIdx.x * kRowItems + q)];
    sum += v[q];
  }
  uint64_t tile_sum;
  uint64_t run = block_scan(sum, s_warp, &tile_sum);
  join_max_count(v, totals + k + jj);
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kRowItems; ++q) {
    s_cnt[pad(threadIdx.x * kRowItems + q)] = uint32_t(run);
    run += v[q];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kRowItems; ++q) {
    const int loc = q * kThreads + threadIdx.x;
    if (base + loc < np) __stcs(d.local + base + loc, s_cnt[pad(loc)]);
  }
  if (threadIdx.x == 0) {
    d.tile_total[tile] = tile_sum;
    if (tile_sum > 0xffffffffull) atomicOr(status, 4u);  // tile-local offsets would not fit in 32 bits
  }
  if (np <= kRowTile) single_tile_finish(d, tile_sum, totals + jj, s_cnt);
}

// Count phase of a sorted join.  The build side's key column is sorted, so a
// key's group is the run of equal keys.  Every probe row's search is narrowed
// first in kSamples evenly spaced samples of the column held in shared
// memory, then between two neighbouring samples in global memory.  A launch of
// few CTAs (bound by the latency of its dependent loads) searches the run's
// start (first position >= key) and end (first position > key) together in
// K-ary rounds, all searches of a thread in lockstep; a larger launch (bound by
// its loads' throughput) bisects for the start and gallops for the end, fewer
// loads per row.  Counts, group starts and tile-local offsets are then written
// as in the hash count phase.
__device__ __forceinline__ uint64_t sample_pos(uint32_t i, uint64_t n) { return uint64_t(i) * n / kSamples; }


__global__ void __launch_bounds__(kSortedThreads) sorted_count_kernel(const JoinDesc* __restrict__ jd,
                                                                     const uint64_t* first, uint32_t k,
                                                                     uint32_t* __restrict__ status,
                                                                     uint64_t* __restrict__ totals, bool kary) {
  __shared__ uint32_t s_key[kSamples];
  __shared__ uint32_t s_cnt[kRowTile + kRowTile / 32];
  __shared__ uint64_t s_warp[kSortedThreads / 32];
  const uint32_t jj = item_join(first, k, blockIdx.x);
  const JoinDesc& d = jd[jj];
  const uint64_t tile = blockIdx.x - first[jj];
  const uint64_t base = tile * kRowTile, np = d.np, nx = d.nb;
  const uint32_t* __restrict__ x = d.bk.c0;
  auto pad = [](int i) { return i + (i >> 5); };
  for (int i = threadIdx.x; i < kSamples; i += kSortedThreads) s_key[i] = __ldg(x + sample_pos(uint32_t(i), nx));
  __syncthreads();
  // first position >= t, bracketed by the samples: [lo, lo + len]
  auto bracket = [&](uint32_t t, uint64_t* lo, uint64_t* len) {
    uint32_t a = 0, b = kSamples;  // first sample >= t
    while (a < b) {
      const uint32_t m = (a + b) >> 1;
      if (s_key[m] < t) a = m + 1; else b = m;
    }
    *lo = a ? sample_pos(a - 1, nx) + 1 : 0;
    *len = (a < kSamples ? sample_pos(a, nx) : nx) - *lo;
  };
  uint32_t key[kSortedItems];
  uint64_t first_pos[kSortedItems], run_len[kSortedItems];
#pragma unroll
  for (int it = 0; it < kSortedItems; ++it) {
    const uint64_t row = base + it * kSortedThreads + threadIdx.x;
    key[it] = row < np ? __ldcs(d.pk.c0 + row) : 0u;
  }
  if (kary) {
    // latency-bound launch: a key's run is [first position >= key, first
    // position > key), both ends of every row's run searched together, K-ary
    // rounds in lockstep (searches 2i and 2i + 1 are row i's ends)
    constexpr int kS = 2 * kSortedItems;
    const uint32_t* arr[kS];
    uint32_t tgt[kS];
    uint64_t lo[kS], len[kS];
#pragma unroll
    for (int it = 0; it < kSortedItems; ++it) {
      const uint64_t row = base + it * kSortedThreads + threadIdx.x;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int q = 2 * it + e;
        arr[q] = x;
        tgt[q] = key[it] + uint32_t(e);
        if (row >= np || (e && key[it] == 0xffffffffu)) {  // nothing to search; no value exceeds the largest key
          lo[q] = nx;
          len[q] = 0;
        } else {
          bracket(tgt[q], &lo[q], &len[q]);
        }
      }
    }
    lower_bounds_kary<kS, kSearchWays>(arr, tgt, lo, len);
#pragma unroll
    for (int it = 0; it < kSortedItems; ++it) {
      first_pos[it] = lo[2 * it];
      run_len[it] = lo[2 * it + 1] - lo[2 * it];
    }
  } else {
    // throughput-bound launch (fewer loads per row): the run's start by
    // bisection in lockstep, its end by galloping from the start (short runs
    // stay in one cache line), then bisecting
    const uint32_t* arr[kSortedItems];
    uint64_t len[kSortedItems];
#pragma unroll
    for (int it = 0; it < kSortedItems; ++it) {
      arr[it] = x;
      const uint64_t row = base + it * kSortedThreads + threadIdx.x;
      if (row < np) {
        bracket(key[it], &first_pos[it], &len[it]);
      } else {
        first_pos[it] = nx;
        len[it] = 0;
      }
    }
    lower_bounds_kary<kSortedItems, 2>(arr, key, first_pos, len);
#pragma unroll
    for (int it = 0; it < kSortedItems; ++it) {
      const uint32_t v = key[it];
      run_len[it] = 0;
      if (first_pos[it] < nx && __ldg(x + first_pos[it]) == v) {
        uint64_t a = first_pos[it], step = 1;
        while (a + step < nx && __ldg(x + a + step) == v) {
          a += step;
          step <<= 1;
        }
        uint64_t b = min(a + step, nx);  // x[a] == v; x[b] > v or b == nx
        while (b - a > 1) {
          const uint64_t m = a + (b - a) / 2;
          if (__ldg(x + m) == v) a = m; else b = m;
        }
        run_len[it] = a + 1 - first_pos[it];
      }
    }
  }
#pragma unroll
  for (int it = 0; it < kSortedItems; ++it) {
    const int loc = it * kSortedThreads + threadIdx.x;
    const uint64_t row = base + loc;
    uint32_t cnt = 0;
    if (row < np) {
      cnt = uint32_t(run_len[it]);
      __stcs(d.pbeg + row, cnt ? uint32_t(first_pos[it]) : 0u);
    }
    s_cnt[pad(loc)] = cnt;
    const unsigned nz = __ballot_sync(0xffffffffu, cnt != 0);  // the warp's 32 consecutive rows
    if ((threadIdx.x & 31) == 0 && row < np) d.nzmask[row >> 5] = nz;
  }
  __syncthreads();
  uint32_t v[kSortedItems];
  uint64_t sum = 0;
#pragma unroll
  for (int q = 0; q < kSortedItems; ++q) {
    v[q] = s_cnt[pad(threadIdx.x * kSortedItems + q)];
    sum += v[q];
  }
  uint64_t tile_sum;
  uint64_t run = block_scan_n<kSortedThreads>(sum, s_warp, &tile_sum);
  join_max_count(v, totals + k + jj);
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kSortedItems; ++q) {
    s_cnt[pad(threadIdx.x * kSortedItems + q)] = uint32_t(run);
    run += v[q];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kSortedItems; ++q) {
    const int loc = q * kSortedThreads + threadIdx.x;
    if (base + loc < np) __stcs(d.local + base + loc, s_cnt[pad(loc)]);
  }
  if (threadIdx.x == 0) {
    d.tile_total[tile] = tile_sum;
    if (tile_sum > 0xffffffffull) atomicOr(status, 4u);  // tile-local offsets would not fit in 32 bits
  }
  if (np <= kRowTile) single_tile_finish(d, tile_sum, totals + jj, s_cnt);
}

// Output offset of probe row i of a join (i == np gives its row count).
__device__ __forceinline__ uint64_t off_at(const JoinDesc& d, uint64_t i) {
  return i < d.np ? d.tile_base[i / kRowTile] + d.local[i] : d.T;
}


// The first probe row after row i that has a match (one exists: the caller
// holds an output row beyond row i's range), from the match bitmask.
__device__ __forceinline__ uint64_t next_nonzero(const JoinDesc& d, uint64_t i) {
  uint64_t w = (i + 1) >> 5;
  const uint64_t last = d.np >> 5;
  uint32_t m = d.nzmask[w] & (~0u << ((i + 1) & 31));
  while (!m && w < last) m = d.nzmask[++w];
  return (w << 5) + __ffs(m) - 1;
}

// The probe row whose output range holds output row v, searched in [lo, hi).
__device__ __forceinline__ uint64_t row_of(const JoinDesc& d, uint64_t v, uint64_t lo, uint64_t hi) {
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo) / 2;
    if (off_at(d, mid) <= v) lo = mid + 1; else hi = mid;
  }
  return lo - 1;
}


// Merge-path partition of each join's output: part[t] = the probe row whose
// output range holds output row min(t * kWriteTile, T - 1), t in [0, ntiles]:
// first its probe tile (search over tile offsets), then the row inside it.
__global__ void __launch_bounds__(kThreads) write_partition_kernel(const JoinDesc* __restrict__ jd,
                                                                  const uint64_t* first, uint32_t k) {
  const uint32_t j = item_join(first, k, blockIdx.x);
  const JoinDesc& d = jd[j];
  const uint64_t t = (blockIdx.x - first[j]) * kThreads + threadIdx.x;
  const uint64_t ntiles = (d.T + kWriteTile - 1) / kWriteTile;
  if (t > ntiles) return;
  d.part[t] = part_row(d, min(t * uint64_t(kWriteTile), d.T - 1));
}

__device__ __forceinline__ uint32_t upper_bound_u32(const uint32_t* a, uint32_t lo, uint32_t hi, uint32_t v) {
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a[mid] <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Output rows of a write tile are handled in runs of kVec consecutive rows: run
// g * kThreads + tid of the tile belongs to thread tid, so a warp's stores of
// one column cover 512 contiguous bytes (16-byte stores; columns and tiles are
// 16-byte aligned).  Entry g * kVec + w of a thread's arrays is row
// (g * kThreads + tid) * kVec + w.
constexpr int kVec = 4;
constexpr int kRuns = kWriteRows / kVec;

__device__ __forceinline__ uint32_t run_row(int i) {
  return (uint32_t(i / kVec) * kThreads + threadIdx.x) * kVec + uint32_t(i % kVec);
}

template <bool kFull>
__device__ __forceinline__ void store_runs(uint32_t* __restrict__ dst, const uint32_t (&x)[kWriteRows], uint32_t n) {
#pragma unroll
  for (int g = 0; g < kRuns; ++g) {
    const uint32_t q = (uint32_t(g) * kThreads + threadIdx.x) * kVec;
    if (kFull || q + kVec <= n) {
      __stcs(reinterpret_cast<uint4*>(dst + q), make_uint4(x[g * kVec], x[g * kVec + 1], x[g * kVec + 2], x[g * kVec + 3]));
    } else {
#pragma unroll
      for (int w = 0; w < kVec; ++w)
        if (q + w < n) __stcs(dst + q + w, x[g * kVec + w]);
    }
  }
}

// One output column of a tile: row run_row(i) takes src[idx[i] * stride]; the
// gathers are issued before the stores.
template <bool kFull>
__device__ __forceinline__ void write_column(const uint32_t* __restrict__ src, const uint32_t (&idx)[kWriteRows],
                                             uint32_t stride, uint32_t* __restrict__ dst, uint32_t n) {
  uint32_t x[kWriteRows];
#pragma unroll
  for (int i = 0; i < kWriteRows; ++i)
    x[i] = kFull || run_row(i) < n ? __ldg(src + uint64_t(idx[i]) * stride) : 0u;
  store_runs<kFull>(dst, x, n);
}

// A probe-side column in general: a run's first and last rows are gathered, a
// middle row only when its probe row is neither of theirs (probe rows rise
// along a run).
template <bool kFull>
__device__ __forceinline__ void write_column_ends(const uint32_t* __restrict__ src, const uint32_t (&idx)[kWriteRows],
                                                  uint32_t* __restrict__ dst, uint32_t n) {
  uint32_t x[kWriteRows];
#pragma unroll
  for (int g = 0; g < kRuns; ++g) {
    const uint32_t a = idx[g * kVec], b = idx[g * kVec + kVec - 1];
    const bool live = kFull || run_row(g * kVec) < n;
    const uint32_t va = live ? __ldg(src + a) : 0u;
    const uint32_t vb = live ? __ldg(src + b) : 0u;
    x[g * kVec] = va;
    x[g * kVec + kVec - 1] = vb;
#pragma unroll
    for (int w = 1; w < kVec - 1; ++w) {
      const uint32_t i = idx[g * kVec + w];
      x[g * kVec + w] = i == a ? va : i == b ? vb : (live ? __ldg(src + i) : 0u);
    }
  }
  store_runs<kFull>(dst, x, n);
}

// A probe-side column when every run of the warp comes from one probe row
// (runs of consecutive output rows of one row, the common case when rows have
// several matches): one gather per run instead of one per row.
template <bool kFull>
__device__ __forceinline__ void write_column_runs(const uint32_t* __restrict__ src, const uint32_t (&idx)[kWriteRows],
                                                  uint32_t* __restrict__ dst, uint32_t n) {
  uint32_t x[kWriteRows];
#pragma unroll
  for (int g = 0; g < kRuns; ++g) {
    const uint32_t v = kFull || run_row(g * kVec) < n ? __ldg(src + idx[g * kVec]) : 0u;
#pragma unroll
    for (int w = 0; w < kVec; ++w) x[g * kVec + w] = v;
  }
  store_runs<kFull>(dst, x, n);
}

// Two build-side columns stored together (row-major pairs): one 8-byte gather
// per row feeds both; half of the thread's runs at a time.
template <bool kFull>
__device__ __forceinline__ void write_pair(const uint32_t* __restrict__ grouped, const uint32_t (&idx)[kWriteRows],
                                           uint32_t* __restrict__ dst0, uint32_t* __restrict__ dst1, uint32_t n) {
  constexpr int kHalf = kWriteRows / 2;
  // every run of the warp reads four consecutive build rows starting at an even
  // row: two 16-byte loads per run
  bool u = true;
#pragma unroll
  for (int g = 0; g < kRuns; ++g) {
    u &= !(idx[g * kVec] & 1u);
#pragma unroll
    for (int w = 1; w < kVec; ++w) u &= idx[g * kVec + w] == idx[g * kVec] + uint32_t(w);
  }
  if (__all_sync(0xffffffffu, u)) {
#pragma unroll
    for (int g = 0; g < kRuns; ++g) {
      const uint32_t q = (uint32_t(g) * kThreads + threadIdx.x) * kVec;
      const uint4* p = reinterpret_cast<const uint4*>(grouped + uint64_t(idx[g * kVec]) * 2);
      const uint4 a = __ldg(p), b = __ldg(p + 1);
      __stcs(reinterpret_cast<uint4*>(dst0 + q), make_uint4(a.x, a.z, b.x, b.z));
      __stcs(reinterpret_cast<uint4*>(dst1 + q), make_uint4(a.y, a.w, b.y, b.w));
    }
    return;
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint2 v[kHalf];
#pragma unroll
    for (int i = 0; i < kHalf; ++i)
      v[i] = kFull || run_row(h * kHalf + i) < n ? __ldg(reinterpret_cast<const uint2*>(grouped) + idx[h * kHalf + i])
                                                 : make_uint2(0u, 0u);
#pragma unroll
    for (int g = 0; g < kRuns / 2; ++g) {
      const uint32_t q = (uint32_t(h * kRuns / 2 + g) * kThreads + threadIdx.x) * kVec;
      const uint2* r = v + g * kVec;
      if (kFull || q + kVec <= n) {
        __stcs(reinterpret_cast<uint4*>(dst0 + q), make_uint4(r[0].x, r[1].x, r[2].x, r[3].x));
        __stcs(reinterpret_cast<uint4*>(dst1 + q), make_uint4(r[0].y, r[1].y, r[2].y, r[3].y));
      } else {
#pragma unroll
        for (int w = 0; w < kVec; ++w)
          if (q + w < n) {
            __stcs(dst0 + q + w, r[w].x);
            __stcs(dst1 + q + w, r[w].y);
          }
      }
    }
  }
}

// Write phase, persistent: CTAs take write items (a join and one of its output
// tiles of kWriteTile rows) from a device work counter until none are left.
// Per item: (1) the probe rows feeding the tile get their output offsets
// (relative to the tile) and group starts staged in shared memory; (2) every
// thread maps 16 consecutive output rows to (probe row, build row) with one
// 32-bit search and a short walk, into a padded row map; (3) every thread takes
// 16 rows striped over the block (a row per lane), reads their map entries once
// per side, and writes the columns with 16-byte streaming stores.
__global__ void __launch_bounds__(kThreads, kWriteBlocks) join_write_kernel(const JoinDesc* __restrict__ jd, const uint64_t* first,
                                                                 uint32_t k, unsigned long long* __restrict__ queue) {
  // dynamic shared memory (kWriteSmem bytes): the stage and the row map
  extern __shared__ __align__(16) uint32_t s_dyn[];
  uint32_t* s_rel = s_dyn;                   // kStageRows + 1
  uint32_t* s_beg = s_rel + kStageRows + 1;  // kStageRows
  uint32_t* s_pk = s_beg + kStageRows;       // kMapWords: probe row of each output row (relative to the tile's first)
  uint32_t* s_bk = s_pk + kMapWords;         // kMapWords: build row of each output row
  __shared__ uint32_t s_skip;
  __shared__ unsigned long long s_item[2];   // this tile's item and the next one's
  // row q lives at q + q / 32: conflict-free both for the 16 consecutive rows a
  // thread maps and for the rows striped over the block that it gathers
  auto mi = [](uint32_t q) { return q + (q >> 5); };
  const uint64_t nitems = first[k];
  if (threadIdx.x == 0) s_item[0] = atomicAdd(queue, 1ull);
  __syncthreads();
  for (int cur = 0;; cur ^= 1) {
    const uint64_t item = s_item[cur];
    if (item >= nitems) break;
    const uint32_t jj = item_join(first, k, item);
    const JoinDesc& d = jd[jj];
    const uint64_t tile = item - first[jj];
    const uint64_t t0 = tile * kWriteTile;
    const uint32_t n = uint32_t(min(uint64_t(kWriteTile), d.T - t0));
    const uint64_t ilo = d.part[tile];
    const uint64_t ihi = d.part[tile + 1] + 1;  // probe rows [ilo, ihi) can feed this tile
    const uint32_t q0 = threadIdx.x * kWriteRows;
    // Up to kStageChunks * kStageRows feeding rows pass through the stage in
    // chunks; each chunk maps the output rows that fall in its rows' ranges.
    // More feeding rows than that (most of them without a match) are searched
    // in global memory instead.
    const bool staged = ihi - ilo <= uint64_t(kStageChunks) * kStageRows;
    if (!staged && q0 < n) {
      uint64_t i = row_of(d, t0 + q0, ilo, ihi + 1);
      for (int j = 0; j < kWriteRows; ++j) {
        const uint32_t q = q0 + j;
        if (q >= n) break;
        const uint64_t r = t0 + q;
        if (off_at(d, i + 1) <= r) i = next_nonzero(d, i);  // ranges are contiguous: the next matching row
        s_pk[mi(q)] = uint32_t(i - ilo);
        s_bk[mi(q)] = d.pbeg[i] + uint32_t(r - off_at(d, i));
        if (!MQ_IN_BOUNDS(i < d.np && s_bk[mi(q)] < d.nb, d.check)) s_pk[mi(q)] = s_bk[mi(q)] = 0;
      }
    }
    for (uint64_t c0 = ilo; staged && c0 < ihi; c0 += kStageRows) {
      const uint32_t ns = uint32_t(min(uint64_t(kStageRows), ihi - c0));
      for (uint32_t r = threadIdx.x; r <= ns; r += kThreads) {
        const uint64_t v = off_at(d, c0 + r);
        s_rel[r] = v <= t0 ? 0u : uint32_t(min(v - t0, uint64_t(kWriteTile)));
      }
      for (uint32_t r = threadIdx.x; r < ns; r += kThreads) s_beg[r] = d.pbeg[c0 + r];
      if (threadIdx.x == 0 && c0 == ilo) s_skip = uint32_t(t0 - off_at(d, ilo));  // rows of ilo before this tile
      __syncthreads();
      const uint32_t qa = max(q0, s_rel[0]), qb = min(q0 + kWriteRows, min(s_rel[ns], n));
      if (qa < qb) {
        uint32_t r = upper_bound_u32(s_rel, 0, ns + 1, qa) - 1;
        const uint32_t skip = c0 == ilo ? s_skip : 0u, rbase = uint32_t(c0 - ilo);
        for (uint32_t q = qa; q < qb; ++q) {
          if (s_rel[r + 1] <= q) {
            ++r;
            if (s_rel[r + 1] <= q) r = upper_bound_u32(s_rel, r + 1, ns + 1, q) - 1;
          }
          s_pk[mi(q)] = rbase + r;
          s_bk[mi(q)] = s_beg[r] + (q - s_rel[r]) + (r == 0 ? skip : 0u);
          if (!MQ_IN_BOUNDS(ilo + rbase + r < d.np && s_bk[mi(q)] < d.nb, d.check)) s_pk[mi(q)] = s_bk[mi(q)] = 0;
        }
      }
      __syncthreads();
    }
    if (!staged) __syncthreads();
    // the next item, fetched while this tile's columns are written (read after the closing barrier)
    if (threadIdx.x == 0) s_item[cur ^ 1] = atomicAdd(queue, 1ull);
    // probe-side columns, then build-side columns: one index array live at a time
    for (int side = 0; side < 2; ++side) {
      const uint32_t* s_map = side ? s_bk : s_pk;
      uint32_t idx[kWriteRows];
#pragma unroll
      for (int i = 0; i < kWriteRows; ++i) {
        const uint32_t q = run_row(i);
        idx[i] = s_map[mi(q < n ? q : n - 1)];  // rows past the tile's end repeat its last row (never stored)
      }
      const uint32_t st = side ? d.bstride : 1u;
      bool runs_uniform = false;
      if (!side) {
        bool u = true;
#pragma unroll
        for (int g = 0; g < kRuns; ++g) u &= idx[g * kVec] == idx[g * kVec + kVec - 1];
        runs_uniform = __all_sync(0xffffffffu, u);
      }
      if (side && d.grouped && d.nbv == 2) {
        // both build columns from one 8-byte gather per row
        int c0 = -1, c1 = -1;
        for (int c = 0; c < d.ncols; ++c)
          if ((d.from_build >> c) & 1u) (d.src[c] == d.grouped ? c0 : c1) = c;
        if (n == kWriteTile) write_pair<true>(d.grouped, idx, d.out[c0] + t0, d.out[c1] + t0, n);
        else write_pair<false>(d.grouped, idx, d.out[c0] + t0, d.out[c1] + t0, n);
        continue;
      }
      for (int c = 0; c < d.ncols; ++c) {
        if (int((d.from_build >> c) & 1u) != side) continue;
        const uint32_t* src = side ? d.src[c] : d.src[c] + ilo;
        if (runs_uniform) {
          if (n == kWriteTile) write_column_runs<true>(src, idx, d.out[c] + t0, n);
          else write_column_runs<false>(src, idx, d.out[c] + t0, n);
        } else if (!side) {
          if (n == kWriteTile) write_column_ends<true>(src, idx, d.out[c] + t0, n);
          else write_column_ends<false>(src, idx, d.out[c] + t0, n);
        } else if (n == kWriteTile) {
          write_column<true>(src, idx, st, d.out[c] + t0, n);
        } else {
          write_column<false>(src, idx, st, d.out[c] + t0, n);
        }
      }
    }
    __syncthreads();
  }
}

// Stores a chunk of four output rows from ``dst`` (j0 of c rows written so
// far, o the first row's index): one 16-byte store when whole and aligned.
__device__ __forceinline__ void store_chunk(uint32_t* __restrict__ dst, uint64_t o, uint32_t j0, uint32_t c,
                                            const uint32_t (&x)[kVec]) {
  if (j0 + kVec <= c && !((o + j0) & (kVec - 1))) {
    __stcs(reinterpret_cast<uint4*>(dst + j0), make_uint4(x[0], x[1], x[2], x[3]));
  } else {
#pragma unroll
    for (int j = 0; j < kVec; ++j)
      if (j0 + j < c) __stcs(dst + j0 + j, x[j]);
  }
}

// Output rows [o, o + c) of probe row i, whose key group starts at build row
// g: every column in chunks of four output rows.  Two grouped build values per
// row (a build row's pair is one 8-byte word) come together: four rows' pairs
// in one 32-byte load when the chunk is whole and 32-byte aligned, else a
// pair per 8-byte load.
__device__ __forceinline__ void write_dense_row(const JoinDesc& d, int ncols, uint32_t bstride, uint64_t i, uint64_t o,
                                                uint32_t c, uint32_t g) {
  const bool pair = bstride == 2;  // grouped build values, two per row
  for (int col = 0; col < ncols; ++col) {
    const bool from_build = (d.from_build >> col) & 1u;
    if (from_build && pair) continue;
    uint32_t* __restrict__ dst = d.out[col] + o;
    const uint32_t* __restrict__ src = d.src[col];
    const uint32_t pv = from_build ? 0u : __ldg(src + i);
    for (uint32_t j0 = 0; j0 < c; j0 += kVec) {
      uint32_t x[kVec];
#pragma unroll
      for (int j = 0; j < kVec; ++j)
        x[j] = !from_build ? pv : j0 + j < c ? __ldg(src + uint64_t(g + j0 + j) * bstride) : 0u;
      store_chunk(dst, o, j0, c, x);
    }
  }
  if (pair) {
    const uint32_t fb = d.from_build;
    const int c0 = __ffs(fb) - 1, c1 = __ffs(fb & (fb - 1)) - 1;  // the columns of build values 0 and 1
    const uint64_t* __restrict__ grp = reinterpret_cast<const uint64_t*>(d.grouped);
    for (uint32_t j0 = 0; j0 < c; j0 += kVec) {
      const uint32_t r0 = g + j0;
      ulonglong2 w01 = make_ulonglong2(0ull, 0ull), w23 = make_ulonglong2(0ull, 0ull);
      if (j0 + kVec <= c && !(r0 & (kVec - 1))) {
        ld_u64x4_nc(grp + r0, &w01, &w23);
      } else {
        w01.x = __ldg(grp + r0);
        if (j0 + 1 < c) w01.y = __ldg(grp + r0 + 1);
        if (j0 + 2 < c) w23.x = __ldg(grp + r0 + 2);
        if (j0 + 3 < c) w23.y = __ldg(grp + r0 + 3);
      }
      const uint32_t x0[kVec] = {uint32_t(w01.x), uint32_t(w01.y), uint32_t(w23.x), uint32_t(w23.y)};
      const uint32_t x1[kVec] = {uint32_t(w01.x >> 32), uint32_t(w01.y >> 32), uint32_t(w23.x >> 32),
                                 uint32_t(w23.y >> 32)};
      store_chunk(d.out[c0] + o, o, j0, c, x0);
      store_chunk(d.out[c1] + o, o, j0, c, x1);
    }
  }
}

// Write phase of a join whose probe rows have few matches (on average at most
// the autotuned crossover, none more than kDenseCap): a thread per probe row
// writes that row's output rows.  Consecutive threads
// own consecutive probe rows, hence consecutive output ranges, so a warp's
// stores of a column stay within a few lines; every whole aligned run of four
// output rows takes one 16-byte store per column.  No partition, no shared
// memory, no barrier.
__global__ void __launch_bounds__(kThreads, kDenseBlocks) dense_write_kernel(const JoinDesc* __restrict__ jd, const uint64_t* first,
                                                              uint32_t k) {
  const uint32_t jj = item_join(first, k, blockIdx.x);
  const JoinDesc& d = jd[jj];
  const uint64_t tile = blockIdx.x - first[jj];
  const uint64_t base = tile * kRowTile, np = d.np;
  const uint64_t tb = d.tile_base[tile];
  const int ncols = d.ncols;
  const uint32_t bstride = d.bstride;
#pragma unroll kDenseUnroll
  for (int it = 0; it < kRowItems; ++it) {
    const uint64_t i = base + uint64_t(it) * kThreads + threadIdx.x;
    if (i >= np) break;  // later rows of this thread are past the end too
    const uint64_t o = tb + d.local[i];
    const uint64_t e = i + 1 == np ? d.T : ((i + 1) % kRowTile ? tb + d.local[i + 1] : d.tile_base[tile + 1]);
    const uint32_t c = uint32_t(e - o);
    if (!c) continue;
    const uint32_t g = d.pbeg[i];
    if (!MQ_IN_BOUNDS(e <= d.T && uint64_t(g) + c <= d.nb, d.check)) continue;
    write_dense_row(d, ncols, bstride, i, o, c, g);
  }
}

// One pass for a dense hash join whose output size is bounded before the
// count: no probe row has more matches than the largest key group of the
// build side, so capacity ``cap`` = probe rows x that group size holds the
// output.  Each CTA takes the next probe tile by an atomic ticket, looks its
// rows up as the count phase does (keeping each row's count and group start
// in shared memory), scans the counts, learns the tile's output offset by
// decoupled look-back over the tiles before it (a tile publishes its sum as
// soon as its lookups end, before it writes), then writes its rows' output as
// the dense write does.  The probe keys are read once, and no group start or
// offset goes through global memory.  The last tile writes the row count.
// Status bits: 2 a look-back wait gave up, 4 a tile of 2^32 or more rows,
// 8 an output range beyond the capacity or a group beyond the build side.
__global__ void __launch_bounds__(kThreads, kFusedBlocks) fused_dense_kernel(const JoinDesc* __restrict__ jd,
                                                                          uint64_t* __restrict__ scratch,
                                                                          uint32_t* __restrict__ status,
                                                                          uint32_t spin_limit, uint64_t cap,
                                                                          uint64_t* __restrict__ total) {
  __shared__ uint32_t s_cnt[kRowTile + kRowTile / 32];  // counts, then tile-local offsets
  __shared__ uint32_t s_beg[kRowTile];
  __shared__ uint64_t s_warp[kThreads / 32];
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_prefix;
  const JoinDesc& d = jd[0];
  const HashTable t = d.t;
  auto pad = [](int i) { return i + (i >> 5); };
  if (threadIdx.x == 0) s_tile = uint32_t(atomicAdd(reinterpret_cast<unsigned long long*>(scratch), 1ull));
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint64_t base = uint64_t(tile) * kRowTile, np = d.np;
  if (base >= np) return;  // the same for the whole block
  // lookups, kFusedProbeIn rows in flight per thread (keys loaded as they are
  // needed: the registers go to more CTAs per SM)
#pragma unroll
  for (int h0 = 0; h0 < kRowItems; h0 += kFusedProbeIn) {
    uint64_t key[kFusedProbeIn];
    uint32_t b[kFusedProbeIn], sl[kFusedProbeIn];
    ulonglong2 k01[kFusedProbeIn], k23[kFusedProbeIn];
#pragma unroll
    for (int q = 0; q < kFusedProbeIn; ++q) {
      const uint64_t row = base + uint64_t(h0 + q) * kThreads + threadIdx.x;
      key[q] = row < np ? load_key(d.pk, row) : kEmptyKey;
    }
#pragma unroll
    for (int q = 0; q < kFusedProbeIn; ++q)
      if (key[q] != kEmptyKey) load_bucket(t, key[q], &b[q], &k01[q], &k23[q]);
#pragma unroll
    for (int q = 0; q < kFusedProbeIn; ++q) {
      const uint64_t row = base + uint64_t(h0 + q) * kThreads + threadIdx.x;
      sl[q] = row < np ? find_slot(t, key[q], b[q], k01[q], k23[q]) : kNoSlot;
    }
#pragma unroll
    for (int q = 0; q < kFusedProbeIn; ++q) {
      const int loc = (h0 + q) * kThreads + threadIdx.x;
      const uint2 g = sl[q] != kNoSlot ? *group_of(t, sl[q]) : make_uint2(0u, 0u);
      s_beg[loc] = g.x ? group_begin(t, sl[q], g.y) : 0u;
      s_cnt[pad(loc)] = g.x;
    }
  }
  __syncthreads();
  uint32_t v[kRowItems];
  uint64_t sum = 0;
#pragma unroll
  for (int q = 0; q < kRowItems; ++q) {
    v[q] = s_cnt[pad(threadIdx.x * kRowItems + q)];
    sum += v[q];
  }
  uint64_t tile_sum;
  uint64_t run = block_scan(sum, s_warp, &tile_sum);
  if (threadIdx.x < 32) {
    const uint64_t p = lb_tile_prefix(scratch + 1, tile, tile_sum, status, spin_limit);
    if (threadIdx.x == 0) s_prefix = p;
  }
#pragma unroll
  for (int q = 0; q < kRowItems; ++q) {
    s_cnt[pad(threadIdx.x * kRowItems + q)] = uint32_t(run);
    run += v[q];
  }
  __syncthreads();
  const uint64_t prefix = s_prefix;
  if (threadIdx.x == 0) {
    if (base + kRowTile >= np) *total = prefix + tile_sum;
    if (tile_sum > 0xffffffffull) atomicOr(status, 4u);
  }
  const int ncols = d.ncols;
  const uint32_t bstride = d.bstride;
#pragma unroll kDenseUnroll
  for (int it = 0; it < kRowItems; ++it) {
    const int loc = it * kThreads + threadIdx.x;
    const uint64_t i = base + loc;
    if (i >= np) break;  // later rows of this thread are past the end too
    const uint32_t off = s_cnt[pad(loc)];
    const uint32_t c = uint32_t((loc + 1 < kRowTile ? uint64_t(s_cnt[pad(loc + 1)]) : tile_sum) - off);
    if (!c) continue;
    const uint64_t o = prefix + off;
    const uint32_t g = s_beg[loc];
    if (o + c > cap || uint64_t(g) + c > d.nb) {
      atomicOr(status, 8u);
      continue;
    }
    write_dense_row(d, ncols, bstride, i, o, c, g);
  }
}

// Cross products (no shared variable): output row r pairs probe row r / nb
// with build row r % nb; items are output tiles of kWriteTile rows.
__global__ void __launch_bounds__(kThreads) cross_write_kernel(const JoinDesc* __restrict__ jd, const uint64_t* first,
                                                              uint32_t k) {
  const uint32_t jj = item_join(first, k, blockIdx.x);
  const JoinDesc& d = jd[jj];
  const uint64_t t0 = (blockIdx.x - first[jj]) * kWriteTile;
  const uint64_t n = min(uint64_t(kWriteTile), d.T - t0);
  for (uint64_t q = threadIdx.x; q < n; q += kThreads) {
    const uint64_t r = t0 + q;
    const uint64_t i = r / d.nb, b = r - i * d.nb;
    for (int c = 0; c < d.ncols; ++c) {
      const bool fb = (d.from_build >> c) & 1u;
      __stcs(d.out[c] + r, __ldg(d.src[c] + (fb ? b : i)));
    }
  }
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
  for (int q = 0; q < ns; ++q) {
    lay->lkey[q] = find(L, shared[q]);
    lay->rkey[q] = find(R, shared[q]);
    lay->var[n] = shared[q];
    lay->side[n] = 0;
    lay->col[n] = lay->lkey[q];
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
    if (t->nrows && (!t->col[c] || (reinterpret_cast<uintptr_t>(t->col[c]) & 3)))
      return set_error(ctx, MAPSQ_ERR_INVALID, "%s table: column %u is NULL or not 4-byte aligned", which, c);
  }
  if (t->ncols && t->nrows && !t->on_device)
    return set_error(ctx, MAPSQ_ERR_INVALID, "%s table: columns must be on the device", which);
  return MAPSQ_OK;
}

// Host side of one join of a batch.
struct JoinPlan {
  Layout lay;
  const mapsq_table *B = nullptr, *P = nullptr;
  int bside = 1;
  const int *bkey = nullptr, *pkey = nullptr;
  uint64_t nb = 0, np = 0, T = 0, M = 0;
  bool cross = false, hash = false, hll = false, sorted = false;
  uint64_t maxc = 0;  // largest match count of a probe row (after the count phase)
  bool part = false;  // the build side is partitioned by region before the insert (large hash builds)
  std::vector<uint32_t> region_off;  // first row of each region in the partitioned build side
};

// A batch of k joins, split in two halves so that the caller can allocate the
// outputs once their sizes are known: count() runs the map, shuffle and count
// phases and sets every T; write() runs the partition and write phases.
// Device memory comes from ``Mem`` (the context's allocator, or a fixed array
// carved by the caller).
template <class Mem>
struct BatchJoin {
  Ctx* ctx;               // NULL without a context (no profiling, no launch count, pageable copies)
  cudaStream_t stream;
  uint32_t* status;       // device status word
  Mem* mem;
  std::vector<JoinPlan> plans;
  std::vector<JoinDesc> descs;
  JoinDesc* d_descs = nullptr;
  uint64_t* d_first = nullptr;             // kPhases x (k + 1) item offsets
  std::vector<uint64_t> first;             // host copy
  std::vector<uint64_t> host;              // read-back buffer
  std::vector<uint8_t> take;               // joins that write() produces (all by default)
  uint32_t k = 0;
  int algorithm = MAPSQ_JOIN_AUTO;
  uint32_t sorted_ratio = kSortedRatio;
  uint64_t part_min_build = kHllMinBuild;  // build rows from which a hash build is partitioned first
  uint64_t dense_max = kDenseMax;          // largest mean matches per probe row for the dense write
  bool allow_fused = false;                // a single large dense hash join may take one pass (join_batch)
  bool fused = false;                      // it does: plans[0].T is the output's capacity until write()

  // The context's autotuned choices (hash vs sorted, partitioned build, dense write).
  void tune_from(const Ctx* c) {
    sorted_ratio = c->sorted_ratio;
    part_min_build = c->part_min_build;
    dense_max = c->dense_max;
  }
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
  int upload(void* dst, const void* src, size_t bytes) {
    if (ctx) return stage_upload(ctx, dst, src, bytes);
    MQ_TRY(cuda(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, stream), "upload"));
    return cuda(cudaStreamSynchronize(stream), "upload");  // pageable source: wait before it goes away
  }
  // Reads ``words`` 64-bit words into host[0, words) (synchronises the stream).
  int readback(const void* dptr, size_t words) {
    host.assign(words, 0);
    if (ctx && words <= kReadWords) return read_words(ctx, dptr, words, host.data());
    MQ_TRY(cuda(cudaMemcpyAsync(host.data(), dptr, words * 8, cudaMemcpyDeviceToHost, stream), "readback"));
    return cuda(cudaStreamSynchronize(stream), "cudaStreamSynchronize");
  }
  uint64_t* phase_first(int ph) { return d_first + size_t(ph) * (k + 1); }
  uint64_t items(int ph) const { return first[size_t(ph) * (k + 1) + k]; }
  // item offsets of phase ph from per-join item counts
  void set_items(int ph, const std::vector<uint64_t>& per) {
    uint64_t* f = first.data() + size_t(ph) * (k + 1);
    f[0] = 0;
    for (uint32_t j = 0; j < k; ++j) f[j + 1] = f[j] + per[j];
  }

  int prepare(uint32_t nj, const mapsq_table* const* L, const mapsq_table* const* R) {
    k = nj;
    take.assign(k, 1);
    plans.assign(k, JoinPlan{});
    descs.assign(k, JoinDesc{});
    first.assign(size_t(kPhases) * (k + 1), 0);
    for (uint32_t j = 0; j < k; ++j) {
      JoinPlan& pl = plans[j];
      if (!L[j] || !R[j]) return fail(MAPSQ_ERR_INVALID, "NULL table in a join batch");
      MQ_TRY(check_table(ctx, L[j], "left"));
      MQ_TRY(check_table(ctx, R[j], "right"));
      MQ_TRY(make_layout(ctx, L[j], R[j], &pl.lay));
      // build on the smaller side; but a side sorted on the (one) key column that
      // is several times larger than the other is already grouped: it becomes
      // the build side of a sorted join and the other side searches it
      const bool lsorted = pl.lay.nkey == 1 && ((L[j]->sorted_mask >> pl.lay.lkey[0]) & 1u);
      const bool rsorted = pl.lay.nkey == 1 && ((R[j]->sorted_mask >> pl.lay.rkey[0]) & 1u);
      bool build_left = L[j]->nrows < R[j]->nrows;
      const uint64_t nl = L[j]->nrows, nr = R[j]->nrows;
      const uint64_t ratio = algorithm == MAPSQ_JOIN_SORTED ? 0 : sorted_ratio;
      const bool allow = algorithm != MAPSQ_JOIN_HASH && ratio != 0xffffffffu && nl > 0 && nr > 0;
      // both sorted: the larger one is searched
      const bool use_l = allow && lsorted && nl >= ratio * nr && (!rsorted || nl >= nr);
      const bool use_r = allow && !use_l && rsorted && nr >= ratio * nl;
      if (use_l || use_r) {
        build_left = use_l;
        pl.sorted = true;
      }
      pl.B = build_left ? L[j] : R[j];
      pl.P = build_left ? R[j] : L[j];
      pl.bside = build_left ? 0 : 1;
      pl.bkey = build_left ? pl.lay.lkey : pl.lay.rkey;
      pl.pkey = build_left ? pl.lay.rkey : pl.lay.lkey;
      pl.nb = pl.B->nrows;
      pl.np = pl.P->nrows;
      pl.cross = pl.lay.nkey == 0;
      pl.hash = !pl.cross && pl.nb > 0 && pl.np > 0 && !pl.sorted;
      pl.hll = pl.hash && pl.nb >= kHllMinBuild;
      if (pl.nb >= (uint64_t(1) << 31)) return fail(MAPSQ_ERR_UNSUPPORTED, "build side of 2^31 rows or more");
      if (pl.cross && pl.nb && pl.np > UINT64_MAX / pl.nb) return fail(MAPSQ_ERR_BUDGET, "cross product overflows 64 bits");
      JoinDesc& d = descs[j];
      d.check = status;  // the word given at construction (the batch's own word replaces ``status`` later)
      d.nb = pl.nb;
      d.np = pl.np;
      d.cross = pl.cross;
      d.hash = pl.hash;
      d.sorted = pl.sorted;
      if (!pl.cross) {
        d.bk = KeyCols{pl.B->col[pl.bkey[0]], pl.lay.nkey == 2 ? pl.B->col[pl.bkey[1]] : nullptr};
        d.pk = KeyCols{pl.P->col[pl.pkey[0]], pl.lay.nkey == 2 ? pl.P->col[pl.pkey[1]] : nullptr};
      }
      for (int c = pl.lay.nkey; c < pl.lay.ncols; ++c)
        if (pl.lay.side[c] == pl.bside) d.bsrc[d.nbv++] = pl.B->col[pl.lay.col[c]];
    }
    return MAPSQ_OK;
  }

  // Distinct-key estimates of the large build sides, then the table sizes.
  uint32_t pl_rows(uint32_t j) const { return uint32_t(plans[j].nb); }

  int size_tables() {
    std::vector<uint64_t> per(k, 0);
    uint32_t nh = 0;
    for (uint32_t j = 0; j < k; ++j) {
      const JoinPlan& pl = plans[j];
      plans[j].M = pl.hash ? std::max<uint64_t>(1024, 2 * pl.nb) : 0;
      if (pl.hll) {
        per[j] = ceil_div(pl.nb, uint64_t(kRowTile) * kHllSpan);
        ++nh;
      }
    }
    if (nh) {
      uint32_t* regs = nullptr;
      MQ_TRY(mem->get(size_t(nh) * kHllWords, &regs));
      MQ_TRY(cuda(cudaMemsetAsync(regs, 0, size_t(nh) * kHllWords * 4, stream), "memset"));
      uint32_t h = 0;
      for (uint32_t j = 0; j < k; ++j)
        if (plans[j].hll) descs[j].hll = regs + size_t(h++) * kHllWords;
      set_items(PH_HLL, per);
      MQ_TRY(upload_descs());
      int r = rec(K_HLL);
      hll_kernel<<<unsigned(items(PH_HLL)), kThreads, 0, stream>>>(d_descs, phase_first(PH_HLL), k);
      launched();
      double bytes = 0;
      for (auto& pl : plans) bytes += pl.hll ? 4.0 * pl.lay.nkey * pl.nb : 0;
      done(r, bytes);
      MQ_TRY(cuda(cudaGetLastError(), "hll_kernel"));
      MQ_TRY(readback(regs, size_t(nh) * kHllWords / 2));
      h = 0;
      for (uint32_t j = 0; j < k; ++j) {
        if (!plans[j].hll) continue;
        const uint32_t* w = reinterpret_cast<const uint32_t*>(host.data()) + size_t(h++) * kHllWords;
        const double est = hll_estimate(w);
        // load factor about 0.4 (measured: 0.8 and 0.6 probe past the home
        // bucket more often, 0.3 only grows the table)
        plans[j].M = std::min<uint64_t>(plans[j].M, std::max<uint64_t>(1024, uint64_t(2.5 * est) + 1024));
        // the partition's region offsets (exclusive prefix sums of the histogram)
        plans[j].region_off.assign(kRegions, 0);
        uint32_t run = 0;
        for (int r = 0; r < kRegions; ++r) {
          plans[j].region_off[r] = run;
          run += w[kHllRegs + r];
        }
        // partitioned from the autotuned build size on (when the histogram covers every row, as it should)
        plans[j].part = run == pl_rows(j) && plans[j].nb >= part_min_build;
      }
    }
    for (auto& pl : plans) {
      if (pl.M >= 0xfffffff0ull) pl.M = 0xfffffff0ull;
      pl.M = (pl.M + kBucket - 1) / kBucket * kBucket;
    }
    return MAPSQ_OK;
  }

  // Descriptors, item offsets and a zeroed tail go up together, in one copy.
  // The tail holds the status word, the write phase's work counter, the joins'
  // row counts, their largest match counts per probe row, their largest key
  // groups and their numbers of groups, so that each upload resets them and
  // one copy reads back all.
  uint64_t* d_tail = nullptr;
  size_t tail_words() const { return 2 + 4 * size_t(k); }
  size_t blob_bytes() const { return sizeof(JoinDesc) * k + sizeof(uint64_t) * first.size() + sizeof(uint64_t) * tail_words(); }
  int ensure_blob() {
    if (d_descs) return MAPSQ_OK;
    const size_t db = sizeof(JoinDesc) * k, fb = sizeof(uint64_t) * first.size();
    unsigned char* blob = nullptr;
    MQ_TRY(mem->get(blob_bytes(), &blob));
    d_descs = reinterpret_cast<JoinDesc*>(blob);
    d_first = reinterpret_cast<uint64_t*>(blob + db);
    d_tail = reinterpret_cast<uint64_t*>(blob + db + fb);
    status = reinterpret_cast<uint32_t*>(d_tail);
    return MAPSQ_OK;
  }
  int upload_descs() {
    const size_t db = sizeof(JoinDesc) * k, fb = sizeof(uint64_t) * first.size(), tb = sizeof(uint64_t) * tail_words();
    MQ_TRY(ensure_blob());
    blob_host.assign(db + fb + tb, 0);
    memcpy(blob_host.data(), descs.data(), db);
    memcpy(blob_host.data() + db, first.data(), fb);
    return upload(d_descs, blob_host.data(), db + fb + tb);
  }
  std::vector<unsigned char> blob_host;

  // Tables and per-join scratch; item offsets of the build and count phases.
  int allocate() {
    size_t keys = 0, groups = 0;
    for (auto& pl : plans)
      if (pl.hash) {
        keys += pl.M;
        groups += pl.M + 1;
      }
    uint64_t *all_keys = nullptr;
    uint2* all_groups = nullptr;
    MQ_TRY(mem->get(std::max<size_t>(keys, 1), &all_keys));
    MQ_TRY(mem->get(std::max<size_t>(groups, 1), &all_groups));
    if (keys) MQ_TRY(cuda(cudaMemsetAsync(all_keys, 0xff, keys * 8, stream), "memset"));  // all slots empty
    if (groups) MQ_TRY(cuda(cudaMemsetAsync(all_groups, 0, groups * 8, stream), "memset"));
    std::vector<uint64_t> ins(k, 0), slots(k, 0), scat(k, 0), cnt(k, 0), scnt(k, 0);
    // the per-join arrays below, in one block (as the allocator rounds them)
    size_t need = 0;
    auto add = [&need](uint64_t count, size_t elem) { need += ((count * elem ? count * elem : 16) + 255) & ~size_t(255); };
    for (uint32_t j = 0; j < k; ++j) {
      const JoinPlan& pl = plans[j];
      if (!pl.sorted && !pl.hash) continue;
      const uint64_t nt = ceil_div(pl.np, kRowTile);
      add(kEarlyTiles + 1, 8), add(pl.np / 32 + 1, 4), add(pl.np, 4), add(pl.np, 4), add(nt, 8), add(nt + 1, 8);
      if (pl.sorted) continue;
      const uint64_t nslot_tiles = ceil_div(pl.M + 1, kRowTile);
      add(nslot_tiles, 8), add(nslot_tiles + 1, 8), add(pl.nb, 4), add(pl.nb, 4);
      if (descs[j].nbv) add(pl.nb * descs[j].nbv, 4);
    }
    MQ_TRY(mem->reserve(need));
    size_t ko = 0, go = 0;
    for (uint32_t j = 0; j < k; ++j) {
      const JoinPlan& pl = plans[j];
      JoinDesc& d = descs[j];
      if (pl.sorted) {
        const uint64_t nt = ceil_div(pl.np, kRowTile);
        MQ_TRY(mem->get(kEarlyTiles + 1, &d.part));
        MQ_TRY(mem->get(pl.np / 32 + 1, &d.nzmask));
        MQ_TRY(mem->get(pl.np, &d.local));
        MQ_TRY(mem->get(pl.np, &d.pbeg));
        MQ_TRY(mem->get(nt, &d.tile_total));
        MQ_TRY(mem->get(nt + 1, &d.tile_base));
        scnt[j] = nt;
        continue;
      }
      if (!pl.hash) continue;
      d.t.keys = all_keys + ko;
      d.t.group = all_groups + go;
      d.t.M = uint32_t(pl.M);
      ko += pl.M;
      go += pl.M + 1;
      const uint64_t nslot_tiles = ceil_div(pl.M + 1, kRowTile);
      const uint64_t nt = ceil_div(pl.np, kRowTile);
      MQ_TRY(mem->get(nslot_tiles, &d.slot_total));
      MQ_TRY(mem->get(nslot_tiles + 1, &d.t.slot_base));
      MQ_TRY(mem->get(pl.nb, &d.slot_of));
      MQ_TRY(mem->get(pl.nb, &d.rank_of));
      if (d.nbv) MQ_TRY(mem->get(pl.nb * d.nbv, &d.grouped));
      MQ_TRY(mem->get(kEarlyTiles + 1, &d.part));
      MQ_TRY(mem->get(pl.np / 32 + 1, &d.nzmask));
      MQ_TRY(mem->get(pl.np, &d.local));
      MQ_TRY(mem->get(pl.np, &d.pbeg));
      MQ_TRY(mem->get(nt, &d.tile_total));
      MQ_TRY(mem->get(nt + 1, &d.tile_base));
      ins[j] = ceil_div(pl.nb, kRowTile);
      slots[j] = nslot_tiles;
      scat[j] = d.nbv ? ins[j] : 0;
      cnt[j] = nt;
    }
    set_items(PH_INSERT, ins);
    set_items(PH_SLOTS, slots);
    set_items(PH_SCATTER, scat);
    set_items(PH_COUNT, cnt);
    set_items(PH_SORTED, scnt);
    return allocate_partition();
  }

  // Partitioned copies of the large build sides; the insert and the scatter
  // then read the copies (the descriptors point at them).
  std::vector<PartDesc> pdescs;
  std::vector<uint32_t> pcursor;
  unsigned char* d_pblob = nullptr;
  int allocate_partition() {
    std::vector<uint64_t> per(k, 0);
    uint32_t npart = 0;
    for (auto& pl : plans) npart += pl.hash && pl.part;
    set_items(PH_REGION, per);
    if (!npart) return MAPSQ_OK;
    pdescs.assign(k, PartDesc{});
    pcursor.assign(size_t(k) * kRegions, 0);
    MQ_TRY(mem->get(sizeof(PartDesc) * k + 4 * pcursor.size(), &d_pblob));
    uint32_t* d_cursor = reinterpret_cast<uint32_t*>(d_pblob + sizeof(PartDesc) * k);
    for (uint32_t j = 0; j < k; ++j) {
      const JoinPlan& pl = plans[j];
      if (!pl.hash || !pl.part) continue;
      JoinDesc& d = descs[j];
      PartDesc& pd = pdescs[j];
      pd.nkey = pl.lay.nkey;
      pd.n = pl.nb;
      pd.check = d.check;
      pd.cursor = d_cursor + size_t(j) * kRegions;
      for (int q = 0; q < pl.lay.nkey; ++q) pd.src[pd.ncols++] = pl.B->col[pl.bkey[q]];
      for (int c = pl.lay.nkey; c < pl.lay.ncols; ++c)
        if (pl.lay.side[c] == pl.bside) pd.src[pd.ncols++] = pl.B->col[pl.lay.col[c]];
      uint32_t* copy = nullptr;
      MQ_TRY(mem->get(size_t(pl.nb) * pd.ncols, &copy));
      for (int c = 0; c < pd.ncols; ++c) pd.dst[c] = copy + size_t(pl.nb) * c;
      d.bk = KeyCols{pd.dst[0], pl.lay.nkey == 2 ? pd.dst[1] : nullptr};
      for (int v = 0; v < d.nbv; ++v) d.bsrc[v] = pd.dst[pl.lay.nkey + v];
      std::copy(pl.region_off.begin(), pl.region_off.end(), pcursor.begin() + size_t(j) * kRegions);
      per[j] = ceil_div(pl.nb, kPartRows);
    }
    set_items(PH_REGION, per);
    return MAPSQ_OK;
  }

  int partition_phase() {
    if (!items(PH_REGION)) return MAPSQ_OK;
    std::vector<unsigned char> blob(sizeof(PartDesc) * k + 4 * pcursor.size());
    memcpy(blob.data(), pdescs.data(), sizeof(PartDesc) * k);
    memcpy(blob.data() + sizeof(PartDesc) * k, pcursor.data(), 4 * pcursor.size());
    MQ_TRY(upload(d_pblob, blob.data(), blob.size()));
    double bytes = 0;
    for (uint32_t j = 0; j < k; ++j) bytes += 8.0 * pdescs[j].ncols * pdescs[j].n;
    const int r = rec(K_PARTITION_BUILD);
    partition_kernel<<<unsigned(items(PH_REGION)), kPartThreads, 0, stream>>>(
        reinterpret_cast<const PartDesc*>(d_pblob), phase_first(PH_REGION), k);
    launched();
    done(r, bytes);
    return cuda(cudaGetLastError(), "partition_kernel");
  }

  // Build phases of the hash joins: partition, insert, group starts, scatter.
  int build_phases() {
    MQ_TRY(upload_descs());
    MQ_TRY(partition_phase());
    double bytes = 0;
    if (items(PH_INSERT)) {
      for (auto& pl : plans) bytes += pl.hash ? 4.0 * pl.lay.nkey * pl.nb : 0;
      const int r = rec(K_HASH_INSERT);
      hash_insert_kernel<<<unsigned(items(PH_INSERT)), kThreads, 0, stream>>>(d_descs, phase_first(PH_INSERT), k,
                                                                               status);
      launched();
      done(r, bytes);
    }
    if (items(PH_SLOTS)) {
      bytes = 0;
      for (auto& pl : plans) bytes += pl.hash ? 16.0 * (pl.M + 1) : 0;
      const int r = rec(K_PREFIX_SUM);
      slot_scan_kernel<<<unsigned(items(PH_SLOTS)), kThreads, 0, stream>>>(d_descs, phase_first(PH_SLOTS), k,
                                                                          d_tail + 2 + 2 * size_t(k));
      launched();
      tiles_scan_kernel<<<k, 1024, 0, stream>>>(d_descs, k, 0, nullptr);
      launched();
      done(r, bytes);
    }
    if (items(PH_SCATTER)) {
      bytes = 0;
      for (uint32_t j = 0; j < k; ++j) bytes += plans[j].hash ? 4.0 * descs[j].nbv * plans[j].nb : 0;
      const int r = rec(K_HASH_SCATTER);
      hash_scatter_kernel<<<unsigned(items(PH_SCATTER)), kThreads, 0, stream>>>(d_descs, phase_first(PH_SCATTER), k);
      launched();
      done(r, bytes);
    }
    return cuda(cudaGetLastError(), "build phases");
  }

  // Count phases: every probe row's matches, then the tile offsets.
  int probe_phases() {
    double bytes = 0;
    if (items(PH_COUNT)) {
      for (auto& pl : plans) bytes += pl.hash ? 4.0 * pl.lay.nkey * pl.np : 0;
      const int r = rec(K_PROBE_COUNT);
      probe_count_kernel<<<unsigned(items(PH_COUNT)), kThreads, 0, stream>>>(d_descs, phase_first(PH_COUNT), k,
                                                                             status, d_tail + 2);
      launched();
      done(r, bytes);
    }
    if (items(PH_SORTED)) {
      bytes = 0;
      for (auto& pl : plans) bytes += pl.sorted ? 4.0 * pl.np : 0;
      const int r = rec(K_SORTED_COUNT);
      sorted_count_kernel<<<unsigned(items(PH_SORTED)), kSortedThreads, 0, stream>>>(
          d_descs, phase_first(PH_SORTED), k, status, d_tail + 2, items(PH_SORTED) <= kKaryMaxItems);
      launched();
      done(r, bytes);
    }
    // joins of more than one probe tile need the scan of their tile totals
    bool scan = false;
    for (auto& pl : plans) scan |= (pl.hash || pl.sorted) && pl.np > uint64_t(kRowTile);
    if (scan) {
      tiles_scan_kernel<<<k, 1024, 0, stream>>>(d_descs, k, 1, d_tail + 2);
      launched();
    }
    return cuda(cudaGetLastError(), "count phases");
  }

  int count_phases() {
    MQ_TRY(build_phases());
    return probe_phases();
  }

  // Reads the first ``words`` words of the tail into host[] (and the context's
  // status word: an earlier call's write phase may have set it).
  int read_tail(size_t words) {
    host.assign(words, 0);
    if (ctx && words <= kReadWords) return read_words(ctx, d_tail, words, host.data());
    // through the context's pinned buffer when it is large enough (a pageable copy is slower)
    // (words 0-63 of it are left to read_u64 and the status word)
    uint64_t* dst = ctx && words + 64 <= kPinnedWords ? ctx->h_pinned + 64 : host.data();
    MQ_TRY(cuda(cudaMemcpyAsync(dst, d_tail, words * 8, cudaMemcpyDeviceToHost, stream), "readback"));
    if (ctx)
      MQ_TRY(cuda(cudaMemcpyAsync(ctx->h_pinned + 32, ctx->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                  stream), "readback"));
    MQ_TRY(cuda(cudaStreamSynchronize(stream), "cudaStreamSynchronize"));
    if (dst != host.data()) memcpy(host.data(), dst, words * 8);
    return ctx ? check_status(ctx) : MAPSQ_OK;
  }

  // A single dense hash join with a large probe side may take one pass
  // (fused_dense_kernel) if its build groups are even enough that probe rows x
  // the largest group bounds the output closely: that bound is allocated.
  bool fused_candidate() const {
    return allow_fused && ctx && k == 1 && take[0] && plans[0].hash && plans[0].np >= kFusedMinProbe &&
           plans[0].lay.ncols > 0;
  }
  bool fused_fits(uint64_t maxg, uint64_t ngroups) const {
    const JoinPlan& pl = plans[0];
    if (maxg == 0 || maxg > dense_max || maxg > kDenseCap || maxg * ngroups > 2 * pl.nb) return false;
    const uint64_t cap = pl.np * maxg;
    const uint64_t bytes = ((cap + 63) & ~uint64_t(63)) * uint64_t(pl.lay.ncols) * 4;
    return !ctx->budget || ctx->in_use + bytes <= ctx->budget / 2;
  }

  int count() {
    MQ_TRY(size_tables());
    MQ_TRY(ensure_blob());
    // a retry rebuilds the tables in place of the first attempt's (a fixed
    // scratch array would otherwise hold both sets)
    const auto mark = mem->mark();
    for (int attempt = 0;; ++attempt) {
      if (attempt) mem->rewind(mark);
      MQ_TRY(allocate());
      const bool cand = fused_candidate();
      if (cand) {
        // the build first: its largest group and number of groups decide
        MQ_TRY(build_phases());
        MQ_TRY(read_tail(tail_words()));
        const uint32_t st = uint32_t(host[0]);
        if (st & 1u) {
          if (attempt > 0) return fail(MAPSQ_ERR_CUDA, "hash table full");
          plans[0].M = (std::max<uint64_t>(1024, 2 * plans[0].nb) + kBucket - 1) / kBucket * kBucket;
          continue;
        }
        if (st) return fail(MAPSQ_ERR_CUDA, "device status word set");
        const uint64_t maxg = host[2 + 2 * size_t(k)], ngroups = host[2 + 3 * size_t(k)];
        if (fused_fits(maxg, ngroups)) {
          fused = true;
          plans[0].maxc = maxg;
          plans[0].T = descs[0].T = plans[0].np * maxg;  // the capacity; write() learns the row count
          return MAPSQ_OK;
        }
        MQ_TRY(probe_phases());
      } else {
        MQ_TRY(count_phases());  // its upload zeroes the status word
      }
      // cross products and joins with an empty side: every row count is known here
      bool device_counts = false;
      for (auto& pl : plans) device_counts |= pl.hash || pl.sorted;
      if (!device_counts) {
        for (uint32_t j = 0; j < k; ++j) {
          plans[j].T = descs[j].T = plans[j].cross ? plans[j].np * plans[j].nb : 0;
          plans[j].maxc = 0;
        }
        return MAPSQ_OK;
      }
      // one read: status word, work counter, row counts and largest counts
      MQ_TRY(read_tail(2 + 2 * size_t(k)));
      const uint32_t st = uint32_t(host[0]);
      if (st & 1u) {
        // a distinct-key estimate far too low: rebuild every table at two slots per build row
        if (attempt > 0) return fail(MAPSQ_ERR_CUDA, "hash table full");
        for (auto& pl : plans)
          if (pl.hash) pl.M = (std::max<uint64_t>(1024, 2 * pl.nb) + kBucket - 1) / kBucket * kBucket;
        continue;
      }
      if (st & 4u)
        return fail(MAPSQ_ERR_UNSUPPORTED, "2048 consecutive probe rows with 2^32 or more matches");
      if (st) return fail(MAPSQ_ERR_CUDA, "device status word set");
      for (uint32_t j = 0; j < k; ++j) {
        const JoinPlan& pl = plans[j];
        plans[j].T = descs[j].T = pl.cross ? pl.np * pl.nb : pl.hash || pl.sorted ? host[2 + j] : 0;
        plans[j].maxc = pl.hash || pl.sorted ? host[2 + k + j] : 0;
      }
      return MAPSQ_OK;
    }
  }

  // Raise a kernel's dynamic shared memory limit to ``bytes``, once per device
  // (``which`` numbers the kernels that need it).
  int set_smem_once(const void* fn, int which, int bytes) {
    static std::atomic<uint64_t> done[3][4] = {};  // per kernel: a bit per device
    int dev = 0;
    MQ_TRY(cuda(cudaGetDevice(&dev), "cudaGetDevice"));
    const uint64_t bit = uint64_t(1) << (dev & 63);
    if (dev < 256 && (done[which][dev >> 6].load() & bit)) return MAPSQ_OK;
    MQ_TRY(cuda(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes), "cudaFuncSetAttribute"));
    if (dev < 256) done[which][dev >> 6] |= bit;
    return MAPSQ_OK;
  }

  // The one-pass join (count() chose it): lookups, scan, look-back and write
  // in one launch over the probe tiles, then one read of the row count, which
  // replaces the capacity in plans[0].T.
  int write_fused(double bytes) {
    const JoinPlan& pl = plans[0];
    const uint64_t ntiles = ceil_div(pl.np, kRowTile), cap = pl.T;
    uint64_t* lb = nullptr;  // ticket, then one look-back word per tile
    MQ_TRY(mem->get(1 + ntiles, &lb));
    MQ_TRY(cuda(cudaMemsetAsync(lb, 0, (1 + ntiles) * sizeof(uint64_t), stream), "memset"));
    MQ_TRY(upload_descs());  // zeroes the tail: status word and row count
    const int r = rec(K_FUSED_JOIN);
    fused_dense_kernel<<<unsigned(ntiles), kThreads, 0, stream>>>(d_descs, lb, status, ctx->wait_spins, cap,
                                                                 d_tail + 2);
    launched();
    done(r, bytes);
    MQ_TRY(cuda(cudaGetLastError(), "fused_dense_kernel"));
    MQ_TRY(read_tail(3));
    const uint32_t st = uint32_t(host[0]);
    if (st & 2u) return set_error(ctx, MAPSQ_ERR_TIMEOUT, "a bounded look-back wait gave up (status 0x%x)", st);
    if (st & 4u) return fail(MAPSQ_ERR_UNSUPPORTED, "2048 consecutive probe rows with 2^32 or more matches");
    if (st) return fail(MAPSQ_ERR_CUDA, "one-pass join: output beyond its capacity");
    plans[0].T = descs[0].T = host[2];
    return MAPSQ_OK;
  }

  // Partition and write phases into out[j] (ncols device columns of T rows each).
  int write(uint32_t* const* const* out) {
    std::vector<uint64_t> part(k, 0), wr(k, 0), cr(k, 0), dn(k, 0);
    double bytes = 0, cbytes = 0, dbytes = 0;
    for (uint32_t j = 0; j < k; ++j) {
      const JoinPlan& pl = plans[j];
      JoinDesc& d = descs[j];
      d.ncols = pl.lay.ncols;
      d.from_build = 0;
      d.bstride = pl.sorted ? 1u : uint32_t(d.nbv);
      uint32_t b = 0;
      double in = 0;
      for (int c = 0; c < pl.lay.ncols; ++c) {
        const bool fb = pl.lay.side[c] == pl.bside && c >= pl.lay.nkey;
        d.out[c] = out[j] ? out[j][c] : nullptr;  // joins not taken have no output table
        if (fb) {
          d.src[c] = pl.cross || pl.sorted ? pl.B->col[pl.lay.col[c]] : d.grouped + b++;
          d.from_build |= 1u << c;
          in += 4.0 * (pl.sorted ? std::min(pl.nb, pl.T) : pl.nb);  // a sorted side is read where it matches
        } else {
          // key columns and the probe side's own columns come from the probe row
          d.src[c] = pl.P->col[c < pl.lay.nkey ? pl.pkey[c] : pl.lay.col[c]];
          if (c >= pl.lay.nkey) in += 4.0 * pl.np;
        }
      }
      if (!pl.T || !pl.lay.ncols || !take[j]) continue;
      if (fused) {
        dbytes += 4.0 * pl.lay.nkey * pl.np + 4.0 * pl.np * pl.lay.ncols * pl.maxc + in;  // counted as written in full
        continue;
      }
      const uint64_t ntiles = ceil_div(pl.T, kWriteTile);
      if (pl.cross) {
        cr[j] = ntiles;
        cbytes += 4.0 * pl.T * pl.lay.ncols + in;
      } else if (pl.T <= dense_max * pl.np && pl.maxc <= kDenseCap) {  // few matches per probe row on average
        dn[j] = ceil_div(pl.np, kRowTile);
        dbytes += 4.0 * pl.T * pl.lay.ncols + in;
      } else {
        if (ntiles > kEarlyTiles) {  // else the count scan wrote the partition
          MQ_TRY(mem->get(ntiles + 1, &d.part));
          part[j] = ceil_div(ntiles + 1, kThreads);
        }
        wr[j] = ntiles;
        bytes += 4.0 * pl.T * pl.lay.ncols + in;
      }
    }
    if (fused) return write_fused(dbytes);
    set_items(PH_PART, part);
    set_items(PH_WRITE, wr);
    set_items(PH_CROSS, cr);
    set_items(PH_DENSE, dn);
    if (!items(PH_WRITE) && !items(PH_CROSS) && !items(PH_DENSE)) return MAPSQ_OK;
    MQ_TRY(upload_descs());
    if (items(PH_WRITE)) {
      unsigned long long* queue = reinterpret_cast<unsigned long long*>(d_tail + 1);  // zeroed by the upload
      if (items(PH_PART)) {
        const int r = rec(K_PARTITION);
        write_partition_kernel<<<unsigned(items(PH_PART)), kThreads, 0, stream>>>(d_descs, phase_first(PH_PART), k);
        launched();
        done(r, 8.0 * items(PH_WRITE));
      }
      int r = rec(K_JOIN_WRITE);
      const unsigned grid = unsigned(std::min<uint64_t>(items(PH_WRITE), 152ull * 4));
      MQ_TRY(set_smem_once(reinterpret_cast<const void*>(join_write_kernel), 0, kWriteSmem));
      join_write_kernel<<<grid, kThreads, kWriteSmem, stream>>>(d_descs, phase_first(PH_WRITE), k, queue);
      launched();
      done(r, bytes);
    }
    if (items(PH_DENSE)) {
      const int r = rec(K_DENSE_WRITE);
      dense_write_kernel<<<unsigned(items(PH_DENSE)), kThreads, 0, stream>>>(d_descs, phase_first(PH_DENSE), k);
      launched();
      done(r, dbytes);
    }
    if (items(PH_CROSS)) {
      int r = rec(K_CROSS_WRITE);
      cross_write_kernel<<<unsigned(items(PH_CROSS)), kThreads, 0, stream>>>(d_descs, phase_first(PH_CROSS), k);
      launched();
      done(r, cbytes);
    }
    MQ_TRY(cuda(cudaGetLastError(), "write phases"));
    return ctx ? checked_sync(ctx) : MAPSQ_OK;
  }
};

}  // namespace

int join_batch(Ctx* ctx, uint32_t k, const mapsq_table* const* L, const mapsq_table* const* R,
               const mapsq_join_opts* opts, TableImpl** out) {
  if (k == 0) return MAPSQ_OK;
  if (opts && (opts->algorithm < MAPSQ_JOIN_AUTO || opts->algorithm > MAPSQ_JOIN_SORTED))
    return set_error(ctx, MAPSQ_ERR_INVALID, "join algorithm %d", opts->algorithm);
  Scratch scratch(ctx);
  BatchJoin<Scratch> bj{ctx, ctx->stream, ctx->d_status, &scratch};
  bj.algorithm = opts ? opts->algorithm : MAPSQ_JOIN_AUTO;
  bj.tune_from(ctx);
  bj.allow_fused = true;
  MQ_TRY(bj.prepare(k, L, R));
  MQ_TRY(bj.count());
  std::vector<TableImpl*> tabs(k, nullptr);
  std::vector<uint32_t* const*> cols(k, nullptr);
  int rc = MAPSQ_OK;
  if (k > 1) {
    // the batch's results in one allocation (each table a view of its part)
    std::vector<uint64_t> rows(k);
    std::vector<uint32_t> nc(k);
    std::vector<const int32_t*> vars(k);
    for (uint32_t j = 0; j < k; ++j) {
      rows[j] = bj.plans[j].T;
      nc[j] = uint32_t(bj.plans[j].lay.ncols);
      vars[j] = bj.plans[j].lay.var;
    }
    rc = tables_alloc_shared(ctx, k, rows.data(), nc.data(), vars.data(), tabs.data());
    for (uint32_t j = 0; j < k && rc == MAPSQ_OK; ++j) cols[j] = tabs[j]->pub.col;
  } else {
    // (a one-pass join's table is allocated at its capacity, then given its row count)
    rc = table_alloc(ctx, bj.plans[0].T, uint32_t(bj.plans[0].lay.ncols), bj.plans[0].lay.var, &tabs[0]);
    if (rc == MAPSQ_OK) cols[0] = tabs[0]->pub.col;
  }
  if (rc == MAPSQ_OK) rc = bj.write(cols.data());
  if (rc != MAPSQ_OK) {
    for (auto* t : tabs) table_release(ctx, t);
    return rc;
  }
  if (bj.fused) tabs[0]->pub.nrows = bj.plans[0].T;
  for (uint32_t j = 0; j < k; ++j) out[j] = tabs[j];
  return MAPSQ_OK;
}

int join_batch_admit(Ctx* ctx, uint32_t k, const mapsq_table* const* L, const mapsq_table* const* R,
                     uint64_t budget_bytes, TableImpl** out, int* status, uint64_t* need) {
  for (uint32_t j = 0; j < k; ++j) {
    out[j] = nullptr;
    status[j] = 1;
    need[j] = 0;
  }
  if (k == 0) return MAPSQ_OK;
  Scratch scratch(ctx);
  BatchJoin<Scratch> bj{ctx, ctx->stream, ctx->d_status, &scratch};
  bj.tune_from(ctx);
  MQ_TRY(bj.prepare(k, L, R));
  MQ_TRY(bj.count());
  // admission in order: result tables are written while they fit in the budget
  uint64_t used = 0;
  for (uint32_t j = 0; j < k; ++j) {
    const uint64_t bytes = 4 * ((bj.plans[j].T + 63) & ~uint64_t(63)) * uint64_t(bj.plans[j].lay.ncols);
    need[j] = bytes;
    bj.take[j] = 0;
    if (budget_bytes && used + bytes > budget_bytes) continue;
    bj.take[j] = 1;
    used += bytes;
  }
  std::vector<TableImpl*> tabs(k, nullptr);
  std::vector<uint32_t* const*> cols(k, nullptr);
  int rc = MAPSQ_OK;
  for (uint32_t j = 0; j < k && rc == MAPSQ_OK; ++j) {
    if (!bj.take[j]) continue;
    rc = table_alloc(ctx, bj.plans[j].T, uint32_t(bj.plans[j].lay.ncols), bj.plans[j].lay.var, &tabs[j]);
    if (rc == MAPSQ_OK) cols[j] = tabs[j]->pub.col;
  }
  if (rc == MAPSQ_OK) rc = bj.write(cols.data());
  if (rc != MAPSQ_OK) {
    for (auto* t : tabs) table_release(ctx, t);
    return rc;
  }
  for (uint32_t j = 0; j < k; ++j)
    if (bj.take[j]) {
      out[j] = tabs[j];
      status[j] = 0;
    }
  return MAPSQ_OK;
}

int join_tables(Ctx* ctx, const mapsq_table* L, const mapsq_table* R, const mapsq_join_opts* opts,
                TableImpl** out) {
  return join_batch(ctx, 1, &L, &R, opts, out);
}

// A join computed slice by slice of its larger input, each slice's result
// copied to the caller's host columns and freed before the next (Algorithm 1
// distributes over a split of one input: a row's matches all lie in the other,
// whole input).  A slice whose count or result does not fit in the context's
// memory (MAPSQ_ERR_BUDGET or MAPSQ_ERR_OOM) is halved and retried.
int join_to_host(Ctx* ctx, const mapsq_table* L, const mapsq_table* R, const mapsq_join_opts* opts,
                 uint32_t* const* host_cols, uint64_t capacity, uint64_t* out_rows, mapsq_table* out,
                 uint32_t* slices) {
  if (opts && (opts->algorithm < MAPSQ_JOIN_AUTO || opts->algorithm > MAPSQ_JOIN_SORTED))
    return set_error(ctx, MAPSQ_ERR_INVALID, "join algorithm %d", opts->algorithm);
  Layout lay;
  MQ_TRY(check_table(ctx, L, "left"));
  MQ_TRY(check_table(ctx, R, "right"));
  MQ_TRY(make_layout(ctx, L, R, &lay));
  if (host_cols)
    for (int c = 0; c < lay.ncols; ++c)
      if (!host_cols[c]) return set_error(ctx, MAPSQ_ERR_INVALID, "host column %d is NULL", c);
  const bool split_left = L->nrows >= R->nrows;
  const mapsq_table* big = split_left ? L : R;
  const uint64_t n = big->nrows;
  uint64_t off = 0, chunk = std::max<uint64_t>(n, 1), total = 0;
  uint32_t nslices = 0;
  bool writing = host_cols != nullptr;  // false once the result is known to overflow the host columns
  do {
    const uint64_t c = std::min(chunk, n - off);
    mapsq_table slice = *big;
    slice.nrows = c;
    for (uint32_t q = 0; q < slice.ncols; ++q)
      if (slice.col[q]) slice.col[q] += off;
    const mapsq_table* A = split_left ? &slice : L;
    const mapsq_table* B = split_left ? R : &slice;
    int rc;
    uint64_t rows = 0;
    {
      Scratch scratch(ctx);
      BatchJoin<Scratch> bj{ctx, ctx->stream, ctx->d_status, &scratch};
      bj.algorithm = opts ? opts->algorithm : MAPSQ_JOIN_AUTO;
      bj.tune_from(ctx);
      rc = bj.prepare(1, &A, &B);
      if (rc == MAPSQ_OK) rc = bj.count();
      if (rc == MAPSQ_OK) rows = bj.plans[0].T;
      if (rc == MAPSQ_OK && writing && total + rows > capacity) writing = false;
      if (rc == MAPSQ_OK && writing && rows) {
        TableImpl* t = nullptr;
        rc = table_alloc(ctx, rows, uint32_t(lay.ncols), lay.var, &t);
        if (rc == MAPSQ_OK) {
          uint32_t* const* cols[1] = {t->pub.col};
          rc = bj.write(cols);
          for (int q = 0; q < lay.ncols && rc == MAPSQ_OK; ++q) {
            const cudaError_t e = cudaMemcpyAsync(host_cols[q] + total, t->pub.col[q], rows * sizeof(uint32_t),
                                                  cudaMemcpyDeviceToHost, ctx->stream);
            if (e != cudaSuccess) rc = cuda_fail(ctx, e, "cudaMemcpyAsync", __FILE__, __LINE__);
          }
          if (rc == MAPSQ_OK) {
            const cudaError_t e = cudaStreamSynchronize(ctx->stream);
            if (e != cudaSuccess) rc = cuda_fail(ctx, e, "cudaStreamSynchronize", __FILE__, __LINE__);
          }
          table_release(ctx, t);
        }
      }
    }
    if (rc == MAPSQ_ERR_BUDGET || rc == MAPSQ_ERR_OOM) {
      if (c <= 1) return rc;  // a single row's join does not fit
      chunk = c / 2;
      continue;
    }
    MQ_TRY(rc);
    total += rows;
    off += c;
    ++nslices;
  } while (off < n);
  *out_rows = total;
  if (slices) *slices = nslices;
  if (host_cols && total > capacity)
    return set_error(ctx, MAPSQ_ERR_BUDGET, "the join has %llu rows, the host columns hold %llu",
                     (unsigned long long)total, (unsigned long long)capacity);
  if (out) {
    memset(out, 0, sizeof(*out));
    out->nrows = host_cols ? total : 0;
    out->ncols = uint32_t(lay.ncols);
    for (int c = 0; c < MAPSQ_MAX_VARS; ++c) out->var[c] = c < lay.ncols ? lay.var[c] : -1;
    for (int c = 0; c < lay.ncols && host_cols; ++c) out->col[c] = host_cols[c];
    out->on_device = 0;
  }
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
constexpr uint64_t kNoAllocMaxRows = uint64_t(1) << 32;   // output rows
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
  int reserve(size_t) { return MAPSQ_OK; }  // one fixed array: nothing to reserve
  size_t mark() const { return used; }
  void rewind(size_t m) { used = m; }  // the stream has finished with everything past m
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
  // the limits hold for the smaller and the larger input, checked before any device work
  const uint64_t n_small = std::min(left->nrows, right->nrows), n_large = std::max(left->nrows, right->nrows);
  if (n_small > kNoAllocMaxBuild || n_large > kNoAllocMaxProbe) return MAPSQ_ERR_INVALID;  // beyond the scratch array
  unsigned char* base = nullptr;
  MQ_TRY(noalloc_scratch(&base));
  Carve carve{base};
  uint32_t* status = nullptr;
  MQ_TRY(carve.get(64, &status));
  BatchJoin<Carve> bj{nullptr, static_cast<cudaStream_t>(cuda_stream), status, &carve};
  // always the hash build on the smaller input: the sorted join would build on
  // a larger, key-sorted side, which the limits above do not cover
  bj.algorithm = MAPSQ_JOIN_HASH;
  MQ_TRY(bj.prepare(1, &left, &right));
  const JoinPlan& pl = bj.plans[0];
  const int ncols = pl.lay.ncols;
  if (ncols && !out_cols) return MAPSQ_ERR_INVALID;
  for (int c = 0; c < ncols; ++c)
    if (!out_cols[c] || (reinterpret_cast<uintptr_t>(out_cols[c]) & 15)) return MAPSQ_ERR_INVALID;
  MQ_TRY(bj.count());
  *out_rows = pl.T;
  if (pl.T > out_capacity_rows) return MAPSQ_ERR_BUDGET;
  if (pl.T > kNoAllocMaxRows) return MAPSQ_ERR_UNSUPPORTED;  // its write partition would not fit in the array
  memset(out, 0, sizeof(*out));
  out->nrows = pl.T;
  out->ncols = uint32_t(ncols);
  out->on_device = 1;
  for (int c = 0; c < MAPSQ_MAX_VARS; ++c) out->var[c] = c < ncols ? pl.lay.var[c] : -1;
  for (int c = 0; c < ncols; ++c) out->col[c] = out_cols[c];
  uint32_t* const* cols[1] = {out_cols};
  return bj.write(cols);
}
