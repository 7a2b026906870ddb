// Single-pass exclusive prefix sum with decoupled look-back (Merrill and
// Garland, "Single-pass Parallel Prefix Scan with Decoupled Look-back", 2016).
//
// A launch scans ``n`` values produced on the fly by a functor (a loaded array,
// or the match counts of a hash probe) and writes their exclusive prefix sums,
// plus the total at index n, in one pass: every CTA takes the next tile by an
// atomic ticket, publishes its tile's sum, then adds the sums of the tiles
// before it as soon as they are published.  Waits on a predecessor are bounded:
// after ``spin_limit`` polls (a launch parameter; kLookbackSpinDefault unless
// the context sets another) the CTA records bit 2 in the status word and goes
// on with the partial prefix it has, so a launch always ends.
#pragma once

#include <cstdint>

namespace mapsq {

constexpr int kLbThreads = 256;
constexpr int kLbItems = 16;
constexpr int kLbTile = kLbThreads * kLbItems;
constexpr uint32_t kLookbackSpinDefault = 1u << 20;  // about 50 ms of polls with 32 ns sleeps

// status word of one tile: flag in the top two bits, sum in the low 62
constexpr uint64_t kLbFlagAggregate = 1ull << 62;
constexpr uint64_t kLbFlagPrefix = 2ull << 62;
constexpr uint64_t kLbValueMask = (1ull << 62) - 1;

// Scratch of a look-back scan: a ticket counter and one status word per tile,
// zeroed before the launch.
inline size_t lookback_scratch_words(uint64_t n) { return 1 + (n + kLbTile - 1) / kLbTile; }

__device__ __forceinline__ int lb_pad(int i) { return i + (i >> 4); }

// Exclusive prefix of this tile (sum of all earlier tiles) by warp-wide look-back.
__device__ __forceinline__ uint64_t lb_tile_prefix(uint64_t* tile_status, uint32_t tile, uint64_t aggregate,
                                                   uint32_t* err, uint32_t spin_limit) {
  const unsigned lane = threadIdx.x & 31;
  if (tile == 0) {
    if (lane == 0) atomicExch(reinterpret_cast<unsigned long long*>(&tile_status[0]), kLbFlagPrefix | aggregate);
    return 0;
  }
  if (lane == 0) atomicExch(reinterpret_cast<unsigned long long*>(&tile_status[tile]), kLbFlagAggregate | aggregate);
  uint64_t prefix = 0;
  int64_t j = int64_t(tile) - 1;  // closest predecessor not yet accounted for
  uint32_t spins = 0;
  while (true) {
    int64_t idx = j - int64_t(lane);
    uint64_t w = 2ull << 62;  // before the first tile: an inclusive prefix of 0
    if (idx >= 0) w = *reinterpret_cast<volatile uint64_t*>(&tile_status[idx]);
    unsigned has_prefix = __ballot_sync(0xffffffffu, (w >> 62) == 2);
    int stop = has_prefix ? __ffs(has_prefix) - 1 : 31;  // closest lane holding an inclusive prefix
    // only the lanes up to that one are needed; wait while one of them is unpublished
    unsigned not_ready = __ballot_sync(0xffffffffu, (w >> 62) == 0) & ((2u << stop) - 1u);
    if (not_ready) {
      if (++spins > spin_limit) {
        if (lane == 0) atomicOr(err, 2u);
        break;
      }
      __nanosleep(32);
      continue;
    }
    uint64_t v = w & kLbValueMask;
    if (int(lane) > stop) v = 0;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    prefix += v;
    if (has_prefix) break;
    j -= 32;
  }
  if (lane == 0)
    atomicExch(reinterpret_cast<unsigned long long*>(&tile_status[tile]), kLbFlagPrefix | ((prefix + aggregate) & kLbValueMask));
  return prefix;
}

// A producer fills the tile's values in row order: ``fill(base, n, s)`` writes
// s[lb_pad(k)] = value of row base + k for k in [0, kLbTile), 0 past row n.
// Values are below 2^32.  Rows are striped over the threads for coalescing.
struct LbArrayProducer {
  const uint32_t* in;
  __device__ __forceinline__ void fill(uint64_t base, uint64_t n, uint64_t* s) const {
#pragma unroll 4
    for (int k = 0; k < kLbItems; ++k) {
      const int local = k * kLbThreads + threadIdx.x;
      const uint64_t row = base + local;
      s[lb_pad(local)] = row < n ? uint64_t(in[row]) : 0ull;
    }
  }
};

// A sink receives the exclusive prefix sum of every row (``store``) and the
// total (``total``, called once).
template <class OutT>
struct LbArraySink {
  OutT* out;  // n + 1 entries: prefix sums, then the total
  uint64_t n;
  __device__ __forceinline__ void store(uint64_t row, uint64_t v) const { out[row] = OutT(v); }
  __device__ __forceinline__ void total(uint64_t v) const { out[n] = OutT(v); }
};

// Block-wide exclusive scan of the tile held in ``s_val`` (kLbTile values in
// row order, padded by lb_pad): each thread scans 16 consecutive values, the
// threads' sums are scanned with warp shuffles.  Returns this thread's
// exclusive prefix (within the tile) in *thread_excl and the tile's sum.
__device__ __forceinline__ uint64_t lb_block_scan(const uint64_t* s_val, uint64_t* s_warp, uint64_t* thread_excl) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint64_t sum = 0;
#pragma unroll
  for (int k = 0; k < kLbItems; ++k) sum += s_val[lb_pad(tid * kLbItems + k)];
  uint64_t inc = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint64_t t = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += t;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  uint64_t warp_excl = 0, tile_sum = 0;
#pragma unroll
  for (int w = 0; w < kLbThreads / 32; ++w) {
    uint64_t x = s_warp[w];
    if (w < warp) warp_excl += x;
    tile_sum += x;
  }
  *thread_excl = warp_excl + inc - sum;
  return tile_sum;
}

// One tile of the scan over n values: ``sink`` receives every row's exclusive
// prefix sum and the total.  ``scratch`` = [ticket, status[ntiles]], zeroed
// before the launch; a ticket past the last tile does nothing.
template <class Producer, class Sink>
__device__ __forceinline__ void lookback_scan_tile(const Producer& prod, uint64_t n, const Sink& sink,
                                                   uint64_t* scratch, uint32_t* err, uint32_t spin_limit) {
  __shared__ uint64_t s_val[kLbTile + kLbTile / 16];
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_warp[kLbThreads / 32];
  __shared__ uint64_t s_prefix;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_tile = uint32_t(atomicAdd(reinterpret_cast<unsigned long long*>(&scratch[0]), 1ull));
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint64_t base = uint64_t(tile) * kLbTile;
  if (base >= n) return;  // the same for the whole block
  prod.fill(base, n, s_val);
  __syncthreads();
  uint64_t excl;
  const uint64_t tile_sum = lb_block_scan(s_val, s_warp, &excl);
  if (warp == 0) {
    uint64_t p = lb_tile_prefix(scratch + 1, tile, tile_sum, err, spin_limit);
    if (lane == 0) s_prefix = p;
  }
  __syncthreads();
  uint64_t run = s_prefix + excl;
#pragma unroll
  for (int k = 0; k < kLbItems; ++k) {
    const int idx = lb_pad(tid * kLbItems + k);
    uint64_t v = s_val[idx];
    s_val[idx] = run;
    run += v;
  }
  __syncthreads();
#pragma unroll 4
  for (int k = 0; k < kLbItems; ++k) {
    const int local = k * kLbThreads + tid;
    const uint64_t row = base + local;
    if (row < n) sink.store(row, s_val[lb_pad(local)]);
  }
  if (base + kLbTile >= n && tid == 0) sink.total(s_prefix + tile_sum);
}

}  // namespace mapsq
