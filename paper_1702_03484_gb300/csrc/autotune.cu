// Autotuner of the join's choices, per size and skew, on this GPU.
//
// Every choice computes the same result (Algorithm 1); which one is faster
// depends on the sizes, the key skew and the GPU:
// * hash build vs search of a sorted side: the hash join streams the larger
//   side once after building a table of the smaller, the sorted join searches
//   the sorted side once per row of the other side -- timed on joins of
//   decreasing other-side sizes (the ratio of sorted-side rows to other-side
//   rows from which the sorted join is never slower);
// * region partition of a hash build side or not, per build size (it pays
//   once the table and the grouped values outgrow the L2);
// * dense write (a thread per probe row) or partitioned write (output tiles
//   spread over all SMs), per key-group size: the dense write is balanced
//   while groups are small; a join takes it when its mean number of matches
//   per probe row is at most the measured crossover (and no row has more
//   than kDenseCap matches).
// The context keeps the three choices; AUTO joins, queries and the serving
// loop use them.
#include <algorithm>
#include <cstring>

#include "internal.cuh"

namespace mapsq {

namespace {

// Sorted side: key i / 2 (each key twice), value i.
__global__ void sorted_side_kernel(uint32_t* __restrict__ key, uint32_t* __restrict__ val, uint64_t n) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
    key[i] = uint32_t(i >> 1);
    val[i] = uint32_t(i);
  }
}

// Other side: keys uniform over [0, domain) from a counter hash (SplitMix64's
// finaliser), value i.
__global__ void other_side_kernel(uint32_t* __restrict__ key, uint32_t* __restrict__ val, uint64_t n,
                                  uint64_t domain) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
    uint64_t z = (i + 1) * 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    key[i] = uint32_t(((z >> 32) * domain) >> 32);
    val[i] = uint32_t(i);
  }
}

// Keys of ``nkeys`` distinct ids, scattered over uint32 by a bijective mix:
// the build side has row i on id i % nkeys, the probe side a uniform id per
// row (a counter hash); values are row numbers.
__device__ __forceinline__ uint32_t mixed_id(uint64_t id) {
  uint64_t z = (id + 0x632be59bd9b4e019ull) * 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return uint32_t(z ^ (z >> 31));
}

__global__ void build_side_kernel(uint32_t* __restrict__ key, uint32_t* __restrict__ val, uint64_t n, uint64_t nkeys) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
    key[i] = mixed_id(i % nkeys);
    val[i] = uint32_t(i);
  }
}

__global__ void probe_side_kernel(uint32_t* __restrict__ key, uint32_t* __restrict__ val, uint64_t n, uint64_t nkeys) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
    key[i] = mixed_id((uint64_t(mixed_id(i ^ 0x5bd1e995u)) * nkeys) >> 32);
    val[i] = uint32_t(i);
  }
}

// Best of three joins of X and Y by ``algorithm``, in milliseconds (CUDA events
// around the whole call, which includes its synchronisation).
int time_join(Ctx* ctx, const mapsq_table* X, const mapsq_table* Y, int algorithm, double* ms) {
  mapsq_join_opts opts{};
  opts.algorithm = algorithm;
  cudaEvent_t a, b;
  MQ_CUDA(cudaEventCreate(&a));
  MQ_CUDA(cudaEventCreate(&b));
  double best = 1e30;
  int rc = MAPSQ_OK;
  for (int rep = 0; rep < 4 && rc == MAPSQ_OK; ++rep) {  // the first one warms up
    TableImpl* out = nullptr;
    cudaEventRecord(a, ctx->stream);
    rc = join_tables(ctx, Y, X, &opts, &out);
    cudaEventRecord(b, ctx->stream);
    if (rc != MAPSQ_OK) break;
    table_release(ctx, out);
    if (cudaEventSynchronize(b) != cudaSuccess) {
      rc = cuda_fail(ctx, cudaGetLastError(), "cudaEventSynchronize", __FILE__, __LINE__);
      break;
    }
    float t = 0.f;
    cudaEventElapsedTime(&t, a, b);
    if (rep > 0) best = std::min(best, double(t));
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms = best;
  return rc;
}

// Synthetic hash join: a build side of nb rows over nb / g keys (g rows per
// key) and a probe side of np rows; returns the best of three times with the
// context's current choices.
int time_hash_join(Ctx* ctx, uint64_t nb, uint64_t g, uint64_t np, double* ms) {
  Scratch scratch(ctx);
  uint32_t *bk = nullptr, *bv = nullptr, *pk = nullptr, *pv = nullptr;
  MQ_TRY(scratch.get(nb, &bk));
  MQ_TRY(scratch.get(nb, &bv));
  MQ_TRY(scratch.get(np, &pk));
  MQ_TRY(scratch.get(np, &pv));
  const uint64_t nkeys = std::max<uint64_t>(1, nb / g);
  build_side_kernel<<<unsigned(std::min<uint64_t>(ceil_div(nb, 256), 152ull * 8)), 256, 0, ctx->stream>>>(bk, bv, nb, nkeys);
  probe_side_kernel<<<unsigned(std::min<uint64_t>(ceil_div(np, 256), 152ull * 8)), 256, 0, ctx->stream>>>(pk, pv, np, nkeys);
  ctx->launches += 2;
  MQ_CUDA(cudaGetLastError());
  mapsq_table B{}, P{};
  B.nrows = nb;
  B.ncols = 2;
  B.var[0] = 0;
  B.var[1] = 1;
  B.col[0] = bk;
  B.col[1] = bv;
  B.on_device = 1;
  P = B;
  P.nrows = np;
  P.var[1] = 2;
  P.col[0] = pk;
  P.col[1] = pv;
  return time_join(ctx, &B, &P, MAPSQ_JOIN_HASH, ms);
}

// The size and skew axes: the partitioned build per build size, the dense
// write per key-group size (the context's fields are set to force each way
// while timing, then to the choices).
int tune_hash_choices(Ctx* ctx, mapsq_autotune_result* r) {
  const uint64_t never = ~uint64_t(0);
  const uint64_t saved_part = ctx->part_min_build, saved_dense = ctx->dense_max;
  int rc = MAPSQ_OK;
  r->part_points = 0;
  for (uint64_t nb = uint64_t(1) << 16; nb <= (uint64_t(1) << 24) && rc == MAPSQ_OK; nb <<= 2) {
    const uint32_t i = r->part_points++;
    r->part_rows[i] = nb;
    ctx->part_min_build = 0;
    rc = time_hash_join(ctx, nb, 2, 4 * nb, &r->part_on_ms[i]);
    ctx->part_min_build = never;
    if (rc == MAPSQ_OK) rc = time_hash_join(ctx, nb, 2, 4 * nb, &r->part_off_ms[i]);
  }
  uint64_t part_min = never;
  for (int i = int(r->part_points) - 1; i >= 0 && r->part_on_ms[i] <= r->part_off_ms[i]; --i) part_min = r->part_rows[i];
  r->dense_points = 0;
  for (uint32_t g = 4; g <= 64 && rc == MAPSQ_OK; g *= 2) {
    const uint32_t i = r->dense_points++;
    r->group[i] = g;
    ctx->part_min_build = part_min;
    ctx->dense_max = never;
    rc = time_hash_join(ctx, uint64_t(1) << 20, g, uint64_t(1) << 20, &r->dense_ms[i]);
    ctx->dense_max = 0;
    if (rc == MAPSQ_OK) rc = time_hash_join(ctx, uint64_t(1) << 20, g, uint64_t(1) << 20, &r->partitioned_ms[i]);
  }
  if (rc != MAPSQ_OK) {  // keep the choices the context had
    ctx->part_min_build = saved_part;
    ctx->dense_max = saved_dense;
    return rc;
  }
  uint64_t dense_max = 0;
  for (uint32_t i = 0; i < r->dense_points && r->dense_ms[i] <= r->partitioned_ms[i]; ++i) dense_max = r->group[i];
  if (dense_max == 0) dense_max = 1;  // a row of one match is written the same way by both
  ctx->part_min_build = part_min;
  ctx->dense_max = dense_max;
  r->part_min_build = part_min;
  r->dense_max = uint32_t(dense_max);
  return MAPSQ_OK;
}

}  // namespace

int autotune(Ctx* ctx, uint64_t n, mapsq_autotune_result* res) {
  if (n == 0) n = uint64_t(1) << 22;
  if (n < 2048 || n >= (uint64_t(1) << 31)) return set_error(ctx, MAPSQ_ERR_INVALID, "sorted_rows %llu", (unsigned long long)n);
  Scratch scratch(ctx);
  uint32_t *xk = nullptr, *xv = nullptr, *yk = nullptr, *yv = nullptr;
  MQ_TRY(scratch.get(n, &xk));
  MQ_TRY(scratch.get(n, &xv));
  MQ_TRY(scratch.get(n, &yk));
  MQ_TRY(scratch.get(n, &yv));
  const unsigned grid = unsigned(std::min<uint64_t>(ceil_div(n, 256), 152ull * 8));
  sorted_side_kernel<<<grid, 256, 0, ctx->stream>>>(xk, xv, n);
  other_side_kernel<<<grid, 256, 0, ctx->stream>>>(yk, yv, n, (n + 1) / 2);
  ctx->launches += 2;
  MQ_CUDA(cudaGetLastError());
  mapsq_table X{}, Y{};
  X.nrows = n;
  X.ncols = 2;
  X.var[0] = 0;
  X.var[1] = 1;
  X.col[0] = xk;
  X.col[1] = xv;
  X.on_device = 1;
  X.sorted_mask = 1u;
  Y = X;
  Y.var[1] = 2;
  Y.col[0] = yk;
  Y.col[1] = yv;
  Y.sorted_mask = 0u;
  mapsq_autotune_result r{};
  r.sorted_rows = n;
  uint32_t chosen = 0xffffffffu;
  for (uint32_t ratio = 1; ratio <= 2048 && r.points < 12 && n / ratio >= 1; ratio *= 2) {
    Y.nrows = n / ratio;
    const uint32_t i = r.points++;
    r.ratio[i] = ratio;
    MQ_TRY(time_join(ctx, &X, &Y, MAPSQ_JOIN_HASH, &r.hash_ms[i]));
    MQ_TRY(time_join(ctx, &X, &Y, MAPSQ_JOIN_SORTED, &r.sorted_ms[i]));
  }
  // the smallest ratio from which the sorted join is never slower
  for (int i = int(r.points) - 1; i >= 0 && r.sorted_ms[i] <= r.hash_ms[i]; --i) chosen = r.ratio[i];
  r.sorted_ratio = chosen;
  ctx->sorted_ratio = chosen;
  MQ_TRY(tune_hash_choices(ctx, &r));
  if (res) *res = r;
  return MAPSQ_OK;
}

}  // namespace mapsq

using namespace mapsq;

extern "C" {

int mapsq_autotune(mapsq_ctx* ctx, uint64_t sorted_rows, mapsq_autotune_result* out) {
  if (!ctx) return MAPSQ_ERR_INVALID;
  std::lock_guard<std::recursive_mutex> cl(ctx->mu);
  if (ctx->server) return set_error(ctx, MAPSQ_ERR_BUSY, "the serving loop is running");
  MQ_CUDA(cudaSetDevice(ctx->device));
  return autotune(ctx, sorted_rows, out);
}

int mapsq_set_sorted_ratio(mapsq_ctx* ctx, uint32_t ratio) {
  if (!ctx) return MAPSQ_ERR_INVALID;
  std::lock_guard<std::recursive_mutex> cl(ctx->mu);
  if (ctx->server) return set_error(ctx, MAPSQ_ERR_BUSY, "the serving loop is running");
  if (ratio == 0) return set_error(ctx, MAPSQ_ERR_INVALID, "sorted ratio 0");
  ctx->sorted_ratio = ratio;
  return MAPSQ_OK;
}

}  // extern "C"
