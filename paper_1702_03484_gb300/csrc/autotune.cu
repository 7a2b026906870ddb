// Autotuner of the AUTO join choice (hash build vs. search of a sorted side).
//
// Both algorithms compute the same result (Algorithm 1); which one is faster
// depends on the sizes and on the GPU: the hash join streams the larger side
// once after building a table of the smaller, the sorted join searches the
// sorted side once per row of the other side.  mapsq_autotune times both on
// synthetic joins of decreasing other-side sizes and keeps, in the context,
// the ratio of sorted-side rows to other-side rows from which the sorted join
// is never slower; AUTO joins use it.
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
