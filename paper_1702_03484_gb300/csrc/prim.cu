// Device primitives: single-pass exclusive prefix sum and a vectorised column copy.
#include "internal.cuh"
#include "lookback.cuh"

namespace mapsq {

namespace {

template <class OutT>
__global__ void __launch_bounds__(kLbThreads) prefix_sum_kernel(const uint32_t* __restrict__ in, uint64_t n,
                                                                OutT* __restrict__ out, uint64_t* scratch,
                                                                uint32_t* err, uint32_t spin_limit) {
  LbArrayProducer v{in};
  LbArraySink<OutT> sink{out, n};
  lookback_scan_tile(v, n, sink, scratch, err, spin_limit);
}

__global__ void copy_u32_kernel(uint32_t* __restrict__ dst, const uint32_t* __restrict__ src, uint64_t n) {
  uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  bool vec = ((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15) == 0;
  if (vec) {
    uint64_t n4 = n / 4;
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += stride) d4[i] = s4[i];
    for (uint64_t i = n4 * 4 + uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
  } else {
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
  }
}

// ``withhold_first``: the ticket counter starts at 1, so no CTA takes the
// first tile and every other tile's look-back waits for a predecessor that is
// never published (the bounded-wait self-test).
template <class OutT>
int prefix_sum_impl(Ctx* ctx, const uint32_t* in, OutT* out, uint64_t n, bool withhold_first = false) {
  if (n == 0) {
    MQ_CUDA(cudaMemsetAsync(out, 0, sizeof(OutT), ctx->stream));
    return MAPSQ_OK;
  }
  uint64_t ntiles = ceil_div(n, kLbTile);
  if (ntiles > 0x7fffffffULL) return set_error(ctx, MAPSQ_ERR_INVALID, "prefix sum of %llu items", (unsigned long long)n);
  Scratch scratch(ctx);
  uint64_t* lb = nullptr;
  MQ_TRY(scratch.get(lookback_scratch_words(n), &lb));
  MQ_CUDA(cudaMemsetAsync(lb, 0, lookback_scratch_words(n) * sizeof(uint64_t), ctx->stream));
  if (withhold_first) {
    static const uint64_t one = 1;
    MQ_CUDA(cudaMemcpyAsync(lb, &one, sizeof one, cudaMemcpyHostToDevice, ctx->stream));
  }
  int rec = prof_begin(ctx, K_PREFIX_SUM);
  prefix_sum_kernel<OutT><<<unsigned(ntiles), kLbThreads, 0, ctx->stream>>>(in, n, out, lb, ctx->d_status,
                                                                            ctx->wait_spins);
  ++ctx->launches;
  prof_end(ctx, rec, double(n) * (sizeof(uint32_t) + sizeof(OutT)));
  MQ_CUDA(cudaGetLastError());
  return MAPSQ_OK;
}

}  // namespace

int prefix_sum_u32_u64(Ctx* ctx, const uint32_t* in, uint64_t* out, uint64_t n) {
  return prefix_sum_impl<uint64_t>(ctx, in, out, n);
}

int prefix_sum_u32_u32(Ctx* ctx, const uint32_t* in, uint32_t* out, uint64_t n) {
  return prefix_sum_impl<uint32_t>(ctx, in, out, n);
}

int prefix_sum_withheld(Ctx* ctx, const uint32_t* in, uint64_t* out, uint64_t n) {
  return prefix_sum_impl<uint64_t>(ctx, in, out, n, true);
}

int copy_u32(Ctx* ctx, uint32_t* dst, const uint32_t* src, uint64_t n) {
  if (n == 0) return MAPSQ_OK;
  int rec = prof_begin(ctx, K_COPY);
  uint64_t blocks = std::min<uint64_t>(ceil_div(n / 4 + 1, 256), 152ull * 16);
  copy_u32_kernel<<<unsigned(blocks), 256, 0, ctx->stream>>>(dst, src, n);
  ++ctx->launches;
  MQ_CUDA(cudaGetLastError());
  prof_end(ctx, rec, double(n) * 8.0);
  return MAPSQ_OK;
}

}  // namespace mapsq
