// Pattern scan: the partial matches of one triple pattern (Section 1; the
// partial-matching step of Section 2), read from the sorted store instead of a
// CPU engine.
//
// With a constant predicate p the candidates are p's segment of the store.  A
// constant subject selects a run of the (p, s, o) order, a constant object a
// run of the (p, o, s) order; both runs are found by binary search on the
// device and the remaining variable's column is copied out.  Two variables
// copy the whole segment; one variable in both places keeps the rows with
// s == o.  Two constants test membership and give 0 or 1 empty binding.
#include <algorithm>
#include <cstring>

#include "internal.cuh"

namespace mapsq {

namespace {

struct RangeQuery {
  uint64_t b, e;     // predicate segment
  uint32_t v0, v1;   // constants
  int32_t kind;
  int32_t pad;
};

struct StoreCols {
  const uint32_t* so_s;
  const uint32_t* so_o;
  const uint32_t* os_o;
  const uint32_t* os_s;
};

// Warp-cooperative search in the sorted run a[lo, hi): the first index whose
// value is >= v (upper = false) or > v (upper = true).  Each round the 32
// lanes test 32 evenly spaced positions, which narrows the range 32-fold: about
// five dependent loads for ten million rows instead of twenty-four.
__device__ __forceinline__ uint64_t warp_bound(const uint32_t* a, uint64_t lo, uint64_t hi, uint32_t v, bool upper) {
  const unsigned lane = threadIdx.x & 31;
  while (hi - lo > 32) {
    const uint64_t step = (hi - lo + 31) / 32;
    const uint64_t pos = lo + lane * step;
    const bool below = pos < hi && (upper ? a[pos] <= v : a[pos] < v);
    const int c = __popc(__ballot_sync(0xffffffffu, below));  // the lanes below v form a prefix
    if (c == 0) return lo;
    const uint64_t nlo = lo + uint64_t(c - 1) * step + 1;
    const uint64_t nhi = c < 32 ? min(hi, lo + uint64_t(c) * step) : hi;
    lo = nlo;
    hi = nhi;
  }
  const uint64_t pos = lo + lane;
  const bool below = pos < hi && (upper ? a[pos] <= v : a[pos] < v);
  return lo + __popc(__ballot_sync(0xffffffffu, below));
}

// The end of the run of v that starts at lo (the first index > v from lo
// on): most runs (a subject's objects under one predicate, an object's
// subjects) are short, so the 32 positions after lo are tested first, one
// dependent load; a longer run is then searched as above.
__device__ __forceinline__ uint64_t warp_run_end(const uint32_t* a, uint64_t lo, uint64_t hi, uint32_t v) {
  const uint64_t pos = lo + (threadIdx.x & 31);
  const unsigned in = __ballot_sync(0xffffffffu, pos < hi && a[pos] <= v);  // a prefix of the lanes
  if (in != 0xffffffffu) return lo + __popc(in);
  return warp_bound(a, lo + 32, hi, v, true);
}

// One warp per pattern.
__global__ void scan_ranges_kernel(const RangeQuery* __restrict__ q, uint32_t n, StoreCols st,
                                   uint64_t* __restrict__ out) {
  const uint32_t i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (i >= n) return;  // whole warps leave together
  RangeQuery r = q[i];
  uint64_t lo = 0, hi = 0;
  switch (r.kind) {
    case KIND_S_BOUND:
      lo = warp_bound(st.so_s, r.b, r.e, r.v0, false);
      hi = warp_run_end(st.so_s, lo, r.e, r.v0);
      break;
    case KIND_O_BOUND:
      lo = warp_bound(st.os_o, r.b, r.e, r.v1, false);
      hi = warp_run_end(st.os_o, lo, r.e, r.v1);
      break;
    case KIND_EXIST: {
      uint64_t a = warp_bound(st.so_s, r.b, r.e, r.v0, false);
      uint64_t z = warp_run_end(st.so_s, a, r.e, r.v0);
      uint64_t k = warp_bound(st.so_o, a, z, r.v1, false);
      lo = k;
      hi = (k < z && st.so_o[k] == r.v1) ? k + 1 : k;
      break;
    }
    case KIND_TWO_VARS:
    case KIND_SAME_VAR:
      lo = r.b;
      hi = r.e;
      break;
    default:
      break;
  }
  if ((threadIdx.x & 31) == 0) {
    out[2 * i] = lo;
    out[2 * i + 1] = hi;
  }
}

__global__ void same_var_flags_kernel(const uint32_t* __restrict__ s, const uint32_t* __restrict__ o, uint64_t n,
                                      uint32_t* __restrict__ flag) {
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x)
    flag[i] = s[i] == o[i] ? 1u : 0u;
}

__global__ void same_var_compact_kernel(const uint32_t* __restrict__ s, uint64_t n, const uint32_t* __restrict__ flag,
                                        const uint64_t* __restrict__ pos, uint32_t* __restrict__ out) {
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x)
    if (flag[i]) out[pos[i]] = s[i];
}

int32_t pattern_kind(const mapsq_pattern& tp) {
  bool sv = tp.var_mask & MAPSQ_VAR_S, ov = tp.var_mask & MAPSQ_VAR_O;
  if (!sv && !ov) return KIND_EXIST;
  if (!sv) return KIND_S_BOUND;
  if (!ov) return KIND_O_BOUND;
  return tp.s == tp.o ? KIND_SAME_VAR : KIND_TWO_VARS;
}

}  // namespace

int validate_pattern(Ctx* ctx, const mapsq_pattern& tp) {
  if (tp.var_mask & ~(MAPSQ_VAR_S | MAPSQ_VAR_P | MAPSQ_VAR_O))
    return set_error(ctx, MAPSQ_ERR_INVALID, "var_mask 0x%x has unknown bits", tp.var_mask);
  if (tp.var_mask & MAPSQ_VAR_P)
    return set_error(ctx, MAPSQ_ERR_UNSUPPORTED, "variable predicates are not supported");
  if ((tp.var_mask & MAPSQ_VAR_S) && tp.s >= MAPSQ_MAX_VARS)
    return set_error(ctx, MAPSQ_ERR_INVALID, "variable id %u out of range", tp.s);
  if ((tp.var_mask & MAPSQ_VAR_O) && tp.o >= MAPSQ_MAX_VARS)
    return set_error(ctx, MAPSQ_ERR_INVALID, "variable id %u out of range", tp.o);
  return MAPSQ_OK;
}

int scan_ranges(Ctx* ctx, const mapsq_pattern* tps, uint32_t n, PatternRange* out) {
  const Store& st = ctx->store;
  std::vector<RangeQuery> q(n);
  for (uint32_t i = 0; i < n; ++i) {
    const mapsq_pattern& tp = tps[i];
    RangeQuery r{};
    auto it = std::lower_bound(st.pred_id.begin(), st.pred_id.end(), tp.p);
    if (it == st.pred_id.end() || *it != tp.p) {
      r.kind = KIND_NONE;
    } else {
      size_t k = size_t(it - st.pred_id.begin());
      r.b = st.pred_begin[k];
      r.e = st.pred_begin[k + 1];
      r.kind = pattern_kind(tp);
      r.v0 = tp.s;
      r.v1 = tp.o;
    }
    q[i] = r;
  }
  Scratch scratch(ctx);
  RangeQuery* dq = nullptr;
  uint64_t* dout = nullptr;
  MQ_TRY(scratch.get(n, &dq));
  MQ_TRY(scratch.get(2 * size_t(n), &dout));
  MQ_TRY(stage_upload(ctx, dq, q.data(), n * sizeof(RangeQuery)));  // pinned, asynchronous
  StoreCols sc{st.so_s, st.so_o, st.os_o, st.os_s};
  int rec = prof_begin(ctx, K_SCAN_RANGES);
  scan_ranges_kernel<<<(n + 3) / 4, 128, 0, ctx->stream>>>(dq, n, sc, dout);
  ++ctx->launches;
  prof_end(ctx, rec, double(n) * 32);
  MQ_CUDA(cudaGetLastError());
  std::vector<uint64_t> h(2 * size_t(n));
  if (h.size() <= kReadWords) {
    MQ_TRY(read_words(ctx, dout, h.size(), h.data()));
  } else {
    uint64_t* dst = h.size() <= kPinnedWords ? ctx->h_pinned : h.data();  // pinned when it fits
    MQ_CUDA(cudaMemcpyAsync(dst, dout, h.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream));
    MQ_CUDA(cudaStreamSynchronize(ctx->stream));
    if (dst != h.data()) memcpy(h.data(), dst, h.size() * sizeof(uint64_t));
  }
  for (uint32_t i = 0; i < n; ++i) {
    out[i].lo = h[2 * i];
    out[i].hi = h[2 * i + 1];
    out[i].kind = q[i].kind;
    out[i].order = q[i].kind == KIND_O_BOUND ? 1 : q[i].kind == KIND_NONE ? -1 : 0;
  }
  return MAPSQ_OK;
}

int scan_emit(Ctx* ctx, const mapsq_pattern& tp, const PatternRange& r, TableImpl** out, int32_t key_var) {
  const Store& st = ctx->store;
  int32_t vars[2];
  uint32_t nv = 0;
  if (tp.var_mask & MAPSQ_VAR_S) vars[nv++] = int32_t(tp.s);
  if ((tp.var_mask & MAPSQ_VAR_O) && !(nv == 1 && vars[0] == int32_t(tp.o))) vars[nv++] = int32_t(tp.o);
  uint64_t rows = r.hi - r.lo;
  TableImpl* t = nullptr;
  switch (r.kind) {
    case KIND_NONE:
      MQ_TRY(table_alloc(ctx, 0, nv, vars, &t));
      break;
    case KIND_EXIST:
      MQ_TRY(table_alloc(ctx, rows, 0, vars, &t));
      break;
    // a run of the store is already the partial-match table: a view, no copy
    // (the run's remaining column is sorted: o within (p, s), s within (p, o))
    case KIND_S_BOUND: {
      uint32_t* cols[1] = {st.so_o + r.lo};
      MQ_TRY(table_view(ctx, rows, 1, vars, cols, st.shared, &t));
      t->pub.sorted_mask = 1u;
      break;
    }
    case KIND_O_BOUND: {
      uint32_t* cols[1] = {st.os_s + r.lo};
      MQ_TRY(table_view(ctx, rows, 1, vars, cols, st.shared, &t));
      t->pub.sorted_mask = 1u;
      break;
    }
    // the predicate's whole segment: the (p, s, o) order is sorted by s, the
    // (p, o, s) order by o; the join key decides which one is returned
    case KIND_TWO_VARS: {
      const bool by_o = key_var >= 0 && key_var == int32_t(tp.o);
      uint32_t* cols[2] = {by_o ? st.os_s + r.lo : st.so_s + r.lo, by_o ? st.os_o + r.lo : st.so_o + r.lo};
      MQ_TRY(table_view(ctx, rows, 2, vars, cols, st.shared, &t));
      t->pub.sorted_mask = by_o ? 2u : 1u;
      break;
    }
    case KIND_SAME_VAR: {
      Scratch scratch(ctx);
      uint32_t* flag = nullptr;
      uint64_t* pos = nullptr;
      MQ_TRY(scratch.get(rows + 1, &flag));
      MQ_TRY(scratch.get(rows + 1, &pos));
      unsigned grid = unsigned(std::max<uint64_t>(1, std::min<uint64_t>(ceil_div(rows, 256), 152ull * 16)));
      if (rows) {
        const int rec = prof_begin(ctx, K_SCAN_FILTER);
        same_var_flags_kernel<<<grid, 256, 0, ctx->stream>>>(st.so_s + r.lo, st.so_o + r.lo, rows, flag);
        ++ctx->launches;
        prof_end(ctx, rec, double(rows) * 12);
      }
      MQ_TRY(prefix_sum_u32_u64(ctx, flag, pos, rows));
      uint64_t m = 0;
      MQ_TRY(read_u64(ctx, pos + rows, &m, 1));
      MQ_TRY(table_alloc(ctx, m, 1, vars, &t));
      if (rows) {
        const int rec = prof_begin(ctx, K_SCAN_FILTER);
        same_var_compact_kernel<<<grid, 256, 0, ctx->stream>>>(st.so_s + r.lo, rows, flag, pos, t->pub.col[0]);
        ++ctx->launches;
        prof_end(ctx, rec, double(rows) * 8 + double(m) * 4);
      }
      MQ_CUDA(cudaGetLastError());
      t->pub.sorted_mask = 1u;  // kept in the (p, s, o) order
      break;
    }
    default:
      return set_error(ctx, MAPSQ_ERR_INVALID, "bad pattern kind %d", r.kind);
  }
  *out = t;
  return MAPSQ_OK;
}

}  // namespace mapsq
