// Searches of sorted columns with few dependent loads.
//
// A count pass that looks each probe key up in a sorted column is bound by the
// latency of its dependent loads, not by bandwidth: a bisection of n positions
// is log2(n) loads one after another.  Here every search advances K-ary: a
// round loads K - 1 evenly spaced pivots of its range at once and keeps the
// part between the last pivot below the target and the first not below, so a
// search takes log_K(n) rounds; the N searches of a thread advance in lockstep,
// so that the loads of one round of all of them are in flight together.
#pragma once

#include <cstdint>

namespace mapsq {

// Lower bounds: search s finds the first position p in [lo[s], lo[s] + len[s]]
// with a[s][p] >= t[s], given that positions before lo[s] hold smaller values
// and positions from lo[s] + len[s] on hold values not smaller (so p may be
// lo[s] + len[s]).  On return lo[s] = p and len[s] = 0.  A search that starts
// with len[s] = 0 loads nothing.
template <int N, int K, class T>
__device__ __forceinline__ void lower_bounds_kary(const T* const (&a)[N], const T (&t)[N], uint64_t (&lo)[N],
                                                  uint64_t (&len)[N]) {
  static_assert(K >= 2, "at least one pivot per round");
  for (;;) {
    bool more = false;
#pragma unroll
    for (int s = 0; s < N; ++s) more |= len[s] != 0;
    if (!more) return;
    T piv[N][K - 1];
#pragma unroll
    for (int s = 0; s < N; ++s)
#pragma unroll
      for (int i = 1; i < K; ++i) piv[s][i - 1] = len[s] ? __ldg(a[s] + lo[s] + len[s] * i / K) : T(0);
#pragma unroll
    for (int s = 0; s < N; ++s) {
      if (!len[s]) continue;
      // the pivots are in position order, so those below the target come first
      int c = 0;
#pragma unroll
      for (int i = 1; i < K; ++i) c += piv[s][i - 1] < t[s];
      const uint64_t hi = c < K - 1 ? lo[s] + len[s] * uint64_t(c + 1) / K : lo[s] + len[s];
      const uint64_t nlo = c ? lo[s] + len[s] * uint64_t(c) / K + 1 : lo[s];
      lo[s] = nlo;
      len[s] = hi - nlo;
    }
  }
}

}  // namespace mapsq
