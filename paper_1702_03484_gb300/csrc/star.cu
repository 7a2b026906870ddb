// Multi-way join of k tables that share exactly one variable (the partial
// matches of a star of triple patterns around that variable) in one round:
// the key/value framing of Section 1 and Algorithm 1 with k inputs instead of
// two.  The map keys every row by the shared variable; the shuffle is the
// inputs' own order (every table but the driving one is sorted on the key,
// as the store's runs are); the reduce emits, for every key, every
// combination of one row from each table.
//
// A thread per row of the driving table (the smallest, or the one not
// sorted) finds its key's run in every other table (the run's two ends
// searched together: K-ary rounds in a launch of few CTAs, where the latency
// of dependent loads decides, bisection in a larger one, where their number
// does) and counts the product of the run lengths; a prefix sum of the counts
// gives each driving row its output range (one synchronisation reads the
// total); the write kernel gives each thread
// four consecutive output rows, finds their driving row once and decodes each
// row's position inside its range as a mixed-radix number whose digits index
// the other tables' runs (the last table varies fastest).  Output columns: the
// key, then every table's other columns in table order.  Tables that are not
// sorted on the key (more than the driving one) are joined pairwise instead
// (Algorithm 1, one table at a time), which gives the same rows.
#include <algorithm>
#include <vector>

#include "internal.cuh"
#include "search.cuh"

namespace mapsq {

namespace {

constexpr int kMaxStar = 8;
constexpr int kStarThreads = 256;
constexpr int kStarRowsPerThread = 4;
constexpr int kStarWays = 8;               // pivots per search round + 1 in a latency-bound launch
constexpr unsigned kStarKaryMaxBlocks = 152;  // launches of up to this many CTAs search K-ary, larger ones bisect

struct StarDesc {
  int k;                                // tables; table 0 drives
  const uint32_t* key[kMaxStar];        // key column of each table
  uint64_t n[kMaxStar];                 // rows of each table
  int ncols;                            // output columns
  const uint32_t* src[MAPSQ_MAX_VARS];  // column of table tab[c] that output column c copies
  int tab[MAPSQ_MAX_VARS];
  uint32_t* out[MAPSQ_MAX_VARS];
  uint32_t* lo;                         // (k - 1) x n[0]: first row of driving row i's run in table j
  uint32_t* len;                        // (k - 1) x n[0]: the run's length
  uint32_t* cnt;                        // n[0]: output rows of driving row i
  const uint64_t* off;                  // n[0] + 1: exclusive prefix sums of cnt
  uint64_t T;
  uint32_t* check;                      // status word of the checked build's bounds checks
};

template <int W>
__global__ void __launch_bounds__(kStarThreads) star_count_kernel(StarDesc d, uint64_t* __restrict__ status) {
  const uint64_t n0 = d.n[0], stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n0; i += stride) {
    const uint32_t x = __ldg(d.key[0] + i);
    uint64_t c = 1;
    for (int j = 1; j < d.k; ++j) {
      // the run of x in table j: first position >= x and first position > x, searched together
      const uint32_t* arr[2] = {d.key[j], d.key[j]};
      const uint32_t tgt[2] = {x, x + 1u};
      uint64_t lo[2] = {0, x == 0xffffffffu ? d.n[j] : 0};
      uint64_t len[2] = {d.n[j], x == 0xffffffffu ? 0 : d.n[j]};
      lower_bounds_kary<2, W>(arr, tgt, lo, len);
      d.lo[(j - 1) * n0 + i] = uint32_t(lo[0]);
      d.len[(j - 1) * n0 + i] = uint32_t(lo[1] - lo[0]);
      c *= lo[1] - lo[0];
      if (c == 0) break;
      if (c > 0xffffffffull) {  // one key's product of runs beyond 2^32 rows
        atomicOr(reinterpret_cast<unsigned long long*>(status), 1ull);
        c = 0;
        break;
      }
    }
    d.cnt[i] = uint32_t(c);
  }
}

template <int W>
__global__ void __launch_bounds__(kStarThreads) star_write_kernel(StarDesc d) {
  const uint64_t n0 = d.n[0];
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x * kStarRowsPerThread;
  for (uint64_t t0 = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) * kStarRowsPerThread; t0 < d.T; t0 += stride) {
    // the driving row whose output range holds t0: last i with off[i] <= t0,
    // one before the first i with off[i] > t0 (off[0] = 0 <= t0, off[n0] = T > t0)
    const uint64_t* arr[1] = {d.off};
    const uint64_t tgt[1] = {t0 + 1};
    uint64_t lo[1] = {1}, len[1] = {n0 - 1};
    lower_bounds_kary<1, W>(arr, tgt, lo, len);
    uint64_t i = lo[0] - 1;
    const uint64_t tend = min(t0 + kStarRowsPerThread, d.T);
    for (uint64_t t = t0; t < tend; ++t) {
      while (d.off[i + 1] <= t) ++i;  // rows without output are skipped
      uint64_t r = t - d.off[i];
      uint64_t row[kMaxStar];
      row[0] = i;
      for (int j = d.k - 1; j >= 1; --j) {
        const uint32_t L = d.len[(j - 1) * n0 + i];
        row[j] = d.lo[(j - 1) * n0 + i] + r % L;
        r /= L;
      }
      bool ok = true;
      for (int j = 0; j < d.k; ++j) ok = ok && MQ_IN_BOUNDS(row[j] < d.n[j], d.check);
      if (!ok) continue;
      for (int c = 0; c < d.ncols; ++c) d.out[c][t] = __ldg(d.src[c] + row[d.tab[c]]);
    }
  }
}

unsigned star_grid(uint64_t n, uint64_t per_thread) {
  return unsigned(std::max<uint64_t>(1, std::min<uint64_t>(ceil_div(std::max<uint64_t>(n, 1), kStarThreads * per_thread),
                                                           152ull * 16)));
}

int find_col(const mapsq_table* t, int32_t v) {
  for (uint32_t c = 0; c < t->ncols; ++c)
    if (t->var[c] == v) return int(c);
  return -1;
}

}  // namespace

int join_star(Ctx* ctx, uint32_t k, const mapsq_table* const* tabs, int32_t key_var, TableImpl** out) {
  if (k < 2 || k > uint32_t(kMaxStar)) return set_error(ctx, MAPSQ_ERR_INVALID, "star of %u tables (2 to %d)", k, kMaxStar);
  if (key_var < 0 || key_var >= MAPSQ_MAX_VARS) return set_error(ctx, MAPSQ_ERR_INVALID, "key variable %d", key_var);
  // layout: the key, then every table's other columns in table order
  int32_t vars[MAPSQ_MAX_VARS];
  int ncols = 1;
  vars[0] = key_var;
  uint32_t seen = 1u << key_var;
  for (uint32_t j = 0; j < k; ++j) {
    const mapsq_table* t = tabs[j];
    if (!t) return set_error(ctx, MAPSQ_ERR_INVALID, "NULL table %u", j);
    if (t->ncols > MAPSQ_MAX_VARS || (t->ncols && t->nrows && !t->on_device))
      return set_error(ctx, MAPSQ_ERR_INVALID, "table %u: bad columns", j);
    if (find_col(t, key_var) < 0) return set_error(ctx, MAPSQ_ERR_INVALID, "table %u lacks variable %d", j, key_var);
    for (uint32_t c = 0; c < t->ncols; ++c) {
      const int32_t v = t->var[c];
      if (v < 0 || v >= MAPSQ_MAX_VARS) return set_error(ctx, MAPSQ_ERR_INVALID, "table %u: variable id %d", j, v);
      if (t->nrows && (!t->col[c] || (reinterpret_cast<uintptr_t>(t->col[c]) & 3)))
        return set_error(ctx, MAPSQ_ERR_INVALID, "table %u: column %u is NULL or not 4-byte aligned", j, c);
      if (v == key_var) continue;
      if (seen & (1u << v))
        return set_error(ctx, MAPSQ_ERR_INVALID, "variable %d appears twice (a star shares only its key)", v);
      seen |= 1u << v;
      if (ncols == MAPSQ_MAX_VARS) return set_error(ctx, MAPSQ_ERR_INVALID, "more than %d result columns", MAPSQ_MAX_VARS);
      vars[ncols++] = v;
    }
  }
  // the driving table: the only one not sorted on the key, else the smallest
  int unsorted = 0, driver = 0;
  for (uint32_t j = 0; j < k; ++j) {
    const bool sorted = (tabs[j]->sorted_mask >> find_col(tabs[j], key_var)) & 1u;
    if (!sorted) {
      ++unsorted;
      driver = int(j);
    }
  }
  if (unsorted == 0)
    for (uint32_t j = 1; j < k; ++j)
      if (tabs[j]->nrows < tabs[driver]->nrows) driver = int(j);
  if (unsorted > 1) {
    // pairwise joins, Algorithm 1 one table at a time: the layout comes out the same
    TableImpl* acc = nullptr;
    const mapsq_table* a = tabs[0];
    for (uint32_t j = 1; j < k; ++j) {
      TableImpl* next = nullptr;
      const int rc = join_tables(ctx, a, tabs[j], nullptr, &next);
      table_release(ctx, acc);
      if (rc != MAPSQ_OK) return rc;
      acc = next;
      a = &acc->pub;
    }
    *out = acc;
    return MAPSQ_OK;
  }
  StarDesc d{};
  d.k = int(k);
  d.check = ctx->d_status;
  std::vector<int> order;  // table of each StarDesc slot
  order.push_back(driver);
  for (uint32_t j = 0; j < k; ++j)
    if (int(j) != driver) order.push_back(int(j));
  uint64_t n0 = 0;
  bool empty = false;
  for (uint32_t s = 0; s < k; ++s) {
    const mapsq_table* t = tabs[order[s]];
    d.key[s] = t->col[find_col(t, key_var)];
    d.n[s] = t->nrows;
    empty |= t->nrows == 0;
  }
  n0 = d.n[0];
  d.ncols = ncols;
  d.src[0] = d.key[0];
  d.tab[0] = 0;
  {
    int c = 1;
    for (uint32_t j = 0; j < k; ++j) {
      const int slot = int(std::find(order.begin(), order.end(), int(j)) - order.begin());
      for (uint32_t q = 0; q < tabs[j]->ncols; ++q) {
        if (tabs[j]->var[q] == key_var) continue;
        d.src[c] = tabs[j]->col[q];
        d.tab[c] = slot;
        ++c;
      }
    }
  }
  if (empty) return table_alloc(ctx, 0, uint32_t(ncols), vars, out);
  for (uint32_t s = 1; s < k; ++s)
    if (d.n[s] > 0xffffffffull) return set_error(ctx, MAPSQ_ERR_UNSUPPORTED, "a star table of 2^32 rows or more");
  Scratch scratch(ctx);
  uint64_t* off = nullptr;
  MQ_TRY(scratch.get(size_t(k - 1) * n0, &d.lo));
  MQ_TRY(scratch.get(size_t(k - 1) * n0, &d.len));
  MQ_TRY(scratch.get(n0, &d.cnt));
  MQ_TRY(scratch.get(n0 + 2, &off));  // offsets, total, then the status word
  d.off = off;
  MQ_CUDA(cudaMemsetAsync(off + n0 + 1, 0, sizeof(uint64_t), ctx->stream));
  int rec = prof_begin(ctx, K_STAR_COUNT);
  const unsigned gc = star_grid(n0, 1);
  if (gc <= kStarKaryMaxBlocks)
    star_count_kernel<kStarWays><<<gc, kStarThreads, 0, ctx->stream>>>(d, off + n0 + 1);
  else
    star_count_kernel<2><<<gc, kStarThreads, 0, ctx->stream>>>(d, off + n0 + 1);
  ++ctx->launches;
  prof_end(ctx, rec, 4.0 * n0);
  MQ_CUDA(cudaGetLastError());
  MQ_TRY(prefix_sum_u32_u64(ctx, d.cnt, off, n0));
  uint64_t tail[2] = {0, 0};
  MQ_TRY(read_u64(ctx, off + n0, tail, 2));  // one synchronisation: the row count and the status
  if (tail[1]) return set_error(ctx, MAPSQ_ERR_UNSUPPORTED, "a key whose star product exceeds 2^32 rows");
  d.T = tail[0];
  TableImpl* t = nullptr;
  MQ_TRY(table_alloc(ctx, d.T, uint32_t(ncols), vars, &t));
  for (int c = 0; c < ncols; ++c) d.out[c] = t->pub.col[c];
  if (d.T) {
    double bytes = 4.0 * double(d.T) * ncols;
    for (uint32_t s = 0; s < k; ++s) bytes += 4.0 * double(d.n[s]);
    rec = prof_begin(ctx, K_STAR_WRITE);
    const unsigned gw = star_grid(d.T, kStarRowsPerThread);
    if (gw <= kStarKaryMaxBlocks)
      star_write_kernel<kStarWays><<<gw, kStarThreads, 0, ctx->stream>>>(d);
    else
      star_write_kernel<2><<<gw, kStarThreads, 0, ctx->stream>>>(d);
    ++ctx->launches;
    prof_end(ctx, rec, bytes);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      table_release(ctx, t);
      return cuda_fail(ctx, e, "star_write_kernel", __FILE__, __LINE__);
    }
  }
  const int rc = checked_sync(ctx);
  if (rc != MAPSQ_OK) {
    table_release(ctx, t);
    return rc;
  }
  *out = t;
  return MAPSQ_OK;
}

}  // namespace mapsq

using namespace mapsq;

extern "C" int mapsq_join_star(mapsq_ctx* ctx, uint32_t k, const mapsq_table* const* tables, int32_t key_var,
                               mapsq_table** out) {
  if (!ctx || !tables || !out) return ctx ? set_error(ctx, MAPSQ_ERR_INVALID, "NULL argument") : MAPSQ_ERR_INVALID;
  if (ctx->server) return set_error(ctx, MAPSQ_ERR_BUSY, "the serving loop is running");
  MQ_CUDA(cudaSetDevice(ctx->device));
  TableImpl* t = nullptr;
  MQ_TRY(join_star(ctx, k, tables, key_var, &t));
  *out = &t->pub;
  return MAPSQ_OK;
}
