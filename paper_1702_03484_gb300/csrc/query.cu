// BGP evaluation, the host side of the paper's CPU/GPU coprocessing split
// (Section 2): the host orders each BGP's patterns and drives the device's
// pattern scans and joins, one pattern at a time, joining the partial results
// after each match.  Each scan result is a view of the store sorted on the
// variable it will be joined on, so the join may search it instead of hashing.
// Many BGPs are evaluated together: their range searches are one launch, and
// at every level each query's next join goes into one batched join (every
// phase one launch for all of them).
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace mapsq {

namespace {

uint32_t pattern_var_set(const mapsq_pattern& tp) {
  uint32_t m = 0;
  if (tp.var_mask & MAPSQ_VAR_S) m |= 1u << tp.s;
  if (tp.var_mask & MAPSQ_VAR_O) m |= 1u << tp.o;
  return m;
}

}  // namespace

// The centre of a star BGP of 3 to 8 patterns: the one variable that every
// pattern holds, with no other variable in two patterns; -1 otherwise.
int32_t star_centre(const mapsq_pattern* bgp, uint32_t n) {
  if (n < 3 || n > 8) return -1;
  uint32_t common = ~0u, all = 0, twice = 0;
  for (uint32_t i = 0; i < n; ++i) {
    const uint32_t m = pattern_var_set(bgp[i]);
    if (!m) return -1;
    common &= m;
    twice |= all & m;
    all |= m;
  }
  if (__builtin_popcount(common) != 1 || twice != common) return -1;
  return __builtin_ctz(common);
}

// Permute the columns of a result so that its variables are in ascending id
// (a pointer permutation: no data moves; the sorted-column bits follow).
void canonical_columns(mapsq_table* t) {
  const uint32_t n = t->ncols;
  for (uint32_t i = 1; i < n; ++i)
    for (uint32_t j = i; j > 0 && t->var[j - 1] > t->var[j]; --j) {
      std::swap(t->var[j - 1], t->var[j]);
      std::swap(t->col[j - 1], t->col[j]);
      const uint32_t a = (t->sorted_mask >> (j - 1)) & 1u, b = (t->sorted_mask >> j) & 1u;
      t->sorted_mask = (t->sorted_mask & ~(3u << (j - 1))) | (b << (j - 1)) | (a << j);
    }
}

// The one variable that table t shares with pattern tp, or -1 (none, or two):
// the variable a scan result will be joined on, so that it can be returned
// sorted by it.
int32_t shared_var(const mapsq_table& t, const mapsq_pattern& tp) {
  int32_t found = -1;
  int n = 0;
  for (uint32_t c = 0; c < t.ncols; ++c) {
    const int32_t v = t.var[c];
    if (((tp.var_mask & MAPSQ_VAR_S) && int32_t(tp.s) == v) || ((tp.var_mask & MAPSQ_VAR_O) && int32_t(tp.o) == v)) {
      found = v;
      ++n;
    }
  }
  return n == 1 ? found : -1;
}

// Greedy order: the pattern with the fewest matches first, then repeatedly the
// one with the fewest matches among those sharing a variable with the patterns
// already taken (any pattern when none does).
std::vector<uint32_t> plan_order(const mapsq_pattern* bgp, uint32_t n, const PatternRange* ranges) {
  std::vector<uint32_t> rest(n), order;
  for (uint32_t i = 0; i < n; ++i) rest[i] = i;
  auto size_of = [&](uint32_t i) { return ranges[i].hi - ranges[i].lo; };
  std::stable_sort(rest.begin(), rest.end(), [&](uint32_t a, uint32_t b) { return size_of(a) < size_of(b); });
  order.push_back(rest.front());
  rest.erase(rest.begin());
  uint32_t seen = pattern_var_set(bgp[order[0]]);
  while (!rest.empty()) {
    auto it = std::find_if(rest.begin(), rest.end(), [&](uint32_t i) { return (pattern_var_set(bgp[i]) & seen) != 0; });
    if (it == rest.end()) it = rest.begin();
    order.push_back(*it);
    seen |= pattern_var_set(bgp[*it]);
    rest.erase(it);
  }
  return order;
}

int query_batch(Ctx* ctx, uint32_t nq, const mapsq_pattern* const* bgps, const uint32_t* ns, TableImpl** out) {
  // one range search for every pattern of every query
  std::vector<mapsq_pattern> all;
  std::vector<size_t> off(nq + 1, 0);
  for (uint32_t q = 0; q < nq; ++q) {
    if (!bgps[q] || ns[q] == 0) return set_error(ctx, MAPSQ_ERR_INVALID, "NULL or empty BGP %u", q);
    for (uint32_t i = 0; i < ns[q]; ++i) MQ_TRY(validate_pattern(ctx, bgps[q][i]));
    all.insert(all.end(), bgps[q], bgps[q] + ns[q]);
    off[q + 1] = all.size();
  }
  if (!ctx->store.loaded) return set_error(ctx, MAPSQ_ERR_INVALID, "no triple store loaded");
  std::vector<PatternRange> ranges(all.size());
  MQ_TRY(scan_ranges(ctx, all.data(), uint32_t(all.size()), ranges.data()));

  // A pattern without variables only asks whether its triple is in the
  // graph, and its range answers: present, it leaves the query (joining a
  // one-row table without columns changes nothing); absent, the query has no
  // solution.  A query of such patterns alone keeps them (one row, or none,
  // without columns).
  std::vector<std::vector<mapsq_pattern>> qb(nq);
  std::vector<std::vector<PatternRange>> qr(nq);
  std::vector<char> none(nq, 0);
  for (uint32_t q = 0; q < nq; ++q) {
    bool any_var = false;
    for (uint32_t i = 0; i < ns[q]; ++i) any_var |= ranges[off[q] + i].kind != KIND_EXIST;
    for (uint32_t i = 0; i < ns[q]; ++i) {
      const PatternRange& r = ranges[off[q] + i];
      if (any_var && r.kind == KIND_EXIST) {
        none[q] |= r.hi == r.lo;
        continue;
      }
      qb[q].push_back(bgps[q][i]);
      qr[q].push_back(r);
    }
  }
  // an empty result with every variable of the query, in ascending id
  auto empty_result = [&](uint32_t q, TableImpl** t) {
    uint32_t vs = 0;
    for (uint32_t i = 0; i < ns[q]; ++i) vs |= pattern_var_set(bgps[q][i]);
    int32_t vars[MAPSQ_MAX_VARS];
    uint32_t nv = 0;
    for (int v = 0; v < 32 && nv < MAPSQ_MAX_VARS; ++v)
      if ((vs >> v) & 1u) vars[nv++] = v;
    return table_alloc(ctx, 0, nv, vars, t);
  };

  // one query that is a star: its patterns' matches, each sorted on the
  // centre, joined in one round
  const int32_t centre = nq == 1 && !none[0] ? star_centre(qb[0].data(), uint32_t(qb[0].size())) : -1;
  if (centre >= 0) {
    const uint32_t n = uint32_t(qb[0].size());
    std::vector<TableImpl*> parts(n, nullptr);
    int rc = MAPSQ_OK;
    for (uint32_t i = 0; i < n && rc == MAPSQ_OK; ++i) rc = scan_emit(ctx, qb[0][i], qr[0][i], &parts[i], centre);
    TableImpl* res = nullptr;
    if (rc == MAPSQ_OK) {
      std::vector<const mapsq_table*> tabs;
      for (auto* p : parts) tabs.push_back(&p->pub);
      rc = join_star(ctx, n, tabs.data(), centre, &res);
    }
    for (auto* p : parts) table_release(ctx, p);
    if (rc != MAPSQ_OK) return rc;
    canonical_columns(&res->pub);
    out[0] = res;
    return MAPSQ_OK;
  }

  std::vector<std::vector<uint32_t>> order(nq);
  std::vector<TableImpl*> acc(nq, nullptr);
  auto release_all = [&]() {
    for (auto*& a : acc) {
      table_release(ctx, a);
      a = nullptr;
    }
  };
  uint32_t levels = 0;
  for (uint32_t q = 0; q < nq; ++q) {
    const int rc = none[q] ? empty_result(q, &acc[q]) : MAPSQ_OK;
    if (rc != MAPSQ_OK) {
      release_all();
      return rc;
    }
    if (none[q]) continue;
    const uint32_t n = uint32_t(qb[q].size());
    order[q] = plan_order(qb[q].data(), n, qr[q].data());
    const uint32_t first = order[q][0];
    const int rc2 = scan_emit(ctx, qb[q][first], qr[q][first], &acc[q]);
    if (rc2 != MAPSQ_OK) {
      release_all();
      return rc2;
    }
    levels = std::max(levels, n - 1);
  }
  // level l: the (l+1)-th pattern of every query that has one, joined in one batch
  for (uint32_t l = 1; l <= levels; ++l) {
    std::vector<uint32_t> who;
    std::vector<TableImpl*> parts;
    std::vector<const mapsq_table*> L, R;
    int rc = MAPSQ_OK;
    for (uint32_t q = 0; q < nq && rc == MAPSQ_OK; ++q) {
      if (none[q] || l >= qb[q].size()) continue;
      const uint32_t pi = order[q][l];
      TableImpl* part = nullptr;
      rc = scan_emit(ctx, qb[q][pi], qr[q][pi], &part, shared_var(acc[q]->pub, qb[q][pi]));
      if (rc != MAPSQ_OK) break;
      who.push_back(q);
      parts.push_back(part);
      L.push_back(&acc[q]->pub);
      R.push_back(&part->pub);
    }
    std::vector<TableImpl*> joined(who.size(), nullptr);
    if (rc == MAPSQ_OK) rc = join_batch(ctx, uint32_t(who.size()), L.data(), R.data(), nullptr, joined.data());
    for (auto* p : parts) table_release(ctx, p);
    if (rc != MAPSQ_OK) {
      release_all();
      return rc;
    }
    for (size_t i = 0; i < who.size(); ++i) {
      table_release(ctx, acc[who[i]]);
      acc[who[i]] = joined[i];
    }
  }
  for (uint32_t q = 0; q < nq; ++q) {
    canonical_columns(&acc[q]->pub);
    out[q] = acc[q];
  }
  return MAPSQ_OK;
}

}  // namespace mapsq

using namespace mapsq;

extern "C" {

int mapsq_query(mapsq_ctx* ctx, const mapsq_pattern* bgp, uint32_t n, mapsq_table** out) {
  if (!ctx || !bgp || !out || n == 0)
    return ctx ? set_error(ctx, MAPSQ_ERR_INVALID, "NULL argument or empty BGP") : MAPSQ_ERR_INVALID;
  if (ctx->server) return set_error(ctx, MAPSQ_ERR_BUSY, "the serving loop is running");
  MQ_CUDA(cudaSetDevice(ctx->device));
  TableImpl* t = nullptr;
  MQ_TRY(query_batch(ctx, 1, &bgp, &n, &t));
  *out = &t->pub;
  return MAPSQ_OK;
}

int mapsq_query_batch(mapsq_ctx* ctx, uint32_t nq, const mapsq_pattern* const* bgps, const uint32_t* n,
                      mapsq_table** out) {
  if (!ctx || (nq && (!bgps || !n || !out)))
    return ctx ? set_error(ctx, MAPSQ_ERR_INVALID, "NULL argument") : MAPSQ_ERR_INVALID;
  if (ctx->server) return set_error(ctx, MAPSQ_ERR_BUSY, "the serving loop is running");
  if (nq == 0) return MAPSQ_OK;
  MQ_CUDA(cudaSetDevice(ctx->device));
  std::vector<TableImpl*> t(nq, nullptr);
  MQ_TRY(query_batch(ctx, nq, bgps, n, t.data()));
  for (uint32_t q = 0; q < nq; ++q) out[q] = &t[q]->pub;
  return MAPSQ_OK;
}

}  // extern "C"
