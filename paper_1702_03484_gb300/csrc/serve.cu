// Serving loop: continuous batching of BGP queries over the resident store.
//
// Queries arrive (mapsq_submit) while others are on the GPU.  A worker thread
// runs rounds: it admits waiting queries while fewer than max_active are in
// flight and the live intermediate tables stay under the memory budget; new
// queries get their range searches in one launch, their order and their first
// scan; then the next join of every query in flight goes into one batched join
// (every phase one launch for all of them), so that the steps of many queries
// share launches and new arrivals join at any round.  Memory admission uses the
// count pass: after the batch's counts, result tables are written in arrival
// order while they fit in the budget; the rest wait for a later round.  When
// no join fits at all, the youngest query in flight is put back in the queue
// (its tables freed) and admissions pause until a join is written, so the
// oldest queries always progress.  A finished query's result waits for
// mapsq_poll; the time from submission to completion (its kernels done) is
// recorded for the latency statistics.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <cstring>
#include <new>
#include <unordered_map>

#include "internal.cuh"

namespace mapsq {

namespace {

using Clock = std::chrono::steady_clock;

struct Query {
  uint64_t ticket = 0;
  std::vector<mapsq_pattern> bgp;
  Clock::time_point submitted;
  std::vector<PatternRange> ranges;
  std::vector<uint32_t> order;
  uint32_t joined = 0;        // patterns in ``acc`` so far
  TableImpl* acc = nullptr;
  int status = MAPSQ_OK;      // first error met
};

struct Done {
  TableImpl* table;
  int status;
};

uint64_t table_bytes(const TableImpl* t) { return t ? t->bytes : 0; }


}  // namespace

struct Server {
  Ctx* ctx = nullptr;
  uint32_t max_active = 256;
  uint64_t budget = 0;        // bytes of intermediate and result tables in flight (0 = unbounded)
  std::thread worker;
  std::mutex mu;              // guards everything below
  std::condition_variable cv;
  std::deque<Query*> arrivals;
  std::vector<Query*> active;    // worker thread only, like the three below
  std::vector<Query*> requeue;   // put back by round(); admitted before new arrivals
  bool hold = false;             // admissions paused until a join is written
  std::unordered_map<uint64_t, Done> done;
  std::vector<double> latency_ms;
  uint64_t next_ticket = 1, submitted = 0, completed = 0, failed = 0, rows = 0;
  std::atomic<uint64_t> rounds{0}, joins{0}, preempted{0};
  bool stopping = false;

  void finish(Query* q) {
    if (q->status == MAPSQ_OK) {
      canonical_columns(&q->acc->pub);
    } else {
      table_release(ctx, q->acc);
      q->acc = nullptr;
    }
    const double ms = std::chrono::duration<double, std::milli>(Clock::now() - q->submitted).count();
    std::lock_guard<std::mutex> lock(mu);
    if (q->status == MAPSQ_OK) {
      rows += q->acc->pub.nrows;
      ++completed;
    } else {
      ++failed;
    }
    done[q->ticket] = Done{q->acc, q->status};
    latency_ms.push_back(ms);
    delete q;
  }

  uint64_t live_bytes() const {
    uint64_t b = 0;
    for (const Query* q : active) b += table_bytes(q->acc);
    return b;
  }

  // New queries: one range search for all their patterns, their order, first scan.
  void start_queries(std::vector<Query*>& fresh) {
    std::vector<mapsq_pattern> all;
    for (Query* q : fresh)
      if (q->ranges.empty()) all.insert(all.end(), q->bgp.begin(), q->bgp.end());
    std::vector<PatternRange> ranges(all.size());
    const int rc = all.empty() ? MAPSQ_OK : scan_ranges(ctx, all.data(), uint32_t(all.size()), ranges.data());
    size_t off = 0;
    for (Query* q : fresh) {
      const uint32_t n = uint32_t(q->bgp.size());
      if (q->ranges.empty()) {  // a query put back in the queue keeps its ranges and order
        if (rc != MAPSQ_OK) {
          q->status = rc;
          finish(q);
          continue;
        }
        q->ranges.assign(ranges.begin() + off, ranges.begin() + off + n);
        q->order = plan_order(q->bgp.data(), n, q->ranges.data());
        off += n;
      }
      q->status = scan_emit(ctx, q->bgp[q->order[0]], q->ranges[q->order[0]], &q->acc);
      if (q->status != MAPSQ_OK) {
        finish(q);
        continue;
      }
      q->joined = 1;
      active.push_back(q);
    }
    fresh.clear();
  }

  // One round: the next join of every query in flight, in one admitted batch.
  void round() {
    std::vector<Query*> who;
    std::vector<TableImpl*> parts;
    std::vector<const mapsq_table*> L, R;
    for (Query* q : active) {
      if (q->joined >= q->bgp.size()) continue;
      const uint32_t pi = q->order[q->joined];
      TableImpl* part = nullptr;
      q->status = scan_emit(ctx, q->bgp[pi], q->ranges[pi], &part, shared_var(q->acc->pub, q->bgp[pi]));
      if (q->status != MAPSQ_OK) continue;
      who.push_back(q);
      parts.push_back(part);
      L.push_back(&q->acc->pub);
      R.push_back(&part->pub);
    }
    const size_t k = who.size();
    std::vector<TableImpl*> out(k, nullptr);
    std::vector<int> st(k, 1);
    std::vector<uint64_t> need(k, 0);
    const uint64_t live = live_bytes();
    const uint64_t room = budget ? (budget > live ? budget - live : 1) : 0;
    const int rc = join_batch_admit(ctx, uint32_t(k), L.data(), R.data(), room, out.data(), st.data(), need.data());
    for (auto* p : parts) table_release(ctx, p);
    bool progress = false;
    for (size_t i = 0; i < k; ++i) {
      Query* q = who[i];
      if (rc != MAPSQ_OK) {
        q->status = rc;
      } else if (st[i] == 0) {
        table_release(ctx, q->acc);
        q->acc = out[i];
        ++q->joined;
        ++joins;
        progress = true;
      } else if (budget && need[i] + table_bytes(q->acc) > budget) {
        q->status = MAPSQ_ERR_BUDGET;  // cannot fit even with every other query gone
      }
    }
    if (progress) {
      hold = false;
    } else if (rc == MAPSQ_OK && k > 1) {
      // nothing fits beside the others: put the youngest back in the queue and
      // pause admissions until a join is written
      Query* y = who[k - 1];
      if (y->status == MAPSQ_OK) {
        table_release(ctx, y->acc);
        y->acc = nullptr;
        y->joined = 0;
        requeue.push_back(y);
        ++preempted;
        hold = true;
      }
    } else if (rc == MAPSQ_OK && k == 1 && who[0]->status == MAPSQ_OK) {
      who[0]->status = MAPSQ_ERR_BUDGET;
    }
    // a query is complete once its result is written: wait for the round's kernels
    // before any query is handed out, so that latency counts them
    bool completes = false;
    for (Query* q : active) completes |= q->status == MAPSQ_OK && q->joined >= q->bgp.size();
    if (completes) {
      const int e = read_words(ctx, nullptr, 0, nullptr);
      if (e != MAPSQ_OK)
        for (Query* q : active) q->status = q->status == MAPSQ_OK ? e : q->status;
    }
    std::vector<Query*> still;
    for (Query* q : active) {
      if (!requeue.empty() && q == requeue.back() && q->acc == nullptr && q->joined == 0) continue;
      if (q->status != MAPSQ_OK || q->joined >= q->bgp.size())
        finish(q);
      else
        still.push_back(q);
    }
    active.swap(still);
  }

  void run() {
    cudaSetDevice(ctx->device);
    std::vector<Query*> fresh;
    for (;;) {
      {
        std::unique_lock<std::mutex> lock(mu);
        cv.wait(lock, [&] { return stopping || !arrivals.empty() || !active.empty() || !requeue.empty(); });
        if (stopping && arrivals.empty() && active.empty() && requeue.empty()) break;
      }
      std::lock_guard<std::recursive_mutex> cl(ctx->mu);
      if (!hold || active.empty()) {
        hold = false;
        const uint64_t live = live_bytes();
        while (!requeue.empty() && active.size() + fresh.size() < max_active && (!budget || live < budget)) {
          fresh.push_back(requeue.front());
          requeue.erase(requeue.begin());
        }
        std::lock_guard<std::mutex> lock(mu);
        while (!arrivals.empty() && active.size() + fresh.size() < max_active && (!budget || live < budget)) {
          fresh.push_back(arrivals.front());
          arrivals.pop_front();
        }
      }
      if (!fresh.empty()) start_queries(fresh);
      if (!active.empty()) round();
      ++rounds;
    }
  }
};

void server_shutdown(Ctx* ctx) {
  Server* s = ctx->server;
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stopping = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  // results never collected stay owned by the context (freed with it)
  ctx->server = nullptr;
  delete s;
}

}  // namespace mapsq

using namespace mapsq;

extern "C" {

int mapsq_serve_start(mapsq_ctx* ctx, const mapsq_serve_opts* opts) {
  if (!ctx) return MAPSQ_ERR_INVALID;
  std::lock_guard<std::recursive_mutex> cl(ctx->mu);
  if (ctx->server) return set_error(ctx, MAPSQ_ERR_BUSY, "the serving loop is already running");
  if (!ctx->store.loaded) return set_error(ctx, MAPSQ_ERR_INVALID, "no triple store loaded");
  Server* s = new (std::nothrow) Server();
  if (!s) return set_error(ctx, MAPSQ_ERR_OOM, "host allocation failed");
  s->ctx = ctx;
  if (opts) {
    if (opts->max_active) s->max_active = opts->max_active;
    s->budget = opts->mem_budget_bytes;
  }
  ctx->server = s;
  s->worker = std::thread([s] { s->run(); });
  return MAPSQ_OK;
}

int mapsq_submit(mapsq_ctx* ctx, const mapsq_pattern* bgp, uint32_t n, uint64_t* ticket) {
  if (!ctx || !bgp || !ticket || n == 0) return MAPSQ_ERR_INVALID;
  Server* s = ctx->server;
  if (!s) return MAPSQ_ERR_BUSY;
  for (uint32_t i = 0; i < n; ++i) {
    // the pattern checks touch no device state
    if (bgp[i].var_mask & MAPSQ_VAR_P) return MAPSQ_ERR_UNSUPPORTED;
    if (bgp[i].var_mask & ~(MAPSQ_VAR_S | MAPSQ_VAR_P | MAPSQ_VAR_O)) return MAPSQ_ERR_INVALID;
    if (((bgp[i].var_mask & MAPSQ_VAR_S) && bgp[i].s >= MAPSQ_MAX_VARS) ||
        ((bgp[i].var_mask & MAPSQ_VAR_O) && bgp[i].o >= MAPSQ_MAX_VARS))
      return MAPSQ_ERR_INVALID;
  }
  Query* q = new (std::nothrow) Query();
  if (!q) return MAPSQ_ERR_OOM;
  q->bgp.assign(bgp, bgp + n);
  q->submitted = Clock::now();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stopping) {
      delete q;
      return MAPSQ_ERR_BUSY;
    }
    q->ticket = s->next_ticket++;
    ++s->submitted;
    s->arrivals.push_back(q);
    *ticket = q->ticket;
  }
  s->cv.notify_one();
  return MAPSQ_OK;
}

int mapsq_poll(mapsq_ctx* ctx, uint64_t ticket, mapsq_table** out) {
  if (!ctx || !out) return MAPSQ_ERR_INVALID;
  Server* s = ctx->server;
  if (!s) return MAPSQ_ERR_BUSY;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->done.find(ticket);
  if (it == s->done.end()) {
    if (ticket == 0 || ticket >= s->next_ticket) return MAPSQ_ERR_NOT_FOUND;
    *out = nullptr;  // still running (or already collected: then never returned again)
    return MAPSQ_OK;
  }
  const Done d = it->second;
  s->done.erase(it);
  *out = d.table ? &d.table->pub : nullptr;
  return d.status;
}

int mapsq_serve_stats(mapsq_ctx* ctx, mapsq_serve_counters* out) {
  if (!ctx || !out) return MAPSQ_ERR_INVALID;
  Server* s = ctx->server;
  if (!s) return MAPSQ_ERR_BUSY;
  std::vector<double> lat;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->rounds = s->rounds;
    out->batched_joins = s->joins;
    out->result_rows = s->rows;
    out->in_flight = s->submitted - s->completed - s->failed;
    out->preempted = s->preempted;
    lat = s->latency_ms;
  }
  if (!lat.empty()) {
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double p) { return lat[std::min(lat.size() - 1, size_t(p * (lat.size() - 1) + 0.5))]; };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    double sum = 0;
    for (double v : lat) sum += v;
    out->mean_ms = sum / lat.size();
  }
  return MAPSQ_OK;
}

int mapsq_serve_stop(mapsq_ctx* ctx) {
  if (!ctx) return MAPSQ_ERR_INVALID;
  if (!ctx->server) return MAPSQ_ERR_BUSY;
  server_shutdown(ctx);
  return MAPSQ_OK;
}

}  // extern "C"
