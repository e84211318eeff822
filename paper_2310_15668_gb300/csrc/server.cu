// Request serving with continuous batching: a server keeps n_slots worker
// threads, each with its own context and CUDA stream; requests (exact
// count, sampled count or characteristic profile of a hypergraph) wait in a
// queue and are admitted, in arrival order, as soon as a slot is free and
// their estimated device memory fits the budget beside the requests already
// running.  Requests that arrive while others run are admitted as slots and
// memory free up, and their work overlaps on the device through the slots'
// streams.  Every request runs the same library calls as a direct caller
// would (mochy_load, mochy_project, then mochy_count_exact,
// mochy_count_sampled or mochy_profile) on a context of its own, so its
// result does not depend on what else is running.  A MoCHy-A+ request
// whose line graph would take more than a quarter of the budget is run
// without it (mochy_count_sampled_onthefly: same draws, same counts).
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "common.cuh"

namespace mochy {

int64_t estimate_graph_bytes(int64_t n_nodes, int64_t n_edges, const int64_t* off,
                             const int32_t* nodes);   // batch.cu
void release_scratch(mochy_ctx* ctx);                 // api.cu

namespace {

// a queued request is overtaken by at most this many later ones
constexpr int32_t kMaxBypass = 32;

struct Request {
  int64_t ticket = 0;
  int32_t kind = 0;
  int64_t n_nodes = 0;
  std::vector<int64_t> off;
  std::vector<int32_t> nodes;
  int32_t method = MOCHY_A_PLUS;
  int64_t samples = 0;
  int32_t n_random = 0;
  uint64_t seed = 0;
  int64_t est = 0;
  int32_t bypassed = 0;      // later requests admitted while this one waited
  bool onthefly = false;     // MoCHy-A+ without the line graph
  int64_t otf_budget = 0;    // its bitmap budget, bytes
  double t_submit = 0.0;
};

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  // nearest rank
  size_t k = (size_t)std::ceil(q * (double)v.size());
  if (k < 1) k = 1;
  if (k > v.size()) k = v.size();
  return v[k - 1];
}

}  // namespace
}  // namespace mochy

struct mochy_server {
  mochy_config cfg;
  int64_t budget = 0;
  int32_t max_queue = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::unique_ptr<mochy::Request>> pending;
  std::unordered_map<int64_t, std::unique_ptr<mochy_result>> done;
  int64_t next_ticket = 1;
  int64_t reserved = 0, peak_reserved = 0;
  int64_t in_flight = 0, peak_in_flight = 0;
  int64_t submitted = 0, completed = 0, failed = 0, rejected = 0;
  bool stop = false;
  int setup_rc = 0;
  std::vector<std::thread> workers;
  std::vector<double> latency_ms;
  double first_submit = -1.0, last_done = 0.0;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

  double now_ms() const {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace mochy {
namespace {

void run_request(mochy_ctx* ctx, const Request& r, mochy_result& out) {
  int rc = mochy_load(ctx, r.n_nodes, (int64_t)r.off.size() - 1, r.off.data(),
                      r.nodes.empty() ? nullptr : r.nodes.data(), nullptr);
  if (rc >= 0 && r.onthefly) {
    // same draws and counts as the projected call, without the line graph
    rc = mochy_count_sampled_onthefly(ctx, r.samples, r.seed, r.otf_budget, out.counts_h,
                                      out.counts_3h, out.est_h, out.est_3h, &out.n_wedges);
    out.status = rc;
    if (rc < 0) snprintf(out.error, sizeof(out.error), "%s", mochy_last_error());
    release_graph(ctx);
    release_scratch(ctx);
    return;
  }
  if (rc >= 0) rc = mochy_project(ctx, &out.n_wedges, nullptr);
  if (rc >= 0) {
    switch (r.kind) {
      case MOCHY_REQ_EXACT:
        rc = mochy_count_exact(ctx, out.counts_h, out.counts_3h);
        break;
      case MOCHY_REQ_SAMPLED:
        rc = mochy_count_sampled(ctx, r.method, r.samples, r.seed, out.counts_h, out.counts_3h,
                                 out.est_h, out.est_3h);
        break;
      case MOCHY_REQ_PROFILE: {
        std::vector<int64_t> ch((size_t)(r.n_random + 1) * MOCHY_N_H);
        std::vector<int64_t> c3((size_t)(r.n_random + 1) * MOCHY_N_3H);
        rc = mochy_profile(ctx, r.n_random, r.seed, out.sig_h, out.cp_h, out.sig_3h, out.cp_3h,
                           ch.data(), c3.data());
        if (rc >= 0) {
          memcpy(out.counts_h, ch.data(), MOCHY_N_H * 8);
          memcpy(out.counts_3h, c3.data(), MOCHY_N_3H * 8);
        }
        break;
      }
      default:
        rc = fail(MOCHY_E_INVALID, "unknown request kind");
    }
  }
  out.status = rc;
  if (rc < 0) snprintf(out.error, sizeof(out.error), "%s", mochy_last_error());
  // give the memory back before the next request is admitted
  release_graph(ctx);
  release_scratch(ctx);
}

void worker_main(mochy_server* s) {
  mochy_ctx* ctx = nullptr;
  mochy_config cfg = s->cfg;
  cfg.stream = nullptr;          // a stream of its own per slot
  cfg.hbm_budget_bytes = 0;      // admission is done by the server
  const int rc0 = mochy_create(&ctx, &cfg);
  if (rc0 < 0) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->setup_rc = rc0;
    s->cv_done.notify_all();
    return;
  }
  for (;;) {
    std::unique_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      auto fits = [&]() -> std::deque<std::unique_ptr<Request>>::iterator {
        // first request in arrival order that fits beside the running ones
        // (a request alone always fits: larger ones are refused at submit);
        // once the oldest one has been overtaken kMaxBypass times, nothing
        // overtakes it any more: the others wait until it fits
        for (auto it = s->pending.begin(); it != s->pending.end(); ++it) {
          if (s->in_flight == 0 || s->reserved + (*it)->est <= s->budget) return it;
          if (it == s->pending.begin() && (*it)->bypassed >= kMaxBypass) break;
        }
        return s->pending.end();
      };
      s->cv_work.wait(lk, [&] { return s->stop || fits() != s->pending.end(); });
      if (s->stop) break;
      auto it = fits();
      if (it != s->pending.begin()) s->pending.front()->bypassed += 1;
      r = std::move(*it);
      s->pending.erase(it);
      s->reserved += r->est;
      s->peak_reserved = std::max(s->peak_reserved, s->reserved);
      s->in_flight += 1;
      s->peak_in_flight = std::max(s->peak_in_flight, s->in_flight);
    }
    auto res = std::make_unique<mochy_result>();
    memset(res.get(), 0, sizeof(mochy_result));
    const double t_start = s->now_ms();
    run_request(ctx, *r, *res);
    const double t_end = s->now_ms();
    res->queue_ms = t_start - r->t_submit;
    res->service_ms = t_end - t_start;
    res->latency_ms = t_end - r->t_submit;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->reserved -= r->est;
      s->in_flight -= 1;
      if (res->status >= 0) {
        s->completed += 1;
        s->latency_ms.push_back(res->latency_ms);
        s->last_done = std::max(s->last_done, t_end);
      } else {
        s->failed += 1;
      }
      s->done[r->ticket] = std::move(res);
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
  mochy_destroy(ctx);
}

}  // namespace
}  // namespace mochy

using namespace mochy;

extern "C" {

int mochy_server_create(mochy_server** out, const mochy_config* cfg, int32_t n_slots,
                        int32_t max_queue) {
  if (!out) return fail(MOCHY_E_INVALID, "null output handle");
  *out = nullptr;
  if (n_slots < 1 || n_slots > 64) return fail(MOCHY_E_INVALID, "n_slots must be in 1..64");
  if (max_queue < 1) return fail(MOCHY_E_INVALID, "max_queue must be positive");
  auto* s = new (std::nothrow) mochy_server();
  if (!s) return fail(MOCHY_E_NOMEM, "host allocation failed");
  mochy_config_default(&s->cfg);
  if (cfg) s->cfg = *cfg;
  s->max_queue = max_queue;
  s->budget = s->cfg.hbm_budget_bytes;
  if (s->budget <= 0) {
    size_t fr = 0, tot = 0;
    if (cudaSetDevice(s->cfg.device) != cudaSuccess || cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      delete s;
      return fail(MOCHY_E_CUDA, "cannot query device memory");
    }
    s->budget = (int64_t)((double)fr * 0.7);
  }
  for (int32_t i = 0; i < n_slots; ++i) s->workers.emplace_back(worker_main, s);
  *out = s;
  return MOCHY_OK;
}

int mochy_server_submit(mochy_server* s, const mochy_request* req, int64_t* ticket) {
  if (!s || !req || !ticket) return fail(MOCHY_E_INVALID, "null argument");
  *ticket = 0;
  if (req->kind != MOCHY_REQ_EXACT && req->kind != MOCHY_REQ_SAMPLED &&
      req->kind != MOCHY_REQ_PROFILE)
    return fail(MOCHY_E_INVALID, "unknown request kind");
  if (req->n_nodes < 0 || req->n_edges < 0) return fail(MOCHY_E_INVALID, "negative size");
  if (req->n_edges > 0 && (!req->edge_offsets || !req->edge_nodes))
    return fail(MOCHY_E_INVALID, "null array");
  if (req->n_edges > 0 && req->edge_offsets[0] != 0)
    return fail(MOCHY_E_INVALID, "offsets must start at 0");
  if (req->kind == MOCHY_REQ_SAMPLED &&
      (req->samples <= 0 || (req->method != MOCHY_A && req->method != MOCHY_A_PLUS)))
    return fail(MOCHY_E_INVALID, "sampled requests need samples > 0 and a method");
  if (req->kind == MOCHY_REQ_PROFILE && req->n_random <= 0)
    return fail(MOCHY_E_INVALID, "profile requests need n_random > 0");
  const int64_t T = req->n_edges > 0 ? req->edge_offsets[req->n_edges] : 0;
  if (T < 0) return fail(MOCHY_E_INVALID, "bad offsets");
  auto r = std::make_unique<Request>();
  r->kind = req->kind;
  r->n_nodes = req->n_nodes;
  r->off.assign(req->edge_offsets ? req->edge_offsets : nullptr,
                req->edge_offsets ? req->edge_offsets + req->n_edges + 1 : nullptr);
  if (r->off.empty()) r->off.push_back(0);
  if (T > 0) r->nodes.assign(req->edge_nodes, req->edge_nodes + T);
  r->method = req->method;
  r->samples = req->samples;
  r->n_random = req->n_random;
  r->seed = req->seed;
  // a profile holds the input and one copy at a time
  r->est = estimate_graph_bytes(req->n_nodes, req->n_edges, req->edge_offsets, req->edge_nodes) *
           (req->kind == MOCHY_REQ_PROFILE ? 2 : 1);
  // a MoCHy-A+ request whose line graph would take more than a quarter of
  // the budget runs without it (identical results; the memory is the
  // hypergraph, the degree arrays and the membership bitmaps)
  if (req->kind == MOCHY_REQ_SAMPLED && req->method == MOCHY_A_PLUS && r->est > s->budget / 4) {
    r->onthefly = true;
    r->otf_budget = std::min<int64_t>(s->budget / 8, (int64_t)1 << 30);
    r->est = (int64_t)(64.0 * (double)req->n_edges + 48.0 * (double)T +
                       20.0 * (double)req->n_nodes) + r->otf_budget + ((int64_t)1 << 20);
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->setup_rc < 0) return fail(s->setup_rc, "a server slot failed to start");
  if (r->est > s->budget) {
    s->rejected += 1;
    return fail(MOCHY_E_NOMEM, "request needs about " + std::to_string(r->est) +
                                   " bytes, more than the server budget");
  }
  if ((int64_t)s->pending.size() >= s->max_queue) {
    s->rejected += 1;
    return fail(MOCHY_E_BUSY, "request queue is full");
  }
  r->ticket = s->next_ticket++;
  r->t_submit = s->now_ms();
  if (s->first_submit < 0) s->first_submit = r->t_submit;
  *ticket = r->ticket;
  s->pending.push_back(std::move(r));
  s->submitted += 1;
  s->cv_work.notify_one();
  return MOCHY_OK;
}

int mochy_server_poll(mochy_server* s, int64_t ticket, mochy_result* out, int32_t wait_ms) {
  if (!s || !out) return fail(MOCHY_E_INVALID, "null argument");
  if (ticket <= 0) return fail(MOCHY_E_INVALID, "bad ticket");
  std::unique_lock<std::mutex> lk(s->mu);
  if (ticket >= s->next_ticket) return fail(MOCHY_E_INVALID, "unknown ticket");
  auto ready = [&] { return s->done.count(ticket) > 0 || s->setup_rc < 0; };
  if (wait_ms > 0) s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), ready);
  auto it = s->done.find(ticket);
  if (it == s->done.end()) {
    if (s->setup_rc < 0) return fail(s->setup_rc, "a server slot failed to start");
    return 0;
  }
  *out = *it->second;
  s->done.erase(it);
  return 1;
}

int mochy_server_stats(mochy_server* s, mochy_serving_stats* st) {
  if (!s || !st) return fail(MOCHY_E_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  memset(st, 0, sizeof(*st));
  st->submitted = s->submitted;
  st->completed = s->completed;
  st->failed = s->failed;
  st->rejected = s->rejected;
  st->queued = (int64_t)s->pending.size();
  st->in_flight = s->in_flight;
  st->peak_in_flight = s->peak_in_flight;
  st->budget_bytes = s->budget;
  st->peak_reserved_bytes = s->peak_reserved;
  st->p50_ms = percentile(s->latency_ms, 0.50);
  st->p99_ms = percentile(s->latency_ms, 0.99);
  double sum = 0.0, mx = 0.0;
  for (double v : s->latency_ms) {
    sum += v;
    mx = std::max(mx, v);
  }
  st->mean_ms = s->latency_ms.empty() ? 0.0 : sum / (double)s->latency_ms.size();
  st->max_ms = mx;
  const double span = s->last_done - s->first_submit;
  st->throughput_rps = (s->completed > 0 && span > 0.0) ? (double)s->completed / (span / 1e3) : 0.0;
  return MOCHY_OK;
}

int mochy_server_destroy(mochy_server* s) {
  if (!s) return MOCHY_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  delete s;
  return MOCHY_OK;
}

}  // extern "C"
