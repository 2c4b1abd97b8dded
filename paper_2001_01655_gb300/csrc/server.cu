// Serving loop: continuous batching of topology-optimisation solves of mixed sizes.
//
// A request is one design update of one problem: new densities, then the hierarchy refresh
// (Sec. 3.2 setup) and the solve (Sec. 3.1) warm-started from the problem's previous solution,
// which stays on the device between updates (the paper's warm start, Sec. 4).  Worker threads
// (one per slot) take requests in arrival order as soon as a slot is free and the request fits
// the device-memory budget; every problem runs on its own stream, so requests that are in
// flight at the same time overlap on the GPU.  The same problem is never processed by two
// slots at once (its updates are applied in submission order).  Results do not depend on the
// mix: every reduction has a fixed order and each problem has private buffers.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "solver.h"

namespace tomg {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  tomg_problem* P = nullptr;
  std::vector<double> rho, f;
  double* u = nullptr;  // host, nullable
  int nrhs = 1;
  tomg_options opt{};
  size_t bytes = 0;
  Clock::time_point t_submit, t_start, t_end;
  std::vector<tomg_result> res;
  tomg_status status = TOMG_OK;
  std::string error;
  bool done = false;
};

}  // namespace
}  // namespace tomg

struct tomg_server {
  tomg_ctx* ctx = nullptr;
  size_t budget = 0;
  int slots = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<tomg::Request>> queue;
  std::map<uint64_t, std::shared_ptr<tomg::Request>> tickets;
  std::map<tomg_problem*, bool> busy;
  std::map<tomg_problem*, tomg::DBuf<double>*> warm;  // device-resident previous solutions
  // device bytes each problem holds between its updates (hierarchy, solve slots, warm start),
  // measured after its latest update; requests of problems not yet resident count with their
  // estimated footprint while in flight
  std::map<tomg_problem*, size_t> resident;
  std::map<tomg_problem*, int> pending;  // queued + running requests per problem
  size_t resident_total = 0;
  size_t in_flight = 0, peak_in_flight = 0;
  int active = 0, peak_active = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::vector<std::thread> workers;
  std::vector<double> latencies_ms;
  tomg::Clock::time_point t_first{}, t_last{};
  int64_t completed = 0;
};

namespace tomg {
namespace {

// estimated device bytes of a problem that has not run yet: moduli and density, the FP64
// fine stencil (3^d blocks of d x d per node: 648 B per DOF in 3D, 144 in 2D), the coarser
// geometric and algebraic levels with their FP32 copies and block-diagonal inverses, and one
// solve slot's FP64 Krylov vectors and FP32/FP64 V-cycle work vectors
size_t footprint(const tomg_problem* P) {
  const size_t n = (size_t)P->n, nel = (size_t)P->nel;
  const size_t hier = n * (P->dim == 3 ? 648 + 140 : 144 + 100);
  const size_t slot = n * (8 * 8 + 4 * 4 + 4 * 8);
  return nel * 20 + hier + slot + ((size_t)32 << 20);
}

// whether request R may start now; extra = bytes it adds to the device while it runs.  A
// problem that is resident already holds its memory: its requests always start (the resident
// total may exceed the budget when measured footprints exceed the estimates; holding them
// back then would stop every client from finishing and retiring).  A new problem starts when
// its estimated footprint fits beside the resident problems and the other new ones in flight.
bool admissible(const tomg_server* S, const Request& R, size_t* extra) {
  if (S->resident.count(R.P) != 0) {
    *extra = 0;
    return true;
  }
  *extra = R.bytes;
  if (S->active == 0 && S->resident_total == 0) return true;  // always make progress
  return S->resident_total + S->in_flight + *extra <= S->budget;
}

void process(tomg_server* S, Request& R) {
  tomg_problem* P = R.P;
  CK(cudaSetDevice(P->ctx->device));
  set_alloc_stream(P->stream);
  set_density(P, R.rho.data(), 0);
  setup(P, R.opt);
  DBuf<double>* u0;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->warm.find(P);
    if (it == S->warm.end()) it = S->warm.emplace(P, new DBuf<double>()).first;
    u0 = it->second;
  }
  const size_t need = (size_t)P->n * R.nrhs;
  if (u0->n != need) {
    u0->resize(need);
    u0->zero(P->stream);
  }
  DBuf<double> fd;
  fd.resize(need);
  CK(cudaMemcpyAsync(fd.p, R.f.data(), need * 8, cudaMemcpyHostToDevice, P->stream));
  R.res.assign(R.nrhs, tomg_result{});
  R.status = solve(P, R.nrhs, fd.p, u0->p, 1, R.res.data());
  if (R.u) CK(cudaMemcpyAsync(R.u, u0->p, need * 8, cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
}

void worker_loop(tomg_server* S) {
  while (true) {
    std::shared_ptr<Request> R;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      while (true) {
        if (S->stop) return;
        // first request in arrival order whose problem is idle and which fits the budget;
        // a problem already resident on the device adds nothing and is never held up by a
        // new problem that does not fit yet (its client would otherwise never finish and
        // retire, so the new one could never get in)
        for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
          Request& q = **it;
          if (S->busy[q.P]) continue;
          size_t extra = 0;
          if (!admissible(S, q, &extra)) continue;
          R = *it;
          R->bytes = extra;
          S->queue.erase(it);
          break;
        }
        if (R) break;
        S->cv_work.wait(lk);
      }
      S->busy[R->P] = true;
      S->in_flight += R->bytes;
      S->active++;
      S->peak_in_flight = std::max(S->peak_in_flight, S->resident_total + S->in_flight);
      S->peak_active = std::max(S->peak_active, S->active);
      R->t_start = Clock::now();
    }
    try {
      process(S, *R);
    } catch (const Error& e) {
      R->status = e.st;
      R->error = get_error();
    } catch (...) {
      R->status = TOMG_E_CUDA;
      R->error = "unexpected internal error";
    }
    size_t held = 0;
    try {
      held = problem_device_bytes(R->P);
    } catch (...) {
      held = footprint(R->P);
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      R->t_end = Clock::now();
      R->done = true;
      S->busy[R->P] = false;
      S->in_flight -= R->bytes;
      auto w = S->warm.find(R->P);
      held += (w != S->warm.end() && w->second) ? w->second->bytes() : 0;
      auto rs = S->resident.find(R->P);
      if (rs != S->resident.end()) S->resident_total -= rs->second;
      S->resident[R->P] = held;
      S->resident_total += held;
      S->peak_in_flight = std::max(S->peak_in_flight, S->resident_total + S->in_flight);
      if (--S->pending[R->P] == 0) S->pending.erase(R->P);
      S->active--;
      S->latencies_ms.push_back(
          std::chrono::duration<double, std::milli>(R->t_end - R->t_submit).count());
      if (S->completed == 0) S->t_first = R->t_submit;
      S->t_last = R->t_end;
      S->completed++;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
}

}  // namespace
}  // namespace tomg

using namespace tomg;

extern "C" {

tomg_status tomg_server_create(tomg_ctx* ctx, size_t hbm_budget_bytes, int max_slots,
                               tomg_server** out) {
  if (!ctx || !out || max_slots < 1 || max_slots > 64 || hbm_budget_bytes == 0) {
    set_error("tomg_server_create: bad arguments");
    return TOMG_E_INVALID;
  }
  auto* S = new tomg_server();
  S->ctx = ctx;
  S->budget = hbm_budget_bytes;
  S->slots = max_slots;
  for (int k = 0; k < max_slots; k++) S->workers.emplace_back(worker_loop, S);
  *out = S;
  return TOMG_OK;
}

tomg_status tomg_server_submit(tomg_server* S, tomg_problem* P, const double* rho, int nrhs,
                               const double* f, double* u, const tomg_options* opt,
                               uint64_t* ticket) {
  if (!S || !P || !rho || !f || nrhs < 1 || !ticket) {
    set_error("tomg_server_submit: bad arguments");
    return TOMG_E_INVALID;
  }
  auto R = std::make_shared<Request>();
  R->P = P;
  R->rho.assign(rho, rho + P->nel);
  R->f.assign(f, f + (size_t)P->n * nrhs);
  R->u = u;
  R->nrhs = nrhs;
  if (opt) R->opt = *opt;
  else tomg_options_default(&R->opt);
  R->bytes = footprint(P) + (size_t)P->n * 8 * 2 * nrhs;
  if (R->bytes > S->budget) {
    set_error("request needs about %zu bytes, more than the server budget %zu", R->bytes, S->budget);
    return TOMG_E_BUDGET;
  }
  R->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    R->ticket = S->next_ticket++;
    S->tickets[R->ticket] = R;
    S->queue.push_back(R);
    S->pending[P]++;
  }
  S->cv_work.notify_all();
  *ticket = R->ticket;
  return TOMG_OK;
}

tomg_status tomg_server_wait(tomg_server* S, uint64_t ticket, int timeout_ms,
                             tomg_result* results) {
  if (!S) {
    set_error("null server");
    return TOMG_E_INVALID;
  }
  std::shared_ptr<Request> R;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) {
      set_error("unknown ticket %llu", (unsigned long long)ticket);
      return TOMG_E_INVALID;
    }
    R = it->second;
    auto ready = [&] { return R->done; };
    if (timeout_ms < 0) S->cv_done.wait(lk, ready);
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
      set_error("ticket %llu not finished within %d ms", (unsigned long long)ticket, timeout_ms);
      return TOMG_E_TIMEOUT;
    }
    S->tickets.erase(it);
  }
  if (results)
    for (int j = 0; j < R->nrhs && j < (int)R->res.size(); j++) results[j] = R->res[j];
  if (R->status < 0) set_error("%s", R->error.c_str());
  return R->status;
}

tomg_status tomg_server_stats(tomg_server* S, double* p50_ms, double* p99_ms,
                              double* solves_per_s, int64_t* completed, int* peak_active,
                              size_t* peak_bytes) {
  if (!S) {
    set_error("null server");
    return TOMG_E_INVALID;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  std::vector<double> v = S->latencies_ms;
  std::sort(v.begin(), v.end());
  auto pct = [&](double q) {
    if (v.empty()) return 0.0;
    const double pos = q * (v.size() - 1);
    const size_t lo = (size_t)pos;
    const size_t hi = std::min(lo + 1, v.size() - 1);
    return v[lo] + (pos - lo) * (v[hi] - v[lo]);
  };
  if (p50_ms) *p50_ms = pct(0.50);
  if (p99_ms) *p99_ms = pct(0.99);
  const double span = std::chrono::duration<double>(S->t_last - S->t_first).count();
  if (solves_per_s) *solves_per_s = (S->completed > 0 && span > 0) ? S->completed / span : 0.0;
  if (completed) *completed = S->completed;
  if (peak_active) *peak_active = S->peak_active;
  if (peak_bytes) *peak_bytes = S->peak_in_flight;
  return TOMG_OK;
}

tomg_status tomg_server_retire(tomg_server* S, tomg_problem* P, int timeout_ms) {
  if (!S || !P) {
    set_error("tomg_server_retire: bad arguments");
    return TOMG_E_INVALID;
  }
  DBuf<double>* w = nullptr;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    auto idle = [&] { return S->pending.count(P) == 0; };
    if (timeout_ms < 0) S->cv_done.wait(lk, idle);
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), idle)) {
      set_error("problem still has requests after %d ms", timeout_ms);
      return TOMG_E_TIMEOUT;
    }
    auto it = S->warm.find(P);
    if (it != S->warm.end()) {
      w = it->second;
      S->warm.erase(it);
    }
    auto rs = S->resident.find(P);
    if (rs != S->resident.end()) {
      S->resident_total -= rs->second;
      S->resident.erase(rs);
    }
    S->busy.erase(P);
  }
  if (w) {
    try {
      CK(cudaSetDevice(S->ctx->device));
      set_alloc_stream(P->stream);
      CK(cudaStreamSynchronize(P->stream));
    } catch (...) {
    }
    delete w;
  }
  S->cv_work.notify_all();
  return TOMG_OK;
}

tomg_status tomg_server_destroy(tomg_server* S) {
  if (!S) return TOMG_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    for (auto& q : S->queue) {  // never started: finish with an error so waiters return
      q->status = TOMG_E_INVALID;
      q->error = "server destroyed before the request started";
      q->done = true;
    }
    S->queue.clear();
  }
  S->cv_work.notify_all();
  S->cv_done.notify_all();
  for (auto& t : S->workers) t.join();
  cudaSetDevice(S->ctx->device);
  set_alloc_stream(S->ctx->stream);
  for (auto& kv : S->warm) {
    cudaStreamSynchronize(kv.first->stream);
    delete kv.second;
  }
  delete S;
  return TOMG_OK;
}

}  // extern "C"
