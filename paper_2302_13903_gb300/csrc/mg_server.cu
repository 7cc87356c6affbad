// mg_server.cu -- the serving loop: solves of different sizes and boundary
// rules arrive one by one, wait in a queue, and run as soon as a worker slot
// and device memory allow, several at once on separate CUDA streams.
//
// Each worker slot is one host thread with its own non-blocking stream; it
// takes the next admissible request (mg_admission.h), runs mg_solve on a
// resident hierarchy of the request's key, and hands the hierarchy back to
// the pool, where it stays for the next request of that key until the HBM
// budget needs its room.  While one slot waits on its stream (the solve reads
// its convergence scalars every outer iteration), the others keep launching,
// so the kernels of different requests overlap on the device.  Every result
// is the one the same request gives alone: each hierarchy is used by one
// request at a time, and a solve is deterministic given its inputs.  A
// request with host buffers has its rho and phi moved by the copy engines on
// its slot's stream, so its transfers overlap the other slots' solves.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/mg.h"
#include "mg_admission.h"
#include "mg_internal.h"
#include "mg_tickets.h"

namespace {

using Clock = std::chrono::steady_clock;
using mg::admission::Act;
using mg::admission::Decision;
using mg::admission::Key;
using mg::admission::Pool;

constexpr int kHistCap = 64;
constexpr int kMaxBypass = 64;

thread_local std::string g_server_err;

struct Request {
  long long ticket = 0;
  mg_request req{};
  Key key;
  size_t need = 0;
  Clock::time_point t_submit, t_start, t_done;
  bool done = false;
  int waiters = 0;       // threads in mg_server_wait on this ticket
  bool retired = false;  // the ticket no longer resolves (mg_tickets.h)
  mg_status status = MG_OK;
  int n_hist = 0;
  double copy_ms[2] = {};  // host arrays: device time of the copies in and out
  double hist[kHistCap] = {};
};

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

bool pow2(int n) { return n >= 2 && (n & (n - 1)) == 0; }

// 0: device (or managed) memory, 1: host memory, page-locked or not; -1: unknown.
int memory_space(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return 0;
  return 1;
}

}  // namespace

struct mg_server {
  mg_opts opts{};
  int device = 0;
  int slots = 0;
  int max_queue = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  Pool pool{0};
  std::deque<Request*> queue;
  mg::tickets::Book<Request> reqs;
  long long next_ticket = 1;
  long long submitted = 0, completed = 0, rejected = 0, cells_completed = 0;
  int running = 0;
  int head_bypassed = 0;
  unsigned long long gen = 0;  // bumped on every submission and completion
  bool stop = false;
  std::vector<std::thread> workers;
  std::string err;
};

namespace {

void run_worker(mg_server* S) {
  cudaSetDevice(S->device);
  cudaStream_t stream = nullptr;
  if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    stream = nullptr;  // the slot still works, on the legacy stream
  }
  std::unique_lock<std::mutex> lk(S->mu);
  unsigned long long seen = ~0ULL;
  for (;;) {
    if (S->queue.empty() || seen == S->gen) {
      if (S->stop && S->queue.empty()) break;
      S->cv_work.wait(lk, [&] {
        return (S->stop && S->queue.empty()) || (!S->queue.empty() && seen != S->gen);
      });
      continue;
    }
    seen = S->gen;
    Decision dec;
    const int at = mg::admission::pick(
        S->queue.size(), S->head_bypassed, kMaxBypass, [&](size_t i) {
          Decision d = S->pool.admit(S->queue[i]->key, S->queue[i]->need);
          if (d.act == Act::USE || d.act == Act::CREATE) {
            dec = d;
            return true;
          }
          return false;
        });
    if (at < 0) continue;  // nothing fits now: wait for a completion
    Request* r = S->queue[(size_t)at];
    S->queue.erase(S->queue.begin() + at);
    ++S->running;
    r->t_start = Clock::now();
    if (!S->queue.empty()) {  // the pool changed: let the other slots look again
      ++S->gen;
      S->cv_work.notify_all();
    }
    lk.unlock();

    for (void* old : dec.evict) mg_destroy(static_cast<mg_ctx*>(old));
    mg_ctx* ctx = static_cast<mg_ctx*>(dec.ctx);
    mg_status st = MG_OK;
    if (dec.act == Act::CREATE) {
      mg_opts o = S->opts;
      o.lmax = r->req.lmax;
      o.fixed_value = r->req.fixed_value;
      st = mg_create(r->req.nx, r->req.ny, r->req.nz, r->req.dx, r->req.bc, &o, &ctx);
      lk.lock();
      if (st == MG_OK) S->pool.set_ctx(dec.id, ctx);
      else S->pool.drop(dec.id);
      lk.unlock();
    }
    if (st == MG_OK && dec.act == Act::CREATE) mg_ctx_autotune(ctx, stream);  // shapes, cached
    int nh = 0;
    if (st == MG_OK && r->key.host)
      st = mg::solve_host_copies(ctx, r->req.rho, r->req.four_pi_G, r->req.tol, r->req.phi,
                                 r->hist, kHistCap, &nh, stream, r->copy_ms);
    else if (st == MG_OK)
      st = mg_solve(ctx, r->req.rho, r->req.four_pi_G, r->req.tol, r->req.phi, r->hist, kHistCap,
                    &nh, stream);
    const Clock::time_point t_done = Clock::now();

    lk.lock();
    if (ctx) S->pool.release(ctx);
    r->t_done = t_done;
    r->status = st;
    r->n_hist = nh;
    r->done = true;
    --S->running;
    ++S->completed;
    S->cells_completed += (long long)r->req.nx * r->req.ny * r->req.nz;
    ++S->gen;
    S->cv_work.notify_all();
    S->cv_done.notify_all();
  }
  lk.unlock();
  if (stream) cudaStreamDestroy(stream);
}

void fill_result(const Request* r, mg_result* res, double* hist, int hist_cap) {
  std::memset(res, 0, sizeof *res);
  res->done = r->done ? 1 : 0;
  if (!r->done) return;
  res->status = r->status;
  res->n_hist = std::min(r->n_hist, std::max(hist_cap, 0));
  if (hist)
    for (int q = 0; q < res->n_hist; ++q) hist[q] = r->hist[q];
  res->queue_ms = ms_between(r->t_submit, r->t_start);
  res->solve_ms = ms_between(r->t_start, r->t_done);
  res->total_ms = ms_between(r->t_submit, r->t_done);
  res->h2d_ms = r->copy_ms[0];
  res->d2h_ms = r->copy_ms[1];
}

}  // namespace

extern "C" {

mg_status mg_server_create(size_t hbm_budget_bytes, int slots, int max_queue,
                           const mg_opts* opts, mg_server** out) {
  if (!out || hbm_budget_bytes == 0 || slots < 1 || slots > 64 || max_queue < 1) {
    g_server_err = "mg_server_create: invalid argument";
    return MG_ERR_ARG;
  }
  *out = nullptr;
  mg_opts o;
  if (opts) o = *opts;
  else mg_opts_init(&o);
  size_t probe = 0;
  if (mg_required_bytes(2, 2, 2, MG_BC_PERIODIC, &o, &probe) != MG_OK) {
    g_server_err = "mg_server_create: invalid options";
    return MG_ERR_ARG;
  }
  mg_server* S = new mg_server;
  S->opts = o;
  S->slots = slots;
  S->max_queue = max_queue;
  S->pool = Pool(hbm_budget_bytes);
  cudaGetDevice(&S->device);
  try {
    for (int w = 0; w < slots; ++w) S->workers.emplace_back(run_worker, S);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->stop = true;
    }
    S->cv_work.notify_all();
    for (std::thread& t : S->workers) t.join();
    delete S;
    g_server_err = "mg_server_create: could not start the worker threads";
    return MG_ERR_ARG;
  }
  *out = S;
  return MG_OK;
}

mg_status mg_server_submit(mg_server* S, const mg_request* q, long long* ticket) {
  if (!S || !q || !ticket) {
    g_server_err = "mg_server_submit: invalid argument";
    return MG_ERR_ARG;
  }
  *ticket = 0;
  if (!pow2(q->nx) || q->nx != q->ny || q->nx != q->nz || !(q->dx > 0.0) || !q->rho ||
      !q->phi || !(q->tol >= 0.0) || !std::isfinite(q->four_pi_G) || (int)q->bc < 0 ||
      (int)q->bc > 3 || q->lmax < 0 || q->lmax > 4) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->err = "mg_server_submit: invalid request";
    return MG_ERR_ARG;
  }
  mg_opts o = S->opts;
  o.lmax = q->lmax;
  o.fixed_value = q->fixed_value;
  size_t need = 0;
  if (mg_required_bytes(q->nx, q->ny, q->nz, q->bc, &o, &need) != MG_OK) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->err = "mg_server_submit: invalid request";
    return MG_ERR_ARG;
  }
  // rho and phi both in device memory, or both in host memory (page-locked
  // or not); then the hierarchy also keeps device copies of the two arrays
  const int rs = memory_space(q->rho), ps = memory_space(q->phi);
  if (rs < 0 || rs != ps) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->err = "mg_server_submit: rho and phi must both be device arrays or both host arrays";
    return MG_ERR_ARG;
  }
  const bool host = rs == 1;
  if (host) need += 2 * sizeof(double) * (size_t)q->nx * q->ny * q->nz;
  Request* r = new Request;
  r->req = *q;
  r->key.n = q->nx;
  r->key.bc = (int)q->bc;
  r->key.lmax = q->bc == MG_BC_OPEN ? q->lmax : 0;
  r->key.dx = q->dx;
  r->key.fixed_value = q->bc == MG_BC_FIXED ? q->fixed_value : 0.0;
  r->key.host = host;
  r->need = need;
  std::lock_guard<std::mutex> lk(S->mu);
  if (need > S->pool.budget()) {
    delete r;
    ++S->rejected;
    S->err = "mg_server_submit: the grid's hierarchy alone exceeds the HBM budget";
    return MG_ERR_OOM;
  }
  if ((int)S->queue.size() >= S->max_queue || S->stop) {
    delete r;
    ++S->rejected;
    S->err = "mg_server_submit: queue full";
    return MG_ERR_BUSY;
  }
  r->ticket = S->next_ticket++;
  r->t_submit = Clock::now();
  S->reqs.add(r->ticket, r);
  S->queue.push_back(r);
  ++S->submitted;
  ++S->gen;
  S->cv_work.notify_one();
  *ticket = r->ticket;
  return MG_OK;
}

mg_status mg_server_poll(mg_server* S, long long ticket, mg_result* res, double* hist,
                         int hist_cap) {
  if (!S || !res) return MG_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  const mg::tickets::Got got =
      S->reqs.poll(ticket, [&](const Request& r) { fill_result(&r, res, hist, hist_cap); });
  if (got == mg::tickets::Got::UNKNOWN) {
    S->err = "mg_server_poll: unknown or retired ticket";
    return MG_ERR_ARG;
  }
  return MG_OK;
}

mg_status mg_server_wait(mg_server* S, long long ticket, double timeout_s, mg_result* res,
                         double* hist, int hist_cap) {
  if (!S || !res || !(timeout_s >= 0.0)) return MG_ERR_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  const mg::tickets::Got got = S->reqs.wait(
      ticket, lk, S->cv_done, timeout_s,
      [&](const Request& r) { fill_result(&r, res, hist, hist_cap); });
  if (got == mg::tickets::Got::UNKNOWN) {
    S->err = "mg_server_wait: unknown or retired ticket";
    return MG_ERR_ARG;
  }
  return got == mg::tickets::Got::DONE ? MG_OK : MG_ERR_TIMEOUT;
}

mg_status mg_server_get_stats(mg_server* S, mg_server_stats* out) {
  if (!S || !out) return MG_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(out, 0, sizeof *out);
  out->submitted = S->submitted;
  out->completed = S->completed;
  out->rejected = S->rejected;
  out->evictions = S->pool.evictions();
  out->created = S->pool.created();
  out->cells_completed = S->cells_completed;
  out->budget_bytes = S->pool.budget();
  out->resident_bytes = S->pool.resident_bytes();
  out->peak_bytes = S->pool.peak_bytes();
  out->queued = (int)S->queue.size();
  out->running = S->running;
  out->slots = S->slots;
  out->resident = (int)S->pool.residents().size();
  return MG_OK;
}

mg_status mg_server_destroy(mg_server* S) {
  if (!S) return MG_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (std::thread& t : S->workers) t.join();
  for (void* c : S->pool.drain_idle()) mg_destroy(static_cast<mg_ctx*>(c));
  S->reqs.clear();
  delete S;
  return MG_OK;
}

const char* mg_server_last_error(const mg_server* S) {
  if (!S) return g_server_err.c_str();
  // submit and poll write S->err from other threads: hand out this thread's copy
  thread_local std::string copy;
  std::lock_guard<std::mutex> lk(const_cast<mg_server*>(S)->mu);
  copy = S->err;
  return copy.c_str();
}

}  // extern "C"
