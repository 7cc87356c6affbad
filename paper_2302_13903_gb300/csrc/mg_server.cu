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
// Requests of at most kBatchMaxN^3 cells with a periodic, fixed or
// zero-gradient rule on device arrays go through batched hierarchies of
// kBatchSlots grids: a slot that takes one also takes the queued requests of
// the same shape and rule (up to kBatchSlots in all) and solves them in one
// persistent launch.
constexpr int kBatchMaxN = 64;
constexpr int kBatchSlots = 16;

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

// A resident hierarchy of the pool: a solver context, or a batch of
// kBatchSlots grids of one shape (Key::slots > 0).
struct Hier {
  mg_ctx* ctx = nullptr;
  mg_batch* batch = nullptr;
  // a batch serving host arrays: each slot's device copies of rho and phi
  std::vector<double*> dev;
};

void destroy_hier(void* p) {
  Hier* h = static_cast<Hier*>(p);
  if (!h) return;
  if (h->batch) mg_batch_destroy(h->batch);
  if (h->ctx) mg_destroy(h->ctx);
  for (double* d : h->dev) cudaFree(d);
  delete h;
}

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
  long long batched = 0;  // requests solved in a batched launch with others
  int running = 0;
  int head_bypassed = 0;
  unsigned long long gen = 0;  // bumped on every submission and completion
  bool stop = false;
  std::vector<std::thread> workers;
  std::string err;
};

namespace {

// Whether the server's options allow the batched solve (mg_batch_create's
// conditions).
bool batch_opts_ok(const mg_opts& o) {
  return o.batch_small == 1 && o.prec == MG_MIXED && o.pre == 1 && o.post == 1 && o.mode_fmg == 1 &&
         o.inner_fmg == 0 && o.max_cycles <= 64 && o.inner_cycles <= 16 && o.first_cycles <= 17 &&
         o.coarse_literal == 0;
}

// Create the hierarchy of a CREATE decision for request r.
mg_status create_hier(mg_server* S, const Request* r, cudaStream_t stream, Hier** out) {
  Hier* h = new Hier;
  mg_opts o = S->opts;
  o.lmax = r->req.lmax;
  o.fixed_value = r->req.fixed_value;
  mg_status st;
  if (r->key.slots > 0) {
    const int k = r->key.slots;
    std::vector<int> dims(3 * (size_t)k, r->req.nx);
    std::vector<double> dx((size_t)k, r->req.dx), fv((size_t)k, r->req.fixed_value);
    std::vector<mg_bc> bcs((size_t)k, r->req.bc);
    st = mg_batch_create(k, dims.data(), dx.data(), bcs.data(), fv.data(), &o, &h->batch);
    // one CTA per SM: the small grids need no more, and the other slots'
    // solves keep room on every SM
    if (st == MG_OK) st = mg_batch_set_blocks(h->batch, mg::sm_count());
    if (st == MG_OK && r->key.host) {  // device copies of each slot's rho and phi
      const size_t bytes = sizeof(double) * (size_t)r->req.nx * r->req.ny * r->req.nz;
      for (int g = 0; g < 2 * k && st == MG_OK; ++g) {
        double* d = nullptr;
        if (cudaMalloc(&d, bytes) != cudaSuccess) {
          cudaGetLastError();
          st = MG_ERR_OOM;
        } else {
          h->dev.push_back(d);
        }
      }
    }
  } else {
    if (r->req.per_face)
      st = mg_create_faces(r->req.nx, r->req.ny, r->req.nz, r->req.dx, r->req.face_bc,
                           r->req.face_value, &o, &h->ctx);
    else
      st = mg_create(r->req.nx, r->req.ny, r->req.nz, r->req.dx, r->req.bc, &o, &h->ctx);
    if (st == MG_OK) mg_ctx_autotune(h->ctx, stream);  // shapes, cached per process
  }
  if (st != MG_OK) {
    destroy_hier(h);
    h = nullptr;
  }
  *out = h;
  return st;
}

// One batched solve of the requests in `group` (same key) on hierarchy h.
// Host arrays are copied in and out on the slot's stream around the launch.
void solve_group(Hier* h, std::vector<Request*>& group, cudaStream_t stream) {
  const int k = (int)group.size();
  const int slots = group[0]->key.slots;
  const bool host = group[0]->key.host;
  const size_t bytes =
      sizeof(double) * (size_t)group[0]->req.nx * group[0]->req.ny * group[0]->req.nz;
  cudaError_t ce = cudaSuccess;
  std::vector<const double*> rho((size_t)slots, nullptr);
  std::vector<double*> phi((size_t)slots, nullptr);
  std::vector<double> fpg((size_t)slots, 0.0), tol((size_t)slots, 0.0);
  std::vector<double> hist((size_t)slots * kHistCap, 0.0);
  std::vector<int> nh((size_t)slots, 0);
  std::vector<mg_status> sts((size_t)slots, MG_OK);
  for (int g = 0; g < k; ++g) {
    const Request* r = group[(size_t)g];
    rho[(size_t)g] = host ? h->dev[2 * (size_t)g] : r->req.rho;
    phi[(size_t)g] = host ? h->dev[2 * (size_t)g + 1] : r->req.phi;
    fpg[(size_t)g] = r->req.four_pi_G;
    tol[(size_t)g] = r->req.tol;
    if (host && ce == cudaSuccess)
      ce = cudaMemcpyAsync(h->dev[2 * (size_t)g], r->req.rho, bytes, cudaMemcpyHostToDevice,
                           stream);
  }
  mg_status st = ce == cudaSuccess
                     ? mg_batch_solve(h->batch, rho.data(), fpg.data(), tol.data(), phi.data(),
                                      hist.data(), kHistCap, nh.data(), sts.data(), stream)
                     : MG_ERR_CUDA;
  if (host && (st == MG_OK || st == MG_ERR_NOT_CONVERGED || st == MG_ERR_DIVERGED)) {
    for (int g = 0; g < k && ce == cudaSuccess; ++g)
      ce = cudaMemcpyAsync(group[(size_t)g]->req.phi, h->dev[2 * (size_t)g + 1], bytes,
                           cudaMemcpyDeviceToHost, stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(stream);
    if (ce != cudaSuccess) st = MG_ERR_CUDA;
  }
  if (ce != cudaSuccess) cudaGetLastError();
  const bool whole = st == MG_ERR_ARG || st == MG_ERR_CUDA || st == MG_ERR_TIMEOUT;
  for (int g = 0; g < k; ++g) {
    Request* r = group[(size_t)g];
    r->status = whole ? st : sts[(size_t)g];
    r->n_hist = whole ? 0 : nh[(size_t)g];
    for (int q = 0; q < r->n_hist; ++q) r->hist[q] = hist[(size_t)g * kHistCap + q];
  }
}

void run_worker(mg_server* S) {
  cudaSetDevice(S->device);
  cudaStream_t stream = nullptr;
  if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    stream = nullptr;  // the slot still works, on the legacy stream
  }
  std::unique_lock<std::mutex> lk(S->mu);
  unsigned long long seen = ~0ULL;
  std::vector<Request*> group;
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
    group.clear();
    group.push_back(S->queue[(size_t)at]);
    S->queue.erase(S->queue.begin() + at);
    if (group[0]->key.slots > 0) {
      // continuous batching: the queued requests of the same shape and rule
      // join this launch, in arrival order
      for (size_t i = 0; i < S->queue.size() && (int)group.size() < group[0]->key.slots;) {
        if (S->queue[i]->key == group[0]->key) {
          group.push_back(S->queue[i]);
          S->queue.erase(S->queue.begin() + (long)i);
        } else {
          ++i;
        }
      }
    }
    const Clock::time_point t_start = Clock::now();
    for (Request* r : group) r->t_start = t_start;
    S->running += (int)group.size();
    if (!S->queue.empty()) {  // the pool changed: let the other slots look again
      ++S->gen;
      S->cv_work.notify_all();
    }
    lk.unlock();

    for (void* old : dec.evict) destroy_hier(old);
    Hier* h = static_cast<Hier*>(dec.ctx);
    Request* r = group[0];
    mg_status st = MG_OK;
    if (dec.act == Act::CREATE) {
      st = create_hier(S, r, stream, &h);
      lk.lock();
      if (st == MG_OK) S->pool.set_ctx(dec.id, h);
      else S->pool.drop(dec.id);
      lk.unlock();
    }
    if (st != MG_OK) {
      for (Request* q : group) q->status = st;
    } else if (h->batch) {
      solve_group(h, group, stream);
    } else {
      int nh = 0;
      if (r->key.host)
        st = mg::solve_host_copies(h->ctx, r->req.rho, r->req.four_pi_G, r->req.tol, r->req.phi,
                                   r->hist, kHistCap, &nh, stream, r->copy_ms);
      else
        st = mg_solve(h->ctx, r->req.rho, r->req.four_pi_G, r->req.tol, r->req.phi, r->hist,
                      kHistCap, &nh, stream);
      r->status = st;
      r->n_hist = nh;
    }
    const Clock::time_point t_done = Clock::now();

    lk.lock();
    if (h) S->pool.release(h);
    for (Request* q : group) {
      q->t_done = t_done;
      q->done = true;
      ++S->completed;
      S->cells_completed += (long long)q->req.nx * q->req.ny * q->req.nz;
    }
    S->running -= (int)group.size();
    if (group.size() > 1) S->batched += (long long)group.size();
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
  bool faces_ok = q->per_face == 0 || q->per_face == 1;
  int fk = 0;
  if (q->per_face == 1) {
    for (int f = 0; f < 6; ++f) {
      const mg_bc k = q->face_bc[f];
      faces_ok = faces_ok && (k == MG_BC_PERIODIC || k == MG_BC_FIXED || k == MG_BC_ZEROGRAD) &&
                 std::isfinite(q->face_value[f]);
      fk |= ((int)k & 3) << (2 * f);
    }
    for (int a = 0; a < 3; ++a)
      faces_ok = faces_ok && ((q->face_bc[2 * a] == MG_BC_PERIODIC) ==
                              (q->face_bc[2 * a + 1] == MG_BC_PERIODIC));
  }
  if (!pow2(q->nx) || q->nx != q->ny || q->nx != q->nz || !(q->dx > 0.0) || !q->rho ||
      !q->phi || !(q->tol >= 0.0) || !std::isfinite(q->four_pi_G) || !faces_ok ||
      (!q->per_face && ((int)q->bc < 0 || (int)q->bc > 3)) || q->lmax < 0 || q->lmax > 4) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->err = "mg_server_submit: invalid request";
    return MG_ERR_ARG;
  }
  mg_opts o = S->opts;
  o.lmax = q->lmax;
  o.fixed_value = q->fixed_value;
  size_t need = 0;
  // a rule per face: the bytes of a fixed-rule hierarchy plus the face arrays
  // of its levels (at most 4/3 of the finest level's)
  const mg_bc need_bc = q->per_face ? MG_BC_FIXED : q->bc;
  if (mg_required_bytes(q->nx, q->ny, q->nz, need_bc, &o, &need) != MG_OK) {
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
  if (q->per_face) need += 4 * sizeof(double) * 6 * (size_t)(q->nx + 2) * (q->nx + 2) / 3;
  Request* r = new Request;
  r->req = *q;
  r->key.n = q->nx;
  r->key.bc = q->per_face ? (int)MG_BC_MIXED : (int)q->bc;
  r->key.lmax = !q->per_face && q->bc == MG_BC_OPEN ? q->lmax : 0;
  r->key.dx = q->dx;
  r->key.fixed_value = !q->per_face && q->bc == MG_BC_FIXED ? q->fixed_value : 0.0;
  r->key.host = host;
  if (q->per_face) {
    r->key.fk = fk;
    for (int f = 0; f < 6; ++f)
      r->key.fv[f] = q->face_bc[f] == MG_BC_FIXED ? q->face_value[f] : 0.0;
  }
  // small requests with a periodic, fixed or zero-gradient rule: a batched
  // hierarchy of up to kBatchSlots grids, as many as the budget holds (its
  // bytes: that many single hierarchies); the slot count of a shape is fixed
  // by the budget, and a grid's result does not depend on it
  if (!q->per_face && q->nx <= kBatchMaxN && q->bc != MG_BC_OPEN && batch_opts_ok(S->opts) &&
      need > 0) {
    size_t k = S->pool.budget() / need;
    if (k > (size_t)kBatchSlots) k = kBatchSlots;
    if (k >= 1) {
      r->key.slots = (int)k;
      need *= k;
    }
  }
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
  out->batched = S->batched;
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
  for (void* c : S->pool.drain_idle()) destroy_hier(c);
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
