// mg_solver.cu -- solver context, the FMG / V-cycle driver (FP64 and mixed
// precision) and the C ABI of include/mg.h.
//
// The driver is host code that queues kernels on the caller's stream.  Device
// data never comes back to the host except the norms the stopping test needs
// (one 16-byte read per cycle).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "../../include/mg.h"
#include "mg_internal.h"

using mg::Bc;
using mg::Grid;

namespace {

thread_local std::string g_err;  // last error of calls without a context

constexpr int kMaxLevels = 16;

}  // namespace

struct mg_ctx {
  int n = 0;            // cells along x of the finest level (nx)
  int ny = 0, nz = 0;   // cells along y and z (equal to n for cubic grids)
  int L = 0;            // number of levels; level L-1 is the finest
  double h = 0.0;       // finest spacing
  int bc_kind = 0;
  // MG_BC_MIXED: the kind of face q in bits 2q..2q+1 and the fixed faces' values
  int face_mask = 0;
  double face_b[6] = {};
  mg_opts opts{};
  int device = 0;
  // FP64 hierarchy (u64[L-1] is the caller's phi during a solve).
  double* u64[kMaxLevels] = {};
  double* f64[kMaxLevels] = {};
  double* faces[kMaxLevels] = {};  // open / fixed-face boundary values per level
  double* ur64[kMaxLevels] = {};   // FAS: restricted potential per coarse level
  // FP32 hierarchy (mixed precision); u32b is the second buffer of levels the
  // fused kernels handle (they read one buffer and write the other).
  float* u32[kMaxLevels] = {};
  float* u32b[kMaxLevels] = {};
  float* f32[kMaxLevels] = {};
  double* partials = nullptr;  // reduction partials
  int* iflag = nullptr;        // device flags: [0] fixed-point overflow, [1] tensor copy late
  long long* fxbuf = nullptr;  // second integer buffer of the fixed-point outer loop
  int partials_cap = 0;        // doubles in `partials`
  double* scal = nullptr;      // device scalars: [0] |f|^2 sum, [1] |d|^2 sum, [2..31] multipole
  double* pinned = nullptr;    // host mirror of scal
  double* rho_dev_own = nullptr;  // buffers for mg_solve_host
  double* phi_dev_own = nullptr;
  // mg_solve_host with pinned host buffers: the first pass over rho reads it
  // from host memory (and leaves the device copy), the last pass writes phi to
  // host memory (host_phi_written then set); null otherwise
  const double* host_rho = nullptr;
  double* host_phi = nullptr;
  bool host_phi_written = false;
  std::vector<void*> allocs;
  size_t bytes = 0;
  bool dry = false;  // count the bytes of the hierarchy without allocating
  long long last_launches = 0;
  std::string err;
  // Per-kernel timing of finest-level launches.
  int timing = 0;
  std::vector<cudaEvent_t> events;  // pool, used in start/stop pairs
  std::vector<int> pending_class;   // class of each recorded pair in this solve
  double kernel_ms[MG_K_COUNT] = {};
  long long kernel_n[MG_K_COUNT] = {};
  // Launch shapes of the fused legs per level and of the fixed-point outer
  // step (zeros: built-in choice), set by mg_ctx_autotune.
  mg::TileCfg cfg_down[kMaxLevels] = {}, cfg_up[kMaxLevels] = {}, cfg_smooth[kMaxLevels] = {},
              cfg_ud[kMaxLevels] = {};
  int fx_cz = 0;
  // The mixed path's inner FP32 solve (the same launches on the same buffers
  // every outer iteration) as a CUDA graph, captured on its second run and
  // replayed from then on; dropped when the launch shapes change.
  // Two graphs: [0] for 1 + inner_cycles V-cycles, [1] for the first outer
  // iteration's first_cycles when they differ.
  struct InnerGraph {
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;  // kernels in the graph
    int runs = 0;
  } inner[2];
  // the autotuner timed the finest level's fused up-down pass faster than the
  // two legs it replaces (opts.leg_pairs = 0 then fuses them)
  bool pairs_faster = false;
  // per level: the down leg (from a nonzero start / from zero) and the up leg
  // bring their planes in by tensor copies (opts.tensor_copies, autotuner)
  bool tma_down[kMaxLevels] = {}, tma_down0[kMaxLevels] = {}, tma_up[kMaxLevels] = {};
  // their planes per CTA (0: built-in choice)
  int tma_cz_down[kMaxLevels] = {}, tma_cz_down0[kMaxLevels] = {}, tma_cz_up[kMaxLevels] = {};
};

namespace {

int level_n(const mg_ctx* c, int l) { return c->n >> (c->L - 1 - l); }
double level_h(const mg_ctx* c, int l) { return c->h * (double)(1 << (c->L - 1 - l)); }
Grid level_grid(const mg_ctx* c, int l) {
  const int s = c->L - 1 - l;
  return Grid{c->n >> s, c->ny >> s, c->nz >> s};
}
bool is_cubic(const mg_ctx* c) { return c->n == c->ny && c->n == c->nz; }

bool is_pow2(int n) { return n >= 1 && (n & (n - 1)) == 0; }

// Powers of two >= 2 on every axis; a non-cubic grid must have x as a
// longest side (the red-black kernels pair cells along x, so the coarsest
// level, where the shortest side has one cell, keeps at least two along x).
bool dims_ok(int nx, int ny, int nz) {
  if (!is_pow2(nx) || !is_pow2(ny) || !is_pow2(nz) || nx < 2 || ny < 2 || nz < 2) return false;
  const bool cubic = nx == ny && nx == nz;
  return cubic || (nx >= ny && nx >= nz);
}

struct Fail {
  mg_status st;
};

}  // namespace

void mg::set_last_error(const std::string& msg) { g_err = msg; }

namespace {

void check(mg_ctx* c, cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    char buf[256];
    std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    if (c) c->err = buf;
    g_err = buf;
    throw Fail{MG_ERR_CUDA};
  }
}

void fail(mg_ctx* c, mg_status st, const std::string& msg) {
  if (c) c->err = msg;
  g_err = msg;
  throw Fail{st};
}

template <typename T>
T* dalloc(mg_ctx* c, size_t count) {
  if (c->dry) {
    c->bytes += count * sizeof(T);
    return nullptr;
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(c, MG_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  c->allocs.push_back(p);
  c->bytes += count * sizeof(T);
  return static_cast<T*>(p);
}

// Whether no face fixes the zero point of phi (Sec. 2.3.6): then the means of
// f and phi are removed.
bool mean_free(const mg_ctx* c) {
  if (c->bc_kind == MG_BC_MIXED) {
    for (int q = 0; q < 6; ++q)
      if (((c->face_mask >> (2 * q)) & 3) == MG_BC_FIXED) return false;
    return true;
  }
  return c->bc_kind == MG_BC_PERIODIC || c->bc_kind == MG_BC_ZEROGRAD;
}

// The device arrays of a context (counted only, when c->dry).
void alloc_hierarchy(mg_ctx* c) {
  const mg_bc bc = (mg_bc)c->bc_kind;
  const bool face_arrays = bc == MG_BC_OPEN || bc == MG_BC_MIXED;
  const mg_opts& o = c->opts;
  const int L = c->L;
  const int F = L - 1;
  for (int l = 0; l < L; ++l) {
    const long long cells = level_grid(c, l).cells();
    if (o.prec == MG_FP64) {
      if (l < F) c->u64[l] = dalloc<double>(c, cells);
      if (l < F && o.fas) c->ur64[l] = dalloc<double>(c, cells);
      c->f64[l] = dalloc<double>(c, cells);
      if (face_arrays) c->faces[l] = dalloc<double>(c, mg::faces_count(level_grid(c, l)));
    } else {
      c->u32[l] = dalloc<float>(c, cells);
      c->f32[l] = dalloc<float>(c, cells);
      if (mg::fused_ok(level_grid(c, l), mg::homogeneous(Bc{(int)bc, 0.0, nullptr, c->face_mask})))
        c->u32b[l] = dalloc<float>(c, cells);
    }
  }
  if (o.prec == MG_MIXED) {
    c->f64[F] = dalloc<double>(c, level_grid(c, F).cells());
    if (face_arrays) c->faces[F] = dalloc<double>(c, mg::faces_count(level_grid(c, F)));
  }
  c->partials_cap = mg::kPartials;
  if (o.prec == MG_MIXED && o.outer_fixed && mg::fx_step_ok(level_grid(c, F))) {
    c->fxbuf = dalloc<long long>(c, level_grid(c, F).cells());
    const int nb = mg::fx_step_blocks(level_grid(c, F), 0);
    if (nb > c->partials_cap) c->partials_cap = nb;
  }
  // partials, then room for two integers per block of the fixed-point step
  c->partials = dalloc<double>(c, 3 * (size_t)c->partials_cap);
  c->scal = dalloc<double>(c, 64);
  c->iflag = dalloc<int>(c, 4);
}

Bc physical_bc(const mg_ctx* c, int l) {
  Bc b{c->bc_kind, c->opts.fixed_value, c->faces[l], c->face_mask};
  return b;
}

// Fill the face arrays of a rule per face with each face's value (levels
// that have one; constant over the face and the same on every level).
void fill_mixed_faces(mg_ctx* c) {
  for (int l = 0; l < c->L; ++l) {
    if (!c->faces[l]) continue;
    const Grid g = level_grid(c, l);
    const size_t fx = (size_t)(g.ny + 2) * (g.nz + 2), fy = (size_t)(g.nx + 2) * (g.nz + 2),
                 fz = (size_t)(g.nx + 2) * (g.ny + 2);
    const size_t len[6] = {fx, fx, fy, fy, fz, fz};
    size_t off = 0;
    for (int q = 0; q < 6; ++q) {
      check(c, mg::launch_fill<double>(c->faces[l] + off, (long long)len[q], c->face_b[q], nullptr),
            "face values");
      off += len[q];
    }
  }
  check(c, cudaStreamSynchronize(nullptr), "sync");
}

// Brackets one finest-level launch with events when timing is on.
struct KTimer {
  mg_ctx* c;
  int cls;
  cudaStream_t s;
  int slot = -1;
  KTimer(mg_ctx* c_, int cls_, bool finest, cudaStream_t s_) : c(c_), cls(cls_), s(s_) {
    if (!c->timing || !finest) return;
    const size_t k = c->pending_class.size();
    if (2 * k + 2 > c->events.size()) {
      if (c->events.size() >= 8192) return;  // pool full: stop timing this solve
      for (int q = 0; q < 256; ++q) {
        cudaEvent_t e;
        check(c, cudaEventCreate(&e), "cudaEventCreate");
        c->events.push_back(e);
      }
    }
    slot = (int)k;
    c->pending_class.push_back(cls);
    check(c, cudaEventRecord(c->events[2 * k], s), "cudaEventRecord");
  }
  ~KTimer() {
    if (slot >= 0) cudaEventRecord(c->events[2 * slot + 1], s);
  }
};

// After the solve's stream is synchronised: add the recorded durations.
void collect_times(mg_ctx* c) {
  for (size_t k = 0; k < c->pending_class.size(); ++k) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->events[2 * k], c->events[2 * k + 1]) == cudaSuccess) {
      c->kernel_ms[c->pending_class[k]] += ms;
      c->kernel_n[c->pending_class[k]] += 1;
    }
  }
  c->pending_class.clear();
}

// ---------------------------------------------------------------------------
// Cycles, templated on the level precision.

// Highest level index the single-CTA bottom solver covers (<= 16^3 cells).
int bottom_top(const mg_ctx* c) {
  if (!is_cubic(c)) return 0;  // the single-CTA bottom solver takes cubes only
  int t = 0;
  while (t + 1 < c->L && t + 1 < mg::kBottomLevels && level_n(c, t + 1) <= mg::kBottomTopN) ++t;
  return t;
}

template <typename T>
void launch_bottom_levels(mg_ctx* c, T** u, T** f, int top, const Bc* bcs, const Bc& hom, bool fmg,
                          cudaStream_t s) {
  int n[mg::kBottomLevels];
  double h[mg::kBottomLevels];
  for (int l = 0; l <= top; ++l) {
    n[l] = level_n(c, l);
    h[l] = level_h(c, l);
  }
  check(c, mg::launch_bottom<T>(u, f, n, h, bcs, hom, c->opts.omega, c->opts.pre, c->opts.post,
                                top, fmg, s),
        "bottom");
}

// COARSEST on level 0 (Sec. 2.3.2): one cell is solved exactly; a level of
// several cells (non-cubic grids) gets N_0,max red-black Gauss-Seidel sweeps
// (omega = 1) from 0, or from its current value when `keep` (FAS).
template <typename T>
void coarsest_solve(mg_ctx* c, T* u0, const T* f0, const Bc& bc, bool keep, cudaStream_t s) {
  const Grid g0 = level_grid(c, 0);
  const double h0 = level_h(c, 0);
  if (g0.cells() == 1) {
    check(c, mg::launch_coarsest<T>(f0, u0, h0, bc, s, keep), "coarsest");
    return;
  }
  if (!keep) check(c, mg::launch_fill<T>(u0, g0.cells(), T(0), s), "fill");
  const int nmax = std::max(g0.nx, std::max(g0.ny, g0.nz));
  for (int q = 0; q < nmax; ++q) {
    check(c, mg::launch_sor<T>(u0, f0, g0, h0, bc, 1.0, 0, s), "coarsest red");
    check(c, mg::launch_sor<T>(u0, f0, g0, h0, bc, 1.0, 1, s), "coarsest black");
  }
}

template <typename T>
struct Pyr {
  T** u;
  T** f;
};

template <typename T>
Pyr<T> pyr(mg_ctx* c);
template <>
Pyr<double> pyr<double>(mg_ctx* c) { return {c->u64, c->f64}; }
template <>
Pyr<float> pyr<float>(mg_ctx* c) { return {c->u32, c->f32}; }

template <typename T>
void smooth_steps(mg_ctx* c, Pyr<T> P, int l, const Bc& bc, int steps, bool zero_guess,
                  cudaStream_t s) {
  const Grid g = level_grid(c, l);
  const double h = level_h(c, l), om = c->opts.omega;
  if (zero_guess && steps == 0) {
    check(c, mg::launch_fill<T>(P.u[l], g.cells(), T(0), s), "fill");
    return;
  }
  const bool fin = (l == c->L - 1);
  for (int q = 0; q < steps; ++q) {
    {
      KTimer t(c, MG_K_SOR, fin, s);
      if (q == 0 && zero_guess)
        check(c, mg::launch_sor_red_zero<T>(P.u[l], P.f[l], g, h, om, s), "sor_red_zero");
      else
        check(c, mg::launch_sor<T>(P.u[l], P.f[l], g, h, bc, om, 0, s), "sor red");
    }
    KTimer t(c, MG_K_SOR, fin, s);
    check(c, mg::launch_sor<T>(P.u[l], P.f[l], g, h, bc, om, 1, s), "sor black");
  }
}

// Algorithm 1 on level l >= 1 with rule bc_top on level l and the homogeneous
// rule `hom` below.  zero_guess: u_l enters as 0 (coarse corrections).
template <typename T>
void vcycle(mg_ctx* c, Pyr<T> P, int l, const Bc& bc_top, const Bc& hom, bool zero_guess,
            cudaStream_t s);

// The same cycle on an FP32 level handled by the fused kernels: one kernel
// per leg, ping-ponging between the level's two buffers.
// Whether level l's down leg takes its planes by tensor copies: opts 1 where
// the kernel applies, 0 where the autotuner timed it faster, 2 never.
bool tma_level(const mg_ctx* c, int l, const Bc& bc, bool zero_guess) {
  if (c->opts.tensor_copies == 2 || !mg::down_tma_ok(level_grid(c, l), bc)) return false;
  return c->opts.tensor_copies == 1 || (zero_guess ? c->tma_down0[l] : c->tma_down[l]);
}

// The same for the up leg.
bool tma_up_level(const mg_ctx* c, int l, const Bc& bc) {
  if (c->opts.tensor_copies == 2 || !mg::up_tma_ok(level_grid(c, l), bc)) return false;
  return c->opts.tensor_copies == 1 || c->tma_up[l];
}

// Steps 5-7 of Algorithm 1 on FP32 level l in one pass: u32[l] plus the
// prolonged correction u32[l-1], smoothed into u32b[l].
cudaError_t launch_up(mg_ctx* c, int l, const Bc& bc, cudaStream_t s) {
  const Grid g = level_grid(c, l);
  const double h = level_h(c, l), om = c->opts.omega;
  if (tma_up_level(c, l, bc))
    return mg::launch_fused_up_tma(c->u32[l], c->u32b[l], c->f32[l], c->u32[l - 1], g, h, om,
                                   c->tma_cz_up[l], c->iflag + 1, s);
  return mg::launch_fused_up(c->u32[l], c->u32b[l], c->f32[l], c->u32[l - 1], g, h, bc, om, s,
                             c->cfg_up[l]);
}

// Steps 1-3 of Algorithm 1 on FP32 level l in one pass, into u32b[l] and
// f32[l-1] (the caller swaps the level's buffers).
cudaError_t launch_down(mg_ctx* c, int l, const Bc& bc, bool zero_guess, cudaStream_t s) {
  const Grid g = level_grid(c, l);
  const double h = level_h(c, l), om = c->opts.omega;
  if (tma_level(c, l, bc, zero_guess))
    return mg::launch_fused_down_tma(c->u32[l], c->u32b[l], c->f32[l], c->f32[l - 1], g, h, om,
                                     zero_guess,
                                     zero_guess ? c->tma_cz_down0[l] : c->tma_cz_down[l],
                                     c->iflag + 1, s);
  return mg::launch_fused_down(c->u32[l], c->u32b[l], c->f32[l], c->f32[l - 1], g, h, bc, om,
                               zero_guess, s, c->cfg_down[l]);
}

void vcycle_fused(mg_ctx* c, int l, const Bc& bc_top, const Bc& hom, bool zero_guess,
                  cudaStream_t s) {
  const Grid g = level_grid(c, l);
  const double h = level_h(c, l), om = c->opts.omega;
  const bool fin = (l == c->L - 1);
  auto swap_level = [&]() { std::swap(c->u32[l], c->u32b[l]); };
  const int pre = c->opts.pre, post = c->opts.post;
  bool zg = zero_guess;
  for (int q = 0; q + 1 < pre; ++q) {  // extra pre-smoothing steps of V(2,.)
    KTimer t(c, MG_K_SOR, fin, s);
    check(c, mg::launch_fused_smooth(c->u32[l], c->u32b[l], c->f32[l], g, h, bc_top, om, zg, s,
                                     c->cfg_smooth[l]),
          "fused smooth");
    swap_level();
    zg = false;
  }
  if (pre >= 1) {  // 1-3
    KTimer t(c, zg ? MG_K_FUSED_DOWN0 : MG_K_FUSED_DOWN, fin, s);
    check(c, launch_down(c, l, bc_top, zg, s), "fused down");
    swap_level();
  } else {
    if (zg) check(c, mg::launch_fill<float>(c->u32[l], g.cells(), 0.f, s), "fill");
    KTimer t(c, MG_K_DEFECT_RESTRICT, fin, s);
    check(c, mg::launch_defect_restrict<float>(c->u32[l], c->f32[l], c->f32[l - 1], g, h, bc_top,
                                               s),
          "defect_restrict");
  }
  Pyr<float> P = pyr<float>(c);
  if (l - 1 == 0)
    coarsest_solve<float>(c, P.u[0], P.f[0], hom, false, s);
  else if (l - 1 <= bottom_top(c))
    launch_bottom_levels<float>(c, P.u, P.f, l - 1, nullptr, hom, false, s);
  else
    vcycle<float>(c, P, l - 1, hom, hom, true, s);
  if (post >= 1) {  // 5-7
    {
      KTimer t(c, MG_K_FUSED_UP, fin, s);
      check(c, launch_up(c, l, bc_top, s), "fused up");
      swap_level();
    }
    for (int q = 1; q < post; ++q) {
      KTimer t(c, MG_K_SOR, fin, s);
      check(c, mg::launch_fused_smooth(c->u32[l], c->u32b[l], c->f32[l], g, h, bc_top, om, false,
                                       s, c->cfg_smooth[l]),
            "fused smooth");
      swap_level();
    }
  } else {
    KTimer t(c, MG_K_PROLONG, fin, s);
    check(c, mg::launch_prolong<float>(c->u32[l - 1], c->u32[l], g, hom, 0, 1, s), "prolong");
  }
}

// Steps 4.1-4.2 of Algorithm 1 below an FP32 level l: the coarse correction
// from the restricted defect in f32[l-1], into u32[l-1] (from zero).
void coarse_correction(mg_ctx* c, int l, const Bc& hom, cudaStream_t s) {
  Pyr<float> P = pyr<float>(c);
  if (l - 1 == 0)
    coarsest_solve<float>(c, P.u[0], P.f[0], hom, false, s);
  else if (l - 1 <= bottom_top(c))
    launch_bottom_levels<float>(c, P.u, P.f, l - 1, nullptr, hom, false, s);
  else
    vcycle<float>(c, P, l - 1, hom, hom, true, s);
}

// Whether `cycles` V(1,1) cycles on FP32 level l from a zero start can run as
// pairs: the first down leg, then the up leg of each cycle fused with the down
// leg of the next (temporal blocking of the smoother), then the last up leg.
bool pairs_ok(const mg_ctx* c, int l, const Bc& bc_top, const Bc& hom, int cycles) {
  const Grid g = level_grid(c, l);
  return cycles >= 2 && c->opts.pre == 1 && c->opts.post == 1 && c->u32b[l] &&
         mg::fused_ok(g, bc_top) && hom.kind == bc_top.kind && hom.fk == bc_top.fk &&
         mg::updown_ok(g, bc_top);
}

bool use_pairs(const mg_ctx* c) {
  return c->opts.leg_pairs == 1 || (c->opts.leg_pairs == 0 && c->pairs_faster);
}

// `cycles` V(1,1) cycles (Algorithm 1) on FP32 level l from a zero correction,
// with every up leg but the last fused with the next cycle's down leg: one
// pass reads u, f and the coarse correction and writes u and the next coarse
// right-hand side, where two passes would move u and f twice.
void vcycles_paired(mg_ctx* c, int l, const Bc& bc_top, const Bc& hom, int cycles,
                    cudaStream_t s) {
  const Grid g = level_grid(c, l);
  const double h = level_h(c, l), om = c->opts.omega;
  const bool fin = (l == c->L - 1);
  auto swap_level = [&]() { std::swap(c->u32[l], c->u32b[l]); };
  {
    KTimer t(c, MG_K_FUSED_DOWN0, fin, s);
    check(c, launch_down(c, l, bc_top, true, s), "fused down");
    swap_level();
  }
  coarse_correction(c, l, hom, s);
  for (int k = 1; k < cycles; ++k) {
    {
      KTimer t(c, MG_K_FUSED_UPDOWN, fin, s);
      check(c, mg::launch_fused_updown(c->u32[l], c->u32b[l], c->f32[l], c->u32[l - 1],
                                       c->f32[l - 1], g, h, bc_top, om, s, c->cfg_ud[l]),
            "fused up-down");
      swap_level();
    }
    coarse_correction(c, l, hom, s);
  }
  KTimer t(c, MG_K_FUSED_UP, fin, s);
  check(c, launch_up(c, l, bc_top, s), "fused up");
  swap_level();
}

template <typename T>
void vcycle(mg_ctx* c, Pyr<T> P, int l, const Bc& bc_top, const Bc& hom, bool zero_guess,
            cudaStream_t s) {
  const Grid g = level_grid(c, l);
  const double h = level_h(c, l);
  if constexpr (std::is_same<T, float>::value) {
    // the fused up leg synthesises the coarse correction's ghosts with the
    // level's own rule, so it serves levels whose coarse rule is the same
    if (c->u32b[l] && mg::fused_ok(g, bc_top) && hom.kind == bc_top.kind && hom.fk == bc_top.fk) {
      vcycle_fused(c, l, bc_top, hom, zero_guess, s);
      return;
    }
  }
  const bool fin = (l == c->L - 1);
  smooth_steps<T>(c, P, l, bc_top, c->opts.pre, zero_guess, s);                        // 1
  {
    KTimer t(c, MG_K_DEFECT_RESTRICT, fin, s);
    check(c, mg::launch_defect_restrict<T>(P.u[l], P.f[l], P.f[l - 1], g, h, bc_top, s),  // 2-3
          "defect_restrict");
  }
  if (l - 1 == 0)
    coarsest_solve<T>(c, P.u[0], P.f[0], hom, false, s);                               // 4.1
  else if (l - 1 <= bottom_top(c))
    launch_bottom_levels<T>(c, P.u, P.f, l - 1, nullptr, hom, false, s);                 // 4.2
  else
    vcycle<T>(c, P, l - 1, hom, hom, true, s);                                         // 4.2
  {
    KTimer t(c, MG_K_PROLONG, fin, s);
    check(c, mg::launch_prolong<T>(P.u[l - 1], P.u[l], g, hom, 0, 1, s), "prolong");    // 5-6
  }
  smooth_steps<T>(c, P, l, bc_top, c->opts.post, false, s);                            // 7
}

// Algorithm 2 with rule bcs[l] on every level.
template <typename T>
void fmg(mg_ctx* c, Pyr<T> P, const Bc* bcs, const Bc& hom, cudaStream_t s) {
  const int lb = bottom_top(c);
  for (int l = c->L - 1; l > lb; --l)
    check(c, mg::launch_restrict<T>(P.f[l], P.f[l - 1], level_grid(c, l), s), "restrict");
  if (lb > 0 || level_grid(c, 0).cells() == 1)
    launch_bottom_levels<T>(c, P.u, P.f, lb, bcs, hom, true, s);  // levels 0 .. lb
  else
    coarsest_solve<T>(c, P.u[0], P.f[0], bcs[0], false, s);
  for (int l = lb + 1; l < c->L; ++l) {
    {
      KTimer t(c, MG_K_FMG_PROLONG, l == c->L - 1, s);
      check(c, mg::launch_prolong<T>(P.u[l - 1], P.u[l], level_grid(c, l), bcs[l - 1], 1, 0, s),
            "fmg_prolong");
    }
    vcycle<T>(c, P, l, bcs[l], hom, false, s);
  }
}

// Algorithm 3 on level l >= 1 (FP64 path): every level solves the original
// equation with its own physical rule (bcs[l]); the coarse-grid correction
// psi - phi_bar is prolonged with the homogeneous rule.
void vcycle_fas(mg_ctx* c, int l, const Bc* bcs, const Bc& hom, cudaStream_t s) {
  Pyr<double> P = pyr<double>(c);
  const Grid g = level_grid(c, l), gc = level_grid(c, l - 1);
  const double h = level_h(c, l);
  const bool fin = (l == c->L - 1);
  smooth_steps<double>(c, P, l, bcs[l], c->opts.pre, false, s);                      // 1
  {
    KTimer t(c, MG_K_DEFECT_RESTRICT, fin, s);
    check(c, mg::launch_defect_restrict<double>(P.u[l], P.f[l], P.f[l - 1], g, h, bcs[l], s),
          "defect_restrict");                                                         // 2-3
  }
  check(c, mg::launch_restrict<double>(P.u[l], c->ur64[l - 1], g, s), "restrict phi");  // 4
  check(c, mg::launch_fas_rhs(c->ur64[l - 1], P.f[l - 1], P.u[l - 1], gc, level_h(c, l - 1),
                              bcs[l - 1], s),
        "fas rhs");                                                                   // 5
  if (l - 1 == 0)
    coarsest_solve<double>(c, P.u[0], P.f[0], bcs[0], true, s);                      // 6.1
  else
    vcycle_fas(c, l - 1, bcs, hom, s);                                                // 6.2
  check(c, mg::launch_sub(P.u[l - 1], c->ur64[l - 1], gc.cells(), s), "fas correction");  // 7
  {
    KTimer t(c, MG_K_PROLONG, fin, s);
    check(c, mg::launch_prolong<double>(P.u[l - 1], P.u[l], g, hom, 0, 1, s), "prolong");  // 8-9
  }
  smooth_steps<double>(c, P, l, bcs[l], c->opts.post, false, s);                     // 10
}

// Algorithm 2 with Algorithm 3 as the cycle, every level with its own rule.
void fmg_fas(mg_ctx* c, const Bc* bcs, const Bc& hom, cudaStream_t s) {
  Pyr<double> P = pyr<double>(c);
  for (int l = c->L - 1; l > 0; --l)
    check(c, mg::launch_restrict<double>(P.f[l], P.f[l - 1], level_grid(c, l), s), "restrict");
  coarsest_solve<double>(c, P.u[0], P.f[0], bcs[0], false, s);
  for (int l = 1; l < c->L; ++l) {
    {
      KTimer t(c, MG_K_FMG_PROLONG, l == c->L - 1, s);
      check(c, mg::launch_prolong<double>(P.u[l - 1], P.u[l], level_grid(c, l), bcs[l - 1], 1, 0,
                                          s),
            "fmg_prolong");
    }
    vcycle_fas(c, l, bcs, hom, s);
  }
}

// Fixed-order sums of squares -> host.
double read_scalar(mg_ctx* c, int slot, cudaStream_t s) {
  check(c, cudaMemcpyAsync(c->pinned + slot, c->scal + slot, sizeof(double),
                           cudaMemcpyDeviceToHost, s),
        "read norm");
  check(c, cudaStreamSynchronize(s), "sync");
  return c->pinned[slot];
}

struct StopRule {
  double tol, stall, d0 = -1.0, prev = -1.0;
  int stalls = 0;
  // Returns MG_OK to stop successfully, a failure status to stop, or -1 to go on.
  int decide(double r, int cycles_done, int max_cycles, int n_hist, int hist_cap) {
    if (d0 < 0) d0 = r;
    if (std::isnan(r) || std::isinf(r) || r > 10.0 * d0) return MG_ERR_DIVERGED;
    if (r < tol) return MG_OK;
    if (stalls >= 2) return tol == 0.0 ? MG_OK : MG_ERR_NOT_CONVERGED;
    if (cycles_done >= max_cycles || n_hist >= hist_cap) return MG_ERR_NOT_CONVERGED;
    return -1;
  }
  void record(double r) {
    if (prev >= 0) stalls = (r > stall * prev) ? stalls + 1 : 0;
    prev = r;
  }
};

// Source, mean removal, norm of f, and the open-boundary values.
double prepare_source(mg_ctx* c, const double* rho, double four_pi_G, double* f_fin,
                      bool all_levels_faces, cudaStream_t s) {
  const int F = c->L - 1;
  const Grid gf = level_grid(c, F);
  const long long N = gf.cells();
  const int nb = mg::reduce_blocks(N);
  {
    KTimer t(c, MG_K_SOURCE, true, s);
    check(c, mg::launch_source(rho, f_fin, N, four_pi_G, c->partials, s), "source");
  }
  if (mean_free(c))
    check(c, mg::launch_subtract_mean(f_fin, N, c->partials, nb, c->scal + 40, s), "subtract_mean");
  check(c, mg::launch_sum<double>(f_fin, N, 1, c->partials, s), "sum f^2");
  check(c, mg::launch_finish_sum(c->partials, nb, c->scal + 0, s), "finish f^2");
  if (c->bc_kind == MG_BC_OPEN) {
    int nbm = 0;
    check(c, mg::launch_raw_moments(rho, gf, c->h, c->partials, &nbm, s), "moments");
    check(c, mg::launch_moments_finish(c->partials, nbm, c->h, c->opts.lmax, c->opts.use_com,
                                       c->opts.origin, c->scal + 2, s),
          "moments_finish");
    const double G = four_pi_G / (4.0 * 3.14159265358979323846);
    for (int l = all_levels_faces ? 0 : F; l <= F; ++l)
      check(c, mg::launch_open_faces(level_grid(c, l), level_h(c, l), c->scal + 2, c->opts.lmax,
                                     G, c->faces[l], s),
            "open_faces");
  }
  return std::sqrt(read_scalar(c, 0, s) / (double)N);
}

void remove_mean(mg_ctx* c, double* u, cudaStream_t s) {
  if (!mean_free(c)) return;
  const long long N = level_grid(c, c->L - 1).cells();
  check(c, mg::launch_sum<double>(u, N, 0, c->partials, s), "sum phi");
  check(c, mg::launch_subtract_mean(u, N, c->partials, mg::reduce_blocks(N), c->scal + 40, s),
        "phi mean");
}

double defect_rms(mg_ctx* c, const double* u, const double* f, const Bc& bc, cudaStream_t s) {
  const int F = c->L - 1;
  const Grid g = level_grid(c, F);
  const int nb = mg::reduce_blocks(g.cells());
  {
    KTimer t(c, MG_K_DEFECT_NORM, true, s);
    check(c, mg::launch_defect<double>(u, f, nullptr, g, level_h(c, F), bc, c->partials, s),
          "defect norm");
  }
  check(c, mg::launch_finish_sum(c->partials, nb, c->scal + 1, s), "finish d^2");
  return std::sqrt(read_scalar(c, 1, s) / (double)g.cells());
}

// The rule of the coarse correction levels below a level with rule `top`:
// its homogeneous counterpart, or with coarse_literal zero fixed values on
// zero-gradient faces too (Sec. 2.3.6 taken word for word).
Bc correction_bc(const mg_ctx* c, const Bc& top) {
  Bc z = mg::homogeneous(top);
  if (!c->opts.coarse_literal) return z;
  if (z.kind == mg::BC_ZEROGRAD) return Bc{mg::BC_FIXED, 0.0, nullptr};
  if (z.kind == mg::BC_MIXED) {
    for (int q = 0; q < 6; ++q)
      if (mg::face_kind(z, q) == mg::BC_ZEROGRAD)
        z.fk = (z.fk & ~(3 << (2 * q))) | (mg::BC_FIXED << (2 * q));
    z = mg::collapse_homogeneous(z);
  }
  return z;
}

mg_status solve_fp64(mg_ctx* c, const double* rho, double four_pi_G, double tol, double* phi,
                     double* gacc, double* hist, int hist_cap, int* n_hist, cudaStream_t s) {
  const int F = c->L - 1;
  if (c->host_rho)
    check(c, cudaMemcpyAsync(const_cast<double*>(rho), c->host_rho,
                             sizeof(double) * level_grid(c, F).cells(), cudaMemcpyHostToDevice, s),
          "H2D rho");
  c->u64[F] = phi;
  Pyr<double> P = pyr<double>(c);
  double fnorm = prepare_source(c, rho, four_pi_G, c->f64[F], true, s);
  Bc bcs[kMaxLevels];
  for (int l = 0; l < c->L; ++l) bcs[l] = physical_bc(c, l);
  const Bc hom = correction_bc(c, bcs[F]);
  const bool fas = c->opts.fas != 0;
  if (c->opts.mode_fmg) {
    if (fas) fmg_fas(c, bcs, hom, s);
    else fmg<double>(c, P, bcs, hom, s);
  }
  double dn = defect_rms(c, phi, c->f64[F], bcs[F], s);
  if (fnorm == 0.0) fnorm = dn > 0.0 ? dn : 1.0;
  StopRule rule{tol, c->opts.stall_ratio};
  int n = 0, st = -1;
  double r = dn / fnorm;
  hist[n++] = r;
  rule.record(r);
  for (int cyc = 0;; ++cyc) {
    st = rule.decide(r, cyc, c->opts.max_cycles, n, hist_cap);
    if (st >= 0) break;
    if (fas) vcycle_fas(c, F, bcs, hom, s);
    else vcycle<double>(c, P, F, bcs[F], hom, false, s);
    r = defect_rms(c, phi, c->f64[F], bcs[F], s) / fnorm;
    hist[n++] = r;
    rule.record(r);
  }
  remove_mean(c, phi, s);
  if (gacc) {
    KTimer t(c, MG_K_GRAVITY, true, s);
    check(c, mg::launch_gravity(phi, gacc, level_grid(c, F), c->h, bcs[F], s), "gravity");
  }
  *n_hist = n;
  c->u64[F] = nullptr;
  return (mg_status)st;
}

// FP32 multigrid solve of L e = r into u32[L-1], with r already in f32[L-1]:
// rule `hom` (the homogeneous rule of the finest level) for e itself and in
// FMG, `coarse` for the corrections of e on the levels below.
void inner_solve_launches(mg_ctx* c, const Bc& hom, const Bc& coarse, int cycles,
                          cudaStream_t s) {
  const int F = c->L - 1;
  Pyr<float> P = pyr<float>(c);
  Bc bcs[kMaxLevels];
  for (int l = 0; l < c->L; ++l) bcs[l] = hom;
  if (c->opts.inner_fmg) {
    fmg<float>(c, P, bcs, coarse, s);
  } else if (use_pairs(c) && pairs_ok(c, F, hom, coarse, cycles)) {
    vcycles_paired(c, F, hom, coarse, cycles, s);
    return;
  } else {
    vcycle<float>(c, P, F, hom, coarse, true, s);
  }
  for (int q = 1; q < cycles; ++q) vcycle<float>(c, P, F, hom, coarse, false, s);
}

void drop_inner_graph(mg_ctx* c) {
  for (auto& ig : c->inner) {
    if (ig.exec) cudaGraphExecDestroy(ig.exec);
    ig.exec = nullptr;
    ig.runs = 0;
  }
}

// V-cycles (or FMG and the V-cycles after it) of the inner solve of outer
// iteration `it`.
int inner_count(const mg_ctx* c, int it) {
  return (it == 0 && c->opts.first_cycles > 0) ? c->opts.first_cycles : 1 + c->opts.inner_cycles;
}

// The inner solve of `cycles` V-cycles, from its second run with that count
// on as one CUDA graph launch (not while per-kernel timing is on, on the
// legacy default stream, or inside a capture the caller started).  The
// launches are the same every outer iteration: the same kernels, shapes and
// buffers.
void inner_solve(mg_ctx* c, const Bc& hom, const Bc& coarse, int cycles, cudaStream_t s) {
  mg_ctx::InnerGraph& ig = c->inner[cycles == 1 + c->opts.inner_cycles ? 0 : 1];
  if (ig.exec && !c->timing) {
    check(c, cudaGraphLaunch(ig.exec, s), "inner solve graph");
    mg::g_launches += ig.launches;
    return;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const bool capture = !c->timing && ig.runs >= 1 && s != nullptr &&
                       cudaStreamIsCapturing(s, &cs) == cudaSuccess &&
                       cs == cudaStreamCaptureStatusNone;
  ++ig.runs;
  if (!capture) {
    inner_solve_launches(c, hom, coarse, cycles, s);
    return;
  }
  check(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
  const long long before = mg::g_launches;
  cudaGraph_t graph = nullptr;
  try {
    inner_solve_launches(c, hom, coarse, cycles, s);
  } catch (const Fail&) {
    cudaStreamEndCapture(s, &graph);
    if (graph) cudaGraphDestroy(graph);
    throw;
  }
  check(c, cudaStreamEndCapture(s, &graph), "end capture");
  const cudaError_t e = cudaGraphInstantiate(&ig.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    ig.exec = nullptr;
    check(c, e, "instantiate inner solve graph");
  }
  ig.launches = mg::g_launches - before;
  check(c, cudaGraphLaunch(ig.exec, s), "inner solve graph");
}

mg_status solve_mixed(mg_ctx* c, const double* rho, double four_pi_G, double tol, double* phi,
                      double* gacc, double* hist, int hist_cap, int* n_hist, cudaStream_t s) {
  const int F = c->L - 1;
  const Grid g = level_grid(c, F);
  const long long N = g.cells();
  const int nb = mg::reduce_blocks(N);
  double* f = c->f64[F];
  Bc bc = physical_bc(c, F);
  // one fixed value b on every face, from an FMG start: solve for phi - b,
  // whose faces are zero-fixed (L_h of a constant is zero with the ghosts
  // 2b - phi, cell by cell), and add b at the end -- the zero-value path, and
  // no bits of the fixed-point scale spent on the offset
  const double b_shift =
      (bc.kind == mg::BC_FIXED && bc.value != 0.0 && c->opts.mode_fmg != 0) ? bc.value : 0.0;
  if (b_shift != 0.0) bc.value = 0.0;
  const Bc hom = mg::homogeneous(bc);
  const Bc coarse = correction_bc(c, bc);
  const bool fx = c->opts.outer_fixed != 0 && c->fxbuf != nullptr;
  const bool has_mean = mean_free(c);
  bool zero_values = bc.kind == mg::BC_PERIODIC || bc.kind == mg::BC_ZEROGRAD ||
                     (bc.kind == mg::BC_FIXED && bc.value == 0.0);
  if (bc.kind == mg::BC_MIXED) {
    zero_values = true;
    for (int q = 0; q < 6; ++q)
      if (mg::face_kind(bc, q) == mg::BC_FIXED && c->face_b[q] != 0.0) zero_values = false;
  }
  // From phi = 0 with a rule whose boundary values are 0, L phi = 0 and the
  // first residual is f itself.  On that path (with the fixed-point outer
  // loop) f is never stored as doubles: one pass over rho gives its sum (the
  // mean of f) and maximum, a second writes r32 = (4 pi G rho - mean) * scale
  // with its norm and maximum, and the integer h^2 f is formed from rho when
  // the scale 2^S is known.  Few FP64 operations per cell: on this GPU they,
  // not the bytes, would bound these passes.
  const bool fast = fx && c->opts.mode_fmg && zero_values;
  // open rule from an FMG start: begin from the expansion's monopole and dipole
  const bool open_guess = c->bc_kind == MG_BC_OPEN && c->opts.mode_fmg != 0;

  if (c->host_rho && !fast)
    check(c, cudaMemcpyAsync(const_cast<double*>(rho), c->host_rho, sizeof(double) * N,
                             cudaMemcpyHostToDevice, s),
          "H2D rho");
  double mu = 0.0;     // mean of f (fast path: not subtracted in memory)
  double mf = -1.0;    // max |f - mean| when known
  double fnorm, scale, rn;
  if (fast) {
    {
      KTimer t(c, MG_K_SOURCE, true, s);
      if (c->host_rho)  // rho arrives from host memory in this pass, which leaves the device copy
        check(c, mg::launch_rho_stats_copy(c->host_rho, const_cast<double*>(rho), N, c->partials,
                                           c->scal + 0, s),
              "source stats");
      else
        check(c, mg::launch_rho_stats(rho, N, c->partials, c->scal + 0, s), "source stats");
    }
    // mu and the scale (1 / bound on |f - mean|) on the device: the host
    // learns them, with the first residual's norm and maximum, in the first
    // outer iteration's read (no round trip before the first inner solve)
    check(c, mg::launch_source_scale(c->scal + 0, N, four_pi_G, has_mean, c->scal + 32, s),
          "source scale");
    check(c, mg::launch_rho_to_r32(rho, c->f32[F], N, 0.0, 0.0, c->partials, c->scal + 0, s,
                                   c->scal + 34),
          "r = f - mean");
    fnorm = scale = rn = -1.0;  // known after the first inner solve
  } else {
    fnorm = prepare_source(c, rho, four_pi_G, f, false, s);
    if (open_guess) {
      // the expansion's monopole and dipole as the start: the first residual
      // then has no boundary layer from the face potentials
      const double G = four_pi_G / (4.0 * 3.14159265358979323846);
      check(c, mg::launch_open_guess(phi, g, c->h, c->scal + 2, G, s), "open start");
    } else if (c->opts.mode_fmg) {
      check(c, mg::launch_fill<double>(phi, N, 0.0, s), "zero phi");
    }
    // r = f - L phi, scaled into FP32 so that its RMS is about 1.
    scale = fnorm > 0.0 ? 1.0 / fnorm : 1.0;
    if (c->opts.mode_fmg && zero_values) {
      check(c, mg::launch_scale_to_f32(f, c->f32[F], N, scale, s), "r = f");
      rn = fnorm;
    } else {
      check(c, mg::launch_outer_residual(phi, f, c->f32[F], g, c->h, bc, scale, c->partials, s),
            "outer residual");
      check(c, mg::launch_finish_sum(c->partials, nb, c->scal + 1, s), "finish r^2");
      rn = std::sqrt(read_scalar(c, 1, s) / (double)N);
    }
    if (fnorm == 0.0) {
      fnorm = rn > 0.0 ? rn : 1.0;
      scale = 1.0 / fnorm;
      if (rn > 0.0) {
        check(c, mg::launch_outer_residual(phi, f, c->f32[F], g, c->h, bc, scale, c->partials, s),
              "outer residual");
      }
    }
  }
  StopRule rule{tol, c->opts.stall_ratio};
  int n = 0, st = -1;
  double two_S = 1.0;  // 2^S of the fixed-point representation
  int S = 0;
  bool in_fx = false;  // phi and f hold integers
  bool phi_zero = false;  // the integer phi is all zero (FMG start): not read
  long long* cur = reinterpret_cast<long long*>(phi);  // integer phi (in phi's own storage)
  long long* alt = c->fxbuf;
  // per-block exact sums of the integer phi, (hi, lo) pairs
  long long* psum = reinterpret_cast<long long*>(c->partials + c->partials_cap);
  int nbs = 0;
  const long long* FX = reinterpret_cast<const long long*>(f);
  for (int it = 0;; ++it) {
    if (rn == 0.0) {  // exact already (zero source with a homogeneous rule)
      hist[n++] = 0.0;
      st = MG_OK;
      break;
    }
    inner_solve(c, hom, coarse, inner_count(c, it), s);
    if (fast && it == 0) {
      // one read for the source's scalars, the first residual's norm and
      // maximum, and max |e| after the first inner solve
      check(c, mg::launch_absmax<float>(c->u32[F], N, c->partials, c->scal + 50, s), "max |e|");
      check(c, cudaMemsetAsync(c->scal + 52, 0, sizeof(double), s), "zero");
      check(c, cudaMemcpyAsync(c->pinned, c->scal, 64 * sizeof(double), cudaMemcpyDeviceToHost,
                               s),
            "read scalars");
      check(c, cudaStreamSynchronize(s), "sync");
      mu = c->pinned[32];
      scale = c->pinned[33];
      fnorm = std::sqrt(c->pinned[0] / (double)N) / scale;
      mf = c->pinned[1] / scale;
      rn = fnorm;
      if (fnorm == 0.0) {  // zero source: phi = 0 (the inner solve ran on zeros)
        check(c, mg::launch_fill<double>(phi, N, 0.0, s), "zero phi");
        hist[n++] = 0.0;
        st = MG_OK;
        break;
      }
    }
    const double old_scale = scale;
    scale = 1.0 / rn;  // the next residual is scaled by the current one's size
    if (!fx) {
      {
        KTimer t(c, MG_K_CORRECT, true, s);
        check(c, mg::launch_correct(phi, c->u32[F], N, 1.0 / old_scale, s), "correct");
      }
      KTimer t(c, MG_K_OUTER_RESIDUAL, true, s);
      check(c, mg::launch_outer_residual(phi, f, c->f32[F], g, c->h, bc, scale, c->partials, s),
            "outer residual");
      check(c, mg::launch_finish_sum(c->partials, nb, c->scal + 1, s), "finish r^2");
      rn = std::sqrt(read_scalar(c, 1, s) / (double)N);
    } else {
      if (it == 0) {
        // S such that |phi| < 2^55 and |h^2 f| < 2^58 on the integer grid;
        // phi after this step is at most max|phi_0| + max|e| / scale.
        phi_zero = c->opts.mode_fmg != 0 && !open_guess;
        if (!fast) {  // (the fast path read these with its scalars)
          check(c, mg::launch_absmax<float>(c->u32[F], N, c->partials, c->scal + 50, s),
                "max |e|");
          if (mf < 0.0)
            check(c, mg::launch_absmax<double>(f, N, c->partials, c->scal + 51, s), "max |f|");
          if (!phi_zero)
            check(c, mg::launch_absmax<double>(phi, N, c->partials, c->scal + 52, s),
                  "max |phi|");
          else
            check(c, cudaMemsetAsync(c->scal + 52, 0, sizeof(double), s), "zero");
          check(c, cudaMemcpyAsync(c->pinned + 50, c->scal + 50, 3 * sizeof(double),
                                   cudaMemcpyDeviceToHost, s),
                "read max");
          check(c, cudaStreamSynchronize(s), "sync");
        }
        check(c, cudaMemsetAsync(c->iflag, 0, sizeof(int), s), "clear flag");
        const double mphi = c->pinned[52] + c->pinned[50] / old_scale;
        const double mfh = (mf >= 0.0 ? mf : c->pinned[51]) * c->h * c->h;
        double lim = 0.0;
        if (mphi > 0.0) lim = std::ldexp(1.0, 55) / mphi;
        if (mfh > 0.0 && (lim == 0.0 || std::ldexp(1.0, 58) / mfh < lim))
          lim = std::ldexp(1.0, 58) / mfh;
        if (lim == 0.0) lim = std::ldexp(1.0, 55);
        int e2 = 0;
        std::frexp(lim, &e2);
        S = e2 - 1;
        two_S = std::ldexp(1.0, S);  // largest power of two <= lim
        const double c2 = c->h * c->h * two_S;
        if (fast)
          check(c, mg::launch_rho_to_fx(rho, reinterpret_cast<long long*>(f), N, four_pi_G * c2,
                                        mu * c2, s),
                "h^2 f -> fixed point");
        else
          check(c, mg::launch_f64_to_fx(f, N, 0.0, c2, s), "h^2 f -> fixed point");
        if (!phi_zero) check(c, mg::launch_f64_to_fx(phi, N, 0.0, two_S, s), "phi -> fixed point");
        in_fx = true;
      }
      {
        KTimer t(c, MG_K_OUTER_RESIDUAL, true, s);
        check(c, mg::launch_fx_step(phi_zero ? nullptr : cur, alt, c->u32[F],
                                    (float)(two_S / old_scale), FX, c->f32[F], g, bc, two_S,
                                    (float)(scale / (c->h * c->h * two_S)), c->partials,
                                    c->partials_cap, c->iflag, &nbs, s, c->fx_cz,
                                    has_mean ? psum : nullptr),
              "fixed-point step");
      }
      phi_zero = false;
      std::swap(cur, alt);
      check(c, mg::launch_finish_sum(c->partials, nbs, c->scal + 1, s), "finish r^2");
      rn = std::sqrt(read_scalar(c, 1, s) / (double)N) / scale;
    }
    const double r = rn / fnorm;
    hist[n++] = r;
    rule.record(r);
    st = rule.decide(r, it + 1, c->opts.max_cycles, n, hist_cap);
    if (st >= 0) break;
  }
  int late = 0;  // iflag[1]
  if (in_fx) {
    // phi = (PHI - M) 2^-S, M the integers' mean (periodic / zero gradient)
    // rounded to an integer, from the last step's exact integer sums
    const long long* mean = nullptr;
    if (has_mean) {
      check(c, mg::launch_finish_fx_sum(psum, nbs, N, c->scal + 56, s), "finish sum phi");
      mean = reinterpret_cast<const long long*>(c->scal + 57);
    }
    if (gacc) {
      // phi and g from the integers in one pass; it reads neighbours, so it
      // writes phi into the free integer buffer when the integers are in phi
      const bool alias = cur == reinterpret_cast<long long*>(phi);
      double* out = alias ? reinterpret_cast<double*>(alt) : phi;
      KTimer t(c, MG_K_GRAVITY, true, s);
      check(c, mg::launch_fx_finish_gravity(cur, out, gacc, g, bc, c->h, S, mean, s),
            "fixed point -> phi, g");
      if (alias)
        check(c, cudaMemcpyAsync(phi, out, sizeof(double) * N, cudaMemcpyDeviceToDevice, s),
              "copy phi");
    } else {
      // straight into the caller's pinned host phi when there is one
      double* out = c->host_phi ? c->host_phi : phi;
      check(c, mg::launch_fx_to_f64(cur, out, N, S, mean, s), "fixed point -> phi");
      c->host_phi_written = c->host_phi != nullptr;
      if (b_shift != 0.0) check(c, mg::launch_add_const(out, N, b_shift, s), "phi + b");
    }
    if (gacc && b_shift != 0.0) check(c, mg::launch_add_const(phi, N, b_shift, s), "phi + b");
    // both flags in one read: [0] overflow, [1] a tensor copy that was late
    int flags[2] = {0, 0};
    check(c, cudaMemcpyAsync(c->pinned + 60, c->iflag, 2 * sizeof(int), cudaMemcpyDeviceToHost, s),
          "read flags");
    check(c, cudaStreamSynchronize(s), "sync");
    std::memcpy(flags, c->pinned + 60, 2 * sizeof(int));
    late = flags[1];
    if (flags[0]) {
      c->err = "fixed-point outer loop: |phi| passed 2^60 (the solve diverged)";
      st = MG_ERR_DIVERGED;
    }
  } else {
    remove_mean(c, phi, s);
    if (gacc) {
      KTimer t(c, MG_K_GRAVITY, true, s);
      check(c, mg::launch_gravity(phi, gacc, g, c->h, bc, s), "gravity");
    }
    if (b_shift != 0.0) check(c, mg::launch_add_const(phi, N, b_shift, s), "phi + b");
  }
  bool tma = false;
  for (int l = 1; l < c->L; ++l)
    tma = tma || tma_level(c, l, hom, false) || tma_level(c, l, hom, true) ||
          tma_up_level(c, l, hom);
  if (tma && !in_fx) {  // not read with the overflow flag above
    check(c, cudaMemcpyAsync(c->pinned + 61, c->iflag + 1, sizeof(int), cudaMemcpyDeviceToHost, s),
          "read flag");
    check(c, cudaStreamSynchronize(s), "sync");
    std::memcpy(&late, c->pinned + 61, sizeof(int));
  }
  if (tma) {  // a leg whose tensor copies did not land in time raised iflag[1]
    if (late) {
      check(c, cudaMemsetAsync(c->iflag + 1, 0, sizeof(int), s), "clear flag");
      c->err = "fused leg: a tensor copy did not land in time";
      st = MG_ERR_TIMEOUT;
    }
  }
  *n_hist = n;
  return (mg_status)st;
}

mg_status validate_opts(const mg_opts& o) {
  if (o.prec != MG_FP64 && o.prec != MG_MIXED) return MG_ERR_ARG;
  if (o.pre < 0 || o.pre > 2 || o.post < 0 || o.post > 2 || o.pre + o.post == 0) return MG_ERR_ARG;
  if (!(o.omega > 0.0 && o.omega < 2.0)) return MG_ERR_ARG;
  if (o.max_cycles < 0 || o.lmax < 0 || o.lmax > 4) return MG_ERR_ARG;
  if (o.inner_cycles < 0 || o.inner_cycles > 64) return MG_ERR_ARG;
  if (o.first_cycles < 0 || o.first_cycles > 65) return MG_ERR_ARG;
  if (o.outer_fixed != 0 && o.outer_fixed != 1) return MG_ERR_ARG;
  if (o.fas != 0 && (o.fas != 1 || o.prec != MG_FP64)) return MG_ERR_ARG;
  if (o.coarse_literal != 0 && o.coarse_literal != 1) return MG_ERR_ARG;
  if (o.leg_pairs < 0 || o.leg_pairs > 2) return MG_ERR_ARG;
  if (o.batch_small != 0 && o.batch_small != 1) return MG_ERR_ARG;
  if (o.tensor_copies < 0 || o.tensor_copies > 2) return MG_ERR_ARG;
  if (!(o.stall_ratio > 0.0)) return MG_ERR_ARG;
  for (int r : o.reserved)
    if (r != 0) return MG_ERR_ARG;
  return MG_OK;
}

// ---------------------------------------------------------------------------
// Autotuner of launch shapes.  Each candidate runs on the context's own
// buffers (contents irrelevant: the kernels' cost does not depend on the
// values) a few times between CUDA events on the solve's stream; the fastest
// wins.  Results are kept per process, keyed by device and problem shape, so
// every context of that shape launches identically (and gives identical
// bits); with MG_TUNE_CACHE naming a file they also persist across runs.
enum TuneKind {
  TUNE_DOWN = 0,
  TUNE_UP = 1,
  TUNE_SMOOTH = 2,
  TUNE_FX = 3,
  TUNE_UD = 4,      // shape of the fused up-down pass
  TUNE_UD_WIN = 5,  // cz = 1 when that pass beat the two legs it replaces
  TUNE_TMA = 7,     // tx / cz / ty = 1: tensor copies won for the down leg from zero / the
                    // down leg from a nonzero start / the up leg
  TUNE_TMA_CZ = 8   // tx / cz / ty: those three legs' planes per CTA with tensor copies
};

struct TuneKey {
  int sms, major, minor, kind, nx, ny, nz, periodic;
  bool operator<(const TuneKey& o) const {
    return std::tie(sms, major, minor, kind, nx, ny, nz, periodic) <
           std::tie(o.sms, o.major, o.minor, o.kind, o.nx, o.ny, o.nz, o.periodic);
  }
};

std::mutex g_tune_mu;
std::map<TuneKey, mg::TileCfg> g_tune;
bool g_tune_loaded = false;

void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("MG_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* fp = std::fopen(path, "r");
  if (!fp) return;
  TuneKey k;
  mg::TileCfg v;
  while (std::fscanf(fp, "%d %d %d %d %d %d %d %d %d %d %d", &k.sms, &k.major, &k.minor, &k.kind,
                     &k.nx, &k.ny, &k.nz, &k.periodic, &v.tx, &v.cz, &v.ty) == 11)
    g_tune[k] = v;
  std::fclose(fp);
}

void tune_store_locked(const TuneKey& k, mg::TileCfg v) {
  g_tune[k] = v;
  const char* path = std::getenv("MG_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* fp = std::fopen(path, "a");
  if (!fp) return;
  std::fprintf(fp, "%d %d %d %d %d %d %d %d %d %d %d\n", k.sms, k.major, k.minor, k.kind, k.nx,
               k.ny, k.nz, k.periodic, v.tx, v.cz, v.ty);
  std::fclose(fp);
}

// Milliseconds of `reps` launches of `run` after one untimed one; before each
// timed launch the L2 cache is flushed by writing `flush` (when given), so
// that every launch reads its inputs from HBM as inside a solve.
template <typename Run>
float time_launches(mg_ctx* c, cudaStream_t s, int reps, void* flush, size_t flush_bytes,
                    Run run) {
  check(c, run(), "autotune launch");
  cudaEvent_t a, b;
  check(c, cudaEventCreate(&a), "cudaEventCreate");
  check(c, cudaEventCreate(&b), "cudaEventCreate");
  float total = 0.f;
  for (int q = 0; q < reps; ++q) {
    if (flush) check(c, cudaMemsetAsync(flush, q & 1, flush_bytes, s), "flush L2");
    check(c, cudaEventRecord(a, s), "record");
    check(c, run(), "autotune launch");
    check(c, cudaEventRecord(b, s), "record");
    check(c, cudaEventSynchronize(b), "sync");
    float ms = 0.f;
    check(c, cudaEventElapsedTime(&ms, a, b), "elapsed");
    total += ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return total;
}

void autotune(mg_ctx* c, cudaStream_t s) {
  cudaDeviceProp prop;
  check(c, cudaGetDeviceProperties(&prop, c->device), "cudaGetDeviceProperties");
  const Bc hom = mg::homogeneous(Bc{c->bc_kind, c->opts.fixed_value, nullptr, c->face_mask});
  // the kernels' periodic axes: 1 all (one rule), 0 none (one rule), 8 + the
  // periodic-axis mask for a rule per face
  int periodic = hom.kind == mg::BC_PERIODIC ? 1 : 0;
  if (hom.kind == mg::BC_MIXED) {
    periodic = 8;
    for (int a = 0; a < 3; ++a)
      if (mg::face_kind(hom, 2 * a) == mg::BC_PERIODIC) periodic += 1 << a;
  }
  const double om = c->opts.omega;
  const int F = c->L - 1;
  const int reps = 5;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  tune_load_locked();
  // a buffer twice the L2 size to flush it between timed launches (skipped
  // if it cannot be had)
  const size_t flush_bytes = 2 * (size_t)prop.l2CacheSize;
  void* flush = nullptr;
  if (cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
    cudaGetLastError();
    flush = nullptr;
  }
  struct FreeFlush {
    void* p;
    ~FreeFlush() {
      if (p) cudaFree(p);
    }
  } free_flush{flush};
  if (c->opts.prec == MG_MIXED) {
    for (int l = 1; l <= F; ++l) {
      const Grid g = level_grid(c, l);
      if (!c->u32b[l] || !mg::fused_ok(g, hom)) continue;
      for (int z : {0, 1, 2}) {  // zero-fill the level's buffers once
        float* buf = z == 0 ? c->u32[l] : z == 1 ? c->u32b[l] : c->f32[l];
        check(c, cudaMemsetAsync(buf, 0, sizeof(float) * g.cells(), s), "zero");
      }
      check(c, cudaMemsetAsync(c->u32[l - 1], 0, sizeof(float) * level_grid(c, l - 1).cells(), s),
            "zero");
      const double h = level_h(c, l);
      for (int kind : {TUNE_DOWN, TUNE_UP, TUNE_SMOOTH}) {
        if (kind == TUNE_SMOOTH && c->opts.pre < 2 && c->opts.post < 2) continue;
        const TuneKey key{prop.multiProcessorCount, prop.major, prop.minor, kind, g.nx, g.ny, g.nz,
                          periodic};
        mg::TileCfg best;
        auto hit = g_tune.find(key);
        if (hit != g_tune.end()) {
          best = hit->second;
        } else {
          float best_ms = 1e30f;
          for (int cand_i = 0; cand_i < 36; ++cand_i) {
            {
              const int tx = (cand_i & 1) ? 64 : 32, ty = (cand_i & 2) ? 32 : 16;
              // 8, 16, ..., 64 planes: the chunks that are not powers of two
              // even out the last wave of CTAs on some grids; 4 planes halve
              // the chain of plane steps of a CTA on the small levels, where
              // that chain, not the bytes, sets a launch's time
              const int cz = cand_i < 32 ? 8 * (1 + (cand_i >> 2)) : 4;
              const mg::TileCfg cand{tx, cz, ty};
              if (cz > g.nz || !mg::fused_cfg_ok(g, cand)) continue;
              const float ms = time_launches(c, s, reps, flush, flush_bytes, [&]() {
                if (kind == TUNE_DOWN)
                  return mg::launch_fused_down(c->u32[l], c->u32b[l], c->f32[l], c->f32[l - 1], g,
                                               h, hom, om, false, s, cand);
                if (kind == TUNE_UP)
                  return mg::launch_fused_up(c->u32[l], c->u32b[l], c->f32[l], c->u32[l - 1], g, h,
                                             hom, om, s, cand);
                return mg::launch_fused_smooth(c->u32[l], c->u32b[l], c->f32[l], g, h, hom, om,
                                               false, s, cand);
              });
              if (ms < best_ms) {
                best_ms = ms;
                best = cand;
              }
            }
          }
          tune_store_locked(key, best);
        }
        (kind == TUNE_DOWN ? c->cfg_down : kind == TUNE_UP ? c->cfg_up : c->cfg_smooth)[l] = best;
      }
      // the legs with tensor copies against the per-thread copies: each
      // variant's best z-chunk, then the two winners timed in alternation
      // (three rounds), since they are often within a few per cent
      if (c->opts.tensor_copies == 0 && mg::down_tma_ok(g, hom)) {
        const TuneKey key{prop.multiProcessorCount, prop.major, prop.minor, TUNE_TMA, g.nx, g.ny,
                          g.nz, periodic};
        const TuneKey czkey{prop.multiProcessorCount, prop.major, prop.minor, TUNE_TMA_CZ, g.nx,
                            g.ny, g.nz, periodic};
        mg::TileCfg v{0, 0, 0}, w{0, 0, 0};
        auto hit = g_tune.find(key);
        auto czhit = g_tune.find(czkey);
        if (hit != g_tune.end() && czhit != g_tune.end()) {
          v = hit->second;
          w = czhit->second;
        } else {
          auto best_cz = [&](int ty, auto run) {
            float best = 1e30f;
            int bcz = 0;
            for (int cz = 8; cz <= 64; cz += 8) {
              if (cz > g.nz || !mg::fused_cfg_ok(g, mg::TileCfg{64, cz, ty})) continue;
              const float ms = time_launches(c, s, reps, flush, flush_bytes, [&]() { return run(cz); });
              if (ms < best) {
                best = ms;
                bcz = cz;
              }
            }
            return bcz;
          };
          auto second_faster = [&](auto run_a, auto run_b) {
            float a = 0.f, b = 0.f;
            for (int r = 0; r < 3; ++r) {
              a += time_launches(c, s, reps, flush, flush_bytes, run_a);
              b += time_launches(c, s, reps, flush, flush_bytes, run_b);
            }
            return b < a;
          };
          for (const bool zg : {true, false}) {
            const int cz = best_cz(32, [&](int z) {
              return mg::launch_fused_down_tma(c->u32[l], c->u32b[l], c->f32[l], c->f32[l - 1], g,
                                               h, om, zg, z, c->iflag + 1, s);
            });
            const bool win = second_faster(
                [&]() {
                  return mg::launch_fused_down(c->u32[l], c->u32b[l], c->f32[l], c->f32[l - 1], g,
                                               h, hom, om, zg, s, c->cfg_down[l]);
                },
                [&]() {
                  return mg::launch_fused_down_tma(c->u32[l], c->u32b[l], c->f32[l],
                                                   c->f32[l - 1], g, h, om, zg, cz, c->iflag + 1,
                                                   s);
                });
            (zg ? v.tx : v.cz) = win ? 1 : 0;
            (zg ? w.tx : w.cz) = cz;
          }
          if (mg::up_tma_ok(g, hom)) {
            const int cz = best_cz(16, [&](int z) {
              return mg::launch_fused_up_tma(c->u32[l], c->u32b[l], c->f32[l], c->u32[l - 1], g,
                                             h, om, z, c->iflag + 1, s);
            });
            const bool win = second_faster(
                [&]() {
                  return mg::launch_fused_up(c->u32[l], c->u32b[l], c->f32[l], c->u32[l - 1], g,
                                             h, hom, om, s, c->cfg_up[l]);
                },
                [&]() {
                  return mg::launch_fused_up_tma(c->u32[l], c->u32b[l], c->f32[l],
                                                 c->u32[l - 1], g, h, om, cz, c->iflag + 1, s);
                });
            v.ty = win ? 1 : 0;
            w.ty = cz;
          }
          tune_store_locked(key, v);
          tune_store_locked(czkey, w);
        }
        c->tma_down0[l] = v.tx == 1;
        c->tma_down[l] = v.cz == 1;
        c->tma_up[l] = v.ty == 1;
        c->tma_cz_down0[l] = w.tx;
        c->tma_cz_down[l] = w.cz;
        c->tma_cz_up[l] = w.ty;
      }
      // the fused up-down pass of the finest level's inner cycles
      if (l == F && c->opts.leg_pairs != 2 && pairs_ok(c, l, hom, hom, 2)) {
        const TuneKey key{prop.multiProcessorCount, prop.major, prop.minor, TUNE_UD, g.nx, g.ny,
                          g.nz, periodic};
        mg::TileCfg best;
        auto hit = g_tune.find(key);
        if (hit != g_tune.end()) {
          best = hit->second;
        } else {
          float best_ms = 1e30f;
          for (int ty : {16, 32})
            for (int cz : {16, 32, 64, 128}) {
              const mg::TileCfg cand{64, cz, ty};
              if (cz > g.nz || !mg::updown_cfg_ok(g, cand)) continue;
              const float ms = time_launches(c, s, reps, flush, flush_bytes, [&]() {
                return mg::launch_fused_updown(c->u32[l], c->u32b[l], c->f32[l], c->u32[l - 1],
                                               c->f32[l - 1], g, h, hom, om, s, cand);
              });
              if (ms < best_ms) {
                best_ms = ms;
                best = cand;
              }
            }
          tune_store_locked(key, best);
        }
        c->cfg_ud[l] = best;
        // fuse the legs only where the fused pass is the faster (its halo
        // recomputation can cost more than the bytes it saves)
        const TuneKey wkey{prop.multiProcessorCount, prop.major, prop.minor, TUNE_UD_WIN, g.nx,
                           g.ny, g.nz, periodic};
        auto whit = g_tune.find(wkey);
        if (whit != g_tune.end()) {
          c->pairs_faster = whit->second.cz == 1;
        } else {
          const float ud_ms = time_launches(c, s, reps, flush, flush_bytes, [&]() {
            return mg::launch_fused_updown(c->u32[l], c->u32b[l], c->f32[l], c->u32[l - 1],
                                           c->f32[l - 1], g, h, hom, om, s, best);
          });
          const float legs_ms =
              time_launches(c, s, reps, flush, flush_bytes, [&]() {
                return mg::launch_fused_down(c->u32[l], c->u32b[l], c->f32[l], c->f32[l - 1], g,
                                             h, hom, om, false, s, c->cfg_down[l]);
              }) +
              time_launches(c, s, reps, flush, flush_bytes, [&]() {
                return mg::launch_fused_up(c->u32[l], c->u32b[l], c->f32[l], c->u32[l - 1], g, h,
                                           hom, om, s, c->cfg_up[l]);
              });
          c->pairs_faster = ud_ms < legs_ms;
          tune_store_locked(wkey, mg::TileCfg{0, c->pairs_faster ? 1 : 0, 0});
        }
      }
    }
  }
  const Grid g = level_grid(c, F);
  if (c->fxbuf) {
    const TuneKey key{prop.multiProcessorCount, prop.major, prop.minor, TUNE_FX, g.nx, g.ny, g.nz,
                      periodic};
    auto hit = g_tune.find(key);
    if (hit != g_tune.end()) {
      c->fx_cz = hit->second.cz;
    } else {
      // phi_in and F both read the zeroed FP64 source buffer (as integers),
      // phi_out is the second integer buffer.
      long long* q = reinterpret_cast<long long*>(c->f64[F]);
      check(c, cudaMemsetAsync(q, 0, sizeof(long long) * g.cells(), s), "zero");
      check(c, cudaMemsetAsync(c->u32[F], 0, sizeof(float) * g.cells(), s), "zero");
      float best_ms = 1e30f;
      int best = 0;
      for (int cz : {4, 8, 16, 32, 64}) {
        if (cz > g.nz) continue;
        int nb = 0;
        const float ms = time_launches(c, s, reps, flush, flush_bytes, [&]() {
          return mg::launch_fx_step(q, c->fxbuf, c->u32[F], 1.f, q, c->f32[F], g, hom, 1.0, 1.f,
                                    c->partials, c->partials_cap, c->iflag, &nb, s, cz);
        });
        if (ms < best_ms) {
          best_ms = ms;
          best = cz;
        }
      }
      check(c, cudaMemsetAsync(c->iflag, 0, sizeof(int) * 4, s), "clear flag");
      tune_store_locked(key, mg::TileCfg{0, best});
      c->fx_cz = best;
    }
  }
  check(c, cudaStreamSynchronize(s), "sync");
}

}  // namespace

extern "C" {

void mg_opts_init(mg_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->prec = MG_FP64;
  o->mode_fmg = 1;
  o->pre = 1;
  o->post = 1;
  o->omega = 1.15;
  o->max_cycles = 50;
  o->fixed_value = 0.0;
  o->lmax = 4;
  o->use_com = 1;
  o->stall_ratio = 0.9;
  o->inner_fmg = 0;
  o->inner_cycles = 3;
  o->outer_fixed = 1;
  o->fas = 0;
}

const char* mg_status_str(mg_status s) {
  switch (s) {
    case MG_OK: return "MG_OK";
    case MG_ERR_ARG: return "MG_ERR_ARG";
    case MG_ERR_OOM: return "MG_ERR_OOM";
    case MG_ERR_CUDA: return "MG_ERR_CUDA";
    case MG_ERR_NOT_CONVERGED: return "MG_ERR_NOT_CONVERGED";
    case MG_ERR_DIVERGED: return "MG_ERR_DIVERGED";
    case MG_ERR_TIMEOUT: return "MG_ERR_TIMEOUT";
    case MG_ERR_BUSY: return "MG_ERR_BUSY";
  }
  return "MG_ERR_UNKNOWN";
}

const char* mg_last_error(const mg_ctx* c) { return c ? c->err.c_str() : g_err.c_str(); }

size_t mg_ctx_device_bytes(const mg_ctx* c) { return c ? c->bytes : 0; }

long long mg_ctx_last_launches(const mg_ctx* c) { return c ? c->last_launches : 0; }

mg_status mg_ctx_set_timing(mg_ctx* c, int on) {
  if (!c) return MG_ERR_ARG;
  c->timing = on ? 1 : 0;
  for (int k = 0; k < MG_K_COUNT; ++k) {
    c->kernel_ms[k] = 0.0;
    c->kernel_n[k] = 0;
  }
  return MG_OK;
}

mg_status mg_ctx_autotune(mg_ctx* c, void* stream) {
  if (!c) return MG_ERR_ARG;
  try {
    check(c, cudaSetDevice(c->device), "cudaSetDevice");
    drop_inner_graph(c);  // the launch shapes may change
    autotune(c, (cudaStream_t)stream);
  } catch (const Fail& f) {
    cudaStreamSynchronize((cudaStream_t)stream);
    return f.st;
  }
  return MG_OK;
}

mg_status mg_ctx_tile_config(const mg_ctx* c, int level, int kernel, int* tx, int* ty, int* cz) {
  if (!c || !tx || !ty || !cz || level < 0 || level >= c->L) return MG_ERR_ARG;
  mg::TileCfg v;
  const Bc hom = mg::homogeneous(Bc{c->bc_kind, c->opts.fixed_value, nullptr, c->face_mask});
  const bool fp32 = c->opts.prec == MG_MIXED && level > 0 && c->u32b[level];
  if (fp32 && kernel == MG_K_FUSED_DOWN && tma_level(c, level, hom, false))
    v = mg::TileCfg{64, c->tma_cz_down[level], 32};  // the leg with tensor copies
  else if (fp32 && kernel == MG_K_FUSED_DOWN0 && tma_level(c, level, hom, true))
    v = mg::TileCfg{64, c->tma_cz_down0[level], 32};
  else if (fp32 && kernel == MG_K_FUSED_UP && tma_up_level(c, level, hom))
    v = mg::TileCfg{64, c->tma_cz_up[level], 16};
  else if (kernel == MG_K_FUSED_DOWN || kernel == MG_K_FUSED_DOWN0) v = c->cfg_down[level];
  else if (kernel == MG_K_FUSED_UPDOWN) v = c->cfg_ud[level];
  else if (kernel == MG_K_FUSED_UP) v = c->cfg_up[level];
  else if (kernel == MG_K_SOR) v = c->cfg_smooth[level];
  else if (kernel == MG_K_OUTER_RESIDUAL) v = mg::TileCfg{0, level == c->L - 1 ? c->fx_cz : 0};
  else return MG_ERR_ARG;
  *tx = v.tx;
  *ty = v.ty;
  *cz = v.cz;
  return MG_OK;
}

mg_status mg_ctx_tensor_copies(const mg_ctx* c, int level, int* down, int* down0, int* up) {
  if (!c || !down || !down0 || !up || level < 0 || level >= c->L) return MG_ERR_ARG;
  const Bc hom = mg::homogeneous(Bc{c->bc_kind, c->opts.fixed_value, nullptr, c->face_mask});
  const bool fp32 = c->opts.prec == MG_MIXED && level > 0 && c->u32b[level];
  *down = fp32 && tma_level(c, level, hom, false) ? 1 : 0;
  *down0 = fp32 && tma_level(c, level, hom, true) ? 1 : 0;
  *up = fp32 && tma_up_level(c, level, hom) ? 1 : 0;
  return MG_OK;
}

mg_status mg_ctx_kernel_time(const mg_ctx* c, int k, double* total_ms, long long* launches) {
  if (!c || k < 0 || k >= MG_K_COUNT || !total_ms || !launches) return MG_ERR_ARG;
  *total_ms = c->kernel_ms[k];
  *launches = c->kernel_n[k];
  return MG_OK;
}

mg_status mg_destroy(mg_ctx* c) {
  if (!c) return MG_OK;
  drop_inner_graph(c);
  for (cudaEvent_t e : c->events) cudaEventDestroy(e);
  for (void* p : c->allocs) cudaFree(p);
  if (c->pinned) cudaFreeHost(c->pinned);
  delete c;
  return MG_OK;
}

namespace {

// mg_create and mg_create_faces; face_mask / face_b describe a MIXED rule.
mg_status create_ctx(int nx, int ny, int nz, double dx, mg_bc bc, int face_mask,
                     const double* face_b, const mg_opts* opts, mg_ctx** out) {
  if (!out) {
    g_err = "mg_create: ctx is NULL";
    return MG_ERR_ARG;
  }
  *out = nullptr;
  mg_opts o;
  if (opts) o = *opts;
  else mg_opts_init(&o);
  if (!dims_ok(nx, ny, nz) || !(dx > 0.0) || (int)bc < 0 || (int)bc > 4 ||
      validate_opts(o) != MG_OK) {
    g_err = "mg_create: invalid argument (powers of two >= 2 with nx the longest side, dx > 0, "
            "bc, opts)";
    return MG_ERR_ARG;
  }
  mg_ctx* c = new mg_ctx;
  try {
    c->n = nx;
    c->ny = ny;
    c->nz = nz;
    c->h = dx;
    c->bc_kind = (int)bc;
    if (bc == MG_BC_MIXED) {
      c->face_mask = face_mask;
      for (int q = 0; q < 6; ++q) c->face_b[q] = face_b[q];
    }
    c->opts = o;
    const int m = std::min(nx, std::min(ny, nz));
    int L = 1;
    while ((m >> (L - 1)) > 1) ++L;
    if (L > kMaxLevels) fail(c, MG_ERR_ARG, "mg_create: grid too large");
    c->L = L;
    check(c, cudaGetDevice(&c->device), "cudaGetDevice");
    if (bc == MG_BC_OPEN) check(c, mg::prepare_multipole(), "multipole tables");
    alloc_hierarchy(c);
    check(c, cudaMemset(c->iflag, 0, 4 * sizeof(int)), "clear flags");
    if (bc == MG_BC_MIXED) fill_mixed_faces(c);
    check(c, cudaMallocHost(&c->pinned, 64 * sizeof(double)), "cudaMallocHost");
  } catch (const Fail& f) {
    mg_destroy(c);
    return f.st;
  }
  *out = c;
  return MG_OK;
}

}  // namespace

mg_status mg_create(int nx, int ny, int nz, double dx, mg_bc bc, const mg_opts* opts,
                    mg_ctx** out) {
  if (bc == MG_BC_MIXED) {
    g_err = "mg_create: a rule per face is made by mg_create_faces";
    if (out) *out = nullptr;
    return MG_ERR_ARG;
  }
  return create_ctx(nx, ny, nz, dx, bc, 0, nullptr, opts, out);
}

mg_status mg_create_faces(int nx, int ny, int nz, double dx, const mg_bc* face_bc,
                          const double* face_value, const mg_opts* opts, mg_ctx** out) {
  if (out) *out = nullptr;
  if (!face_bc || !out) {
    g_err = "mg_create_faces: face_bc and ctx must not be NULL";
    return MG_ERR_ARG;
  }
  double b[6] = {};
  int mask = 0;
  for (int q = 0; q < 6; ++q) {
    const mg_bc k = face_bc[q];
    if (k != MG_BC_PERIODIC && k != MG_BC_FIXED && k != MG_BC_ZEROGRAD) {
      g_err = "mg_create_faces: a face is periodic, fixed or zero gradient";
      return MG_ERR_ARG;
    }
    b[q] = (k == MG_BC_FIXED && face_value) ? face_value[q] : 0.0;
    if (!std::isfinite(b[q])) {
      g_err = "mg_create_faces: face values must be finite";
      return MG_ERR_ARG;
    }
    mask |= (int)k << (2 * q);
  }
  for (int a = 0; a < 3; ++a)
    if ((face_bc[2 * a] == MG_BC_PERIODIC) != (face_bc[2 * a + 1] == MG_BC_PERIODIC)) {
      g_err = "mg_create_faces: periodic faces come in pairs";
      return MG_ERR_ARG;
    }
  bool same = true;
  for (int q = 1; q < 6; ++q) same = same && face_bc[q] == face_bc[0] && b[q] == b[0];
  if (same) {  // one rule on every face: that rule's own context
    mg_opts o;
    if (opts) o = *opts;
    else mg_opts_init(&o);
    if (face_bc[0] == MG_BC_FIXED) o.fixed_value = b[0];
    return create_ctx(nx, ny, nz, dx, face_bc[0], 0, nullptr, &o, out);
  }
  return create_ctx(nx, ny, nz, dx, MG_BC_MIXED, mask, b, opts, out);
}

mg_status mg_required_bytes(int nx, int ny, int nz, mg_bc bc, const mg_opts* opts,
                            size_t* bytes) {
  if (!bytes) return MG_ERR_ARG;
  *bytes = 0;
  mg_opts o;
  if (opts) o = *opts;
  else mg_opts_init(&o);
  if (!dims_ok(nx, ny, nz) || (int)bc < 0 || (int)bc > 3 || validate_opts(o) != MG_OK) {
    g_err = "mg_required_bytes: invalid argument";
    return MG_ERR_ARG;
  }
  mg_ctx c;
  c.dry = true;
  c.n = nx;
  c.ny = ny;
  c.nz = nz;
  c.h = 1.0;
  c.bc_kind = (int)bc;
  c.opts = o;
  c.L = 1;
  const int m = std::min(nx, std::min(ny, nz));
  while ((m >> (c.L - 1)) > 1) ++c.L;
  if (c.L > kMaxLevels) return MG_ERR_ARG;
  alloc_hierarchy(&c);
  *bytes = c.bytes;
  return MG_OK;
}

mg_status mg_solve(mg_ctx* c, const double* rho, double four_pi_G, double tol, double* phi,
                   double* hist, int hist_cap, int* n_hist, void* stream) {
  return mg_solve_gravity(c, rho, four_pi_G, tol, phi, nullptr, hist, hist_cap, n_hist, stream);
}

mg_status mg_solve_gravity(mg_ctx* c, const double* rho, double four_pi_G, double tol, double* phi,
                           double* g, double* hist, int hist_cap, int* n_hist, void* stream) {
  if (!c) {
    g_err = "mg_solve: ctx is NULL";
    return MG_ERR_ARG;
  }
  if (!rho || !phi || !hist || hist_cap < 1 || !n_hist || !(tol >= 0.0) ||
      !std::isfinite(four_pi_G)) {
    c->err = "mg_solve: invalid argument";
    return MG_ERR_ARG;
  }
  *n_hist = 0;
  cudaStream_t s = (cudaStream_t)stream;
  mg::g_launches = 0;
  mg_status st;
  try {
    check(c, cudaSetDevice(c->device), "cudaSetDevice");
    if (c->opts.prec == MG_FP64)
      st = solve_fp64(c, rho, four_pi_G, tol, phi, g, hist, hist_cap, n_hist, s);
    else
      st = solve_mixed(c, rho, four_pi_G, tol, phi, g, hist, hist_cap, n_hist, s);
    check(c, cudaStreamSynchronize(s), "sync");
    collect_times(c);
  } catch (const Fail& f) {
    st = f.st;
    cudaStreamSynchronize(s);
    c->pending_class.clear();
  }
  c->last_launches = mg::g_launches;
  return st;
}

// Page-locked host memory that this device can address directly (unified
// addressing maps it at the same address).
static bool host_mapped(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky error of an unknown pointer
    return false;
  }
  return a.type == cudaMemoryTypeHost && a.devicePointer == p;
}

mg_status mg_solve_host(mg_ctx* c, const double* rho, double four_pi_G, double tol, double* phi,
                        double* hist, int hist_cap, int* n_hist, void* stream) {
  if (!c || !rho || !phi) {
    g_err = "mg_solve_host: invalid argument";
    return MG_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)level_grid(c, c->L - 1).cells() * sizeof(double);
  try {
    check(c, cudaSetDevice(c->device), "cudaSetDevice");
    if (!c->rho_dev_own) c->rho_dev_own = dalloc<double>(c, bytes / sizeof(double));
    if (!c->phi_dev_own) c->phi_dev_own = dalloc<double>(c, bytes / sizeof(double));
    // Pinned (page-locked, device-mapped) host buffers are read and written by
    // the solve's first and last passes themselves; others go through copies.
    const bool rho_pinned = host_mapped(rho), phi_pinned = host_mapped(phi);
    if (!rho_pinned)
      check(c, cudaMemcpyAsync(c->rho_dev_own, rho, bytes, cudaMemcpyHostToDevice, s), "H2D rho");
    if (!c->opts.mode_fmg)
      check(c, cudaMemcpyAsync(c->phi_dev_own, phi, bytes, cudaMemcpyHostToDevice, s), "H2D phi");
    c->host_rho = rho_pinned ? rho : nullptr;
    c->host_phi = phi_pinned ? phi : nullptr;
    c->host_phi_written = false;
  } catch (const Fail& f) {
    return f.st;
  }
  mg_status st =
      mg_solve(c, c->rho_dev_own, four_pi_G, tol, c->phi_dev_own, hist, hist_cap, n_hist, stream);
  const bool written = c->host_phi_written;
  c->host_rho = nullptr;
  c->host_phi = nullptr;
  c->host_phi_written = false;
  if (st != MG_OK && st != MG_ERR_NOT_CONVERGED) return st;
  try {
    if (!written)
      check(c, cudaMemcpyAsync(phi, c->phi_dev_own, bytes, cudaMemcpyDeviceToHost, s), "D2H phi");
    check(c, cudaStreamSynchronize(s), "sync");
  } catch (const Fail& f) {
    return f.st;
  }
  return st;
}

// ---------------------------------------------------------------------------
// Single-step operators.

size_t mg_faces_count(int nx, int ny, int nz) { return mg::faces_count(Grid{nx, ny, nz}); }

}  // extern "C"

namespace mg {

mg_status solve_host_copies(mg_ctx* c, const double* rho, double four_pi_G, double tol,
                            double* phi, double* hist, int hist_cap, int* n_hist,
                            cudaStream_t s, double* copy_ms) {
  if (!c || !rho || !phi) return MG_ERR_ARG;
  const size_t bytes = (size_t)level_grid(c, c->L - 1).cells() * sizeof(double);
  // events around the two copies (timed only when asked)
  cudaEvent_t ev[4] = {};
  struct Events {
    cudaEvent_t* e;
    ~Events() {
      for (int k = 0; k < 4; ++k)
        if (e[k]) cudaEventDestroy(e[k]);
    }
  } events{ev};
  try {
    check(c, cudaSetDevice(c->device), "cudaSetDevice");
    if (copy_ms)
      for (cudaEvent_t& e : ev) check(c, cudaEventCreate(&e), "cudaEventCreate");
    if (!c->rho_dev_own) c->rho_dev_own = dalloc<double>(c, bytes / sizeof(double));
    if (!c->phi_dev_own) c->phi_dev_own = dalloc<double>(c, bytes / sizeof(double));
    if (copy_ms) check(c, cudaEventRecord(ev[0], s), "record");
    check(c, cudaMemcpyAsync(c->rho_dev_own, rho, bytes, cudaMemcpyHostToDevice, s), "H2D rho");
    if (copy_ms) check(c, cudaEventRecord(ev[1], s), "record");
    if (!c->opts.mode_fmg)
      check(c, cudaMemcpyAsync(c->phi_dev_own, phi, bytes, cudaMemcpyHostToDevice, s), "H2D phi");
  } catch (const Fail& f) {
    cudaStreamSynchronize(s);
    return f.st;
  }
  const mg_status st =
      mg_solve(c, c->rho_dev_own, four_pi_G, tol, c->phi_dev_own, hist, hist_cap, n_hist, s);
  if (st != MG_OK && st != MG_ERR_NOT_CONVERGED) {
    cudaStreamSynchronize(s);  // nothing of this request stays in flight on the context
    return st;
  }
  try {
    if (copy_ms) check(c, cudaEventRecord(ev[2], s), "record");
    check(c, cudaMemcpyAsync(phi, c->phi_dev_own, bytes, cudaMemcpyDeviceToHost, s), "D2H phi");
    if (copy_ms) check(c, cudaEventRecord(ev[3], s), "record");
    check(c, cudaStreamSynchronize(s), "sync");
    if (copy_ms) {
      float a = 0.f, b = 0.f;
      check(c, cudaEventElapsedTime(&a, ev[0], ev[1]), "elapsed");
      check(c, cudaEventElapsedTime(&b, ev[2], ev[3]), "elapsed");
      copy_ms[0] = a;
      copy_ms[1] = b;
    }
  } catch (const Fail& f) {
    cudaStreamSynchronize(s);
    return f.st;
  }
  return st;
}

}  // namespace mg

namespace {

bool op_args_ok(int prec, int nx, int ny, int nz, int bc, const double* faces) {
  if (prec != MG_FP64 && prec != MG_MIXED) return false;
  if (nx < 1 || ny < 1 || nz < 1 || bc < 0 || bc > 3) return false;
  if (bc == MG_BC_OPEN && !faces) return false;
  return true;
}

mg_status op_result(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return MG_OK;
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return MG_ERR_CUDA;
}

template <typename T>
cudaError_t do_smooth(int nx, int ny, int nz, double h, Bc bc, double omega, int steps,
                      int colours, void* u, const void* f, cudaStream_t s) {
  const Grid g{nx, ny, nz};
  for (int q = 0; q < steps; ++q) {
    if (colours == 0 || colours == 1) {
      cudaError_t e = mg::launch_sor<T>((T*)u, (const T*)f, g, h, bc, omega, 0, s);
      if (e != cudaSuccess) return e;
    }
    if (colours == 0 || colours == 2) {
      cudaError_t e = mg::launch_sor<T>((T*)u, (const T*)f, g, h, bc, omega, 1, s);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace

extern "C" {

mg_status mg_op_smooth(int prec, int nx, int ny, int nz, double h, mg_bc bc, double bc_value,
                       const double* faces, double omega, int steps, int colours, void* u,
                       const void* f, void* stream) {
  if (!op_args_ok(prec, nx, ny, nz, bc, faces) || !u || !f || nx % 2 || steps < 0 ||
      colours < 0 || colours > 2) {
    g_err = "mg_op_smooth: invalid argument";
    return MG_ERR_ARG;
  }
  const Bc b{(int)bc, bc_value, faces};
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = prec == MG_FP64 ? do_smooth<double>(nx, ny, nz, h, b, omega, steps, colours, u, f, s)
                                  : do_smooth<float>(nx, ny, nz, h, b, omega, steps, colours, u, f, s);
  return op_result(e, "smooth");
}

mg_status mg_op_defect(int prec, int nx, int ny, int nz, double h, mg_bc bc, double bc_value,
                       const double* faces, const void* u, const void* f, void* d, void* stream) {
  if (!op_args_ok(prec, nx, ny, nz, bc, faces) || !u || !f || !d) {
    g_err = "mg_op_defect: invalid argument";
    return MG_ERR_ARG;
  }
  const Bc b{(int)bc, bc_value, faces};
  const Grid g{nx, ny, nz};
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e =
      prec == MG_FP64
          ? mg::launch_defect<double>((const double*)u, (const double*)f, (double*)d, g, h, b, nullptr, s)
          : mg::launch_defect<float>((const float*)u, (const float*)f, (float*)d, g, h, b, nullptr, s);
  return op_result(e, "defect");
}

mg_status mg_op_gravity(int nx, int ny, int nz, double h, mg_bc bc, double bc_value,
                        const double* faces, const double* phi, double* g, void* stream) {
  if (!op_args_ok(MG_FP64, nx, ny, nz, bc, faces) || !phi || !g || !(h > 0.0)) {
    g_err = "mg_op_gravity: invalid argument";
    return MG_ERR_ARG;
  }
  const Bc b{(int)bc, bc_value, faces};
  const Grid gr{nx, ny, nz};
  return op_result(mg::launch_gravity(phi, g, gr, h, b, (cudaStream_t)stream), "gravity");
}

mg_status mg_op_defect_restrict(int prec, int nx, int ny, int nz, double h, mg_bc bc,
                                double bc_value, const double* faces, const void* u, const void* f,
                                void* fc, void* stream) {
  if (!op_args_ok(prec, nx, ny, nz, bc, faces) || !u || !f || !fc || nx % 2 || ny % 2 || nz % 2) {
    g_err = "mg_op_defect_restrict: invalid argument";
    return MG_ERR_ARG;
  }
  const Bc b{(int)bc, bc_value, faces};
  const Grid g{nx, ny, nz};
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = prec == MG_FP64
                      ? mg::launch_defect_restrict<double>((const double*)u, (const double*)f,
                                                           (double*)fc, g, h, b, s)
                      : mg::launch_defect_restrict<float>((const float*)u, (const float*)f,
                                                          (float*)fc, g, h, b, s);
  return op_result(e, "defect_restrict");
}

mg_status mg_op_restrict(int prec, int nx, int ny, int nz, const void* uf, void* uc, void* stream) {
  if ((prec != MG_FP64 && prec != MG_MIXED) || nx < 2 || ny < 2 || nz < 2 || nx % 2 || ny % 2 ||
      nz % 2 || !uf || !uc) {
    g_err = "mg_op_restrict: invalid argument";
    return MG_ERR_ARG;
  }
  const Grid g{nx, ny, nz};
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = prec == MG_FP64 ? mg::launch_restrict<double>((const double*)uf, (double*)uc, g, s)
                                  : mg::launch_restrict<float>((const float*)uf, (float*)uc, g, s);
  return op_result(e, "restrict");
}

mg_status mg_op_prolong(int prec, int nx, int ny, int nz, mg_bc bc, double bc_value,
                        const double* coarse_faces, int high_order, int add, const void* uc,
                        void* uf, void* stream) {
  if (!op_args_ok(prec, nx, ny, nz, bc, coarse_faces) || nx % 2 || ny % 2 || nz % 2 || !uc || !uf) {
    g_err = "mg_op_prolong: invalid argument";
    return MG_ERR_ARG;
  }
  const Bc b{(int)bc, bc_value, coarse_faces};
  const Grid g{nx, ny, nz};
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = prec == MG_FP64
                      ? mg::launch_prolong<double>((const double*)uc, (double*)uf, g, b, high_order,
                                                   add, s)
                      : mg::launch_prolong<float>((const float*)uc, (float*)uf, g, b, high_order,
                                                  add, s);
  return op_result(e, "prolong");
}

mg_status mg_op_coarsest(int prec, double h, mg_bc bc, double bc_value, const double* faces,
                         const void* f, void* u, void* stream) {
  if (!op_args_ok(prec, 1, 1, 1, bc, faces) || !f || !u) {
    g_err = "mg_op_coarsest: invalid argument";
    return MG_ERR_ARG;
  }
  const Bc b{(int)bc, bc_value, faces};
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = prec == MG_FP64 ? mg::launch_coarsest<double>((const double*)f, (double*)u, h, b, s)
                                  : mg::launch_coarsest<float>((const float*)f, (float*)u, h, b, s);
  return op_result(e, "coarsest");
}

mg_status mg_op_vcycle_down(int nx, int ny, int nz, double h, mg_bc bc, double omega,
                            int zero_guess, const float* u_in, float* u_out, const float* f,
                            float* fc, void* stream) {
  if (!op_args_ok(MG_MIXED, nx, ny, nz, bc, nullptr) || bc == MG_BC_OPEN || nx < 2 || ny < 2 ||
      nz < 2 || nx % 2 || ny % 2 || nz % 2 || (!u_in && !zero_guess) || !u_out || !f || !fc ||
      u_in == u_out) {
    g_err = "mg_op_vcycle_down: invalid argument";
    return MG_ERR_ARG;
  }
  const Bc b{(int)bc, 0.0, nullptr};
  const Grid g{nx, ny, nz};
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (mg::fused_ok(g, b)) {
    e = mg::launch_fused_down(u_in, u_out, f, fc, g, h, b, omega, zero_guess != 0, s);
  } else {
    e = zero_guess ? mg::launch_sor_red_zero<float>(u_out, f, g, h, omega, s)
                   : cudaMemcpyAsync(u_out, u_in, sizeof(float) * g.cells(),
                                     cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && !zero_guess) e = mg::launch_sor<float>(u_out, f, g, h, b, omega, 0, s);
    if (e == cudaSuccess) e = mg::launch_sor<float>(u_out, f, g, h, b, omega, 1, s);
    if (e == cudaSuccess) e = mg::launch_defect_restrict<float>(u_out, f, fc, g, h, b, s);
  }
  return op_result(e, "vcycle_down");
}

mg_status mg_op_vcycle_up(int nx, int ny, int nz, double h, mg_bc bc, double omega,
                          const float* u_in, float* u_out, const float* f, const float* ec,
                          void* stream) {
  if (!op_args_ok(MG_MIXED, nx, ny, nz, bc, nullptr) || bc == MG_BC_OPEN || nx < 2 || ny < 2 ||
      nz < 2 || nx % 2 || ny % 2 || nz % 2 || !u_in || !u_out || !f || !ec || u_in == u_out) {
    g_err = "mg_op_vcycle_up: invalid argument";
    return MG_ERR_ARG;
  }
  const Bc b{(int)bc, 0.0, nullptr};
  const Grid g{nx, ny, nz};
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (mg::fused_ok(g, b)) {
    e = mg::launch_fused_up(u_in, u_out, f, ec, g, h, b, omega, s);
  } else {
    e = cudaMemcpyAsync(u_out, u_in, sizeof(float) * g.cells(), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = mg::launch_prolong<float>(ec, u_out, g, b, 0, 1, s);
    if (e == cudaSuccess) e = mg::launch_sor<float>(u_out, f, g, h, b, omega, 0, s);
    if (e == cudaSuccess) e = mg::launch_sor<float>(u_out, f, g, h, b, omega, 1, s);
  }
  return op_result(e, "vcycle_up");
}

mg_status mg_op_convert(int kind, long long n, const void* in, void* out, void* stream) {
  if (kind < 0 || kind > 4 || n < 0 || (n > 0 && (!in || !out))) {
    g_err = "mg_op_convert: invalid argument";
    return MG_ERR_ARG;
  }
  return op_result(mg::launch_convert(kind, n, in, out, (cudaStream_t)stream), "convert");
}

// A rule per face read from six kinds (periodic in pairs, fixed, zero
// gradient); false when the kinds are not such a rule.
static bool face_rule(const int* kinds, Bc* out) {
  if (!kinds) return false;
  int fk = 0;
  for (int q = 0; q < 6; ++q) {
    if (kinds[q] != MG_BC_PERIODIC && kinds[q] != MG_BC_FIXED && kinds[q] != MG_BC_ZEROGRAD)
      return false;
    fk |= kinds[q] << (2 * q);
  }
  for (int a = 0; a < 3; ++a)
    if ((kinds[2 * a] == MG_BC_PERIODIC) != (kinds[2 * a + 1] == MG_BC_PERIODIC)) return false;
  *out = Bc{mg::BC_MIXED, 0.0, nullptr, fk};
  return true;
}

mg_status mg_op_fused_leg(int leg, int nx, int ny, int nz, double h, const int* face_bc,
                          double omega, int zero_guess, int tx, int ty, int cz,
                          const float* u_in, float* u_out, const float* f, const float* ec,
                          float* fc, void* stream) {
  Bc b{};
  const Grid g{nx, ny, nz};
  const mg::TileCfg cfg{tx, cz, ty};
  const bool down = leg == 0 || leg == 3;
  bool ok = leg >= 0 && leg <= 4 && face_rule(face_bc, &b) && h > 0.0 && omega > 0.0 &&
            omega < 2.0 && u_out && f && (u_in || (down && zero_guess)) && u_in != u_out &&
            (leg == 1 || leg == 4 || fc != nullptr) && (down || ec != nullptr) && (down || !zero_guess);
  if (ok) {
    b = mg::collapse_homogeneous(b);
    ok = mg::fused_ok(g, b) && mg::fused_cfg_ok(g, cfg) && (tx == 0 || tx == 32 || tx == 64) &&
         (ty == 0 || ty == 16 || ty == 32) && cz >= 0;
    if (leg == 2) ok = mg::updown_ok(g, b) && mg::updown_cfg_ok(g, cfg);
    if (leg == 3) ok = ok && mg::down_tma_ok(g, b) && (tx == 0 || tx == 64) && (ty == 0 || ty == 32);
    if (leg == 4) ok = ok && mg::up_tma_ok(g, b) && (tx == 0 || tx == 64) && (ty == 0 || ty == 16);
  }
  if (!ok) {
    g_err = "mg_op_fused_leg: invalid argument, or a grid or shape the fused kernels do not take";
    return MG_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (leg == 0)
    e = mg::launch_fused_down(u_in, u_out, f, fc, g, h, b, omega, zero_guess != 0, s, cfg);
  else if (leg == 1)
    e = mg::launch_fused_up(u_in, u_out, f, ec, g, h, b, omega, s, cfg);
  else if (leg == 2)
    e = mg::launch_fused_updown(u_in, u_out, f, ec, fc, g, h, b, omega, s, cfg);
  else {  // 3, 4: the down and up legs with tensor copies
    volatile int* late = mg::down_tma_op_flag();
    if (!late) return op_result(cudaErrorMemoryAllocation, "fused_leg");
    if (*late) {  // raised by an earlier call's kernel, finished by now
      *late = 0;
      g_err = "mg_op_fused_leg: a tensor copy of an earlier leg-3 call did not land in time";
      return MG_ERR_TIMEOUT;
    }
    if (leg == 3)
      e = mg::launch_fused_down_tma(u_in, u_out, f, fc, g, h, omega, zero_guess != 0, cz,
                                    const_cast<int*>(late), s);
    else
      e = mg::launch_fused_up_tma(u_in, u_out, f, ec, g, h, omega, cz, const_cast<int*>(late), s);
  }
  return op_result(e, "fused_leg");
}

mg_status mg_op_fx_step(int nx, int ny, int nz, const int* face_bc, const double* faces_dev,
                        double two_pow_S, int cz, const long long* phi_in, const float* e,
                        float c, const long long* F, long long* phi_out, float factor, float* r32,
                        void* stream) {
  Bc b{};
  const Grid g{nx, ny, nz};
  bool ok = face_rule(face_bc, &b) && mg::fx_step_ok(g) && nx >= 2 && ny >= 2 && nz >= 2 &&
            e && phi_out && F && r32 && phi_in != phi_out && (cz == 0 || cz >= mg::kFxMinCz) &&
            std::isfinite(two_pow_S) && two_pow_S > 0.0;
  if (!ok) {
    g_err = "mg_op_fx_step: invalid argument, or a grid the fixed-point step does not take";
    return MG_ERR_ARG;
  }
  b.faces = faces_dev;
  if (!faces_dev) b = mg::collapse_homogeneous(b);
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = mg::fx_step_blocks(g, cz);
  double* partials = nullptr;
  int* flag = nullptr;
  cudaError_t err = cudaMalloc(&partials, sizeof(double) * (size_t)nb);
  if (err == cudaSuccess) err = cudaMalloc(&flag, sizeof(int));
  if (err == cudaSuccess) err = cudaMemsetAsync(flag, 0, sizeof(int), s);
  int nb_out = 0;
  if (err == cudaSuccess)
    err = mg::launch_fx_step(phi_in, phi_out, e, c, F, r32, g, b, two_pow_S, factor, partials, nb,
                             flag, &nb_out, s, cz);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  cudaFree(partials);
  cudaFree(flag);
  return op_result(err, "fx_step");
}

mg_status mg_op_multipole_moments(int nx, int ny, int nz, double h, const double* rho, int lmax,
                                  int use_com, double* origin, double* Q, void* stream) {
  if (nx < 1 || ny < 1 || nz < 1 || !rho || !origin || !Q || lmax < 0 || lmax > 4) {
    g_err = "mg_op_multipole_moments: invalid argument";
    return MG_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  double* buf = nullptr;
  double* host = nullptr;
  cudaError_t e = mg::prepare_multipole();
  if (e == cudaSuccess) e = cudaMallocAsync(&buf, (mg::kPartials + 64) * sizeof(double), s);
  if (e != cudaSuccess) return op_result(e, "multipole_moments");
  int nb = 0;
  e = mg::launch_raw_moments(rho, Grid{nx, ny, nz}, h, buf, &nb, s);
  if (e == cudaSuccess)
    e = mg::launch_moments_finish(buf, nb, h, lmax, use_com, origin, buf + mg::kPartials, s);
  if (e == cudaSuccess) e = cudaMallocHost(&host, 32 * sizeof(double));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host, buf + mg::kPartials, 29 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) {
    std::memcpy(Q, host, 25 * sizeof(double));
    std::memcpy(origin, host + 25, 3 * sizeof(double));
  }
  cudaFreeAsync(buf, s);
  cudaStreamSynchronize(s);
  if (host) cudaFreeHost(host);
  return op_result(e, "multipole_moments");
}

mg_status mg_op_open_faces(int nx, int ny, int nz, double h, const double* Q, int lmax, double G,
                           const double* origin, double* faces, void* stream) {
  if (nx < 1 || ny < 1 || nz < 1 || !Q || !origin || !faces || lmax < 0 || lmax > 4) {
    g_err = "mg_op_open_faces: invalid argument";
    return MG_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  double* qo = nullptr;
  cudaError_t e = mg::prepare_multipole();
  if (e == cudaSuccess) e = cudaMallocAsync(&qo, 32 * sizeof(double), s);
  if (e != cudaSuccess) return op_result(e, "open_faces");
  double tmp[28];
  std::memcpy(tmp, Q, 25 * sizeof(double));
  std::memcpy(tmp + 25, origin, 3 * sizeof(double));
  e = cudaMemcpyAsync(qo, tmp, 28 * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = mg::launch_open_faces(Grid{nx, ny, nz}, h, qo, lmax, G, faces, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // tmp is on the stack
  cudaFreeAsync(qo, s);
  return op_result(e, "open_faces");
}

}  // extern "C"
