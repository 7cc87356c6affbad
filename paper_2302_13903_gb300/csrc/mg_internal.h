// mg_internal.h -- types and kernel launchers shared by the translation units
// of the multigrid library.  Host-only header: kernels themselves live in the
// .cu files; this declares what the solver driver may launch.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/mg.h"

namespace mg {

enum BcKind : int { BC_PERIODIC = 0, BC_FIXED = 1, BC_ZEROGRAD = 2, BC_OPEN = 3, BC_MIXED = 4 };

// Cells per side of one level.
struct Grid {
  int nx, ny, nz;
  __host__ __device__ long long cells() const { return (long long)nx * ny * nz; }
};

// Boundary rule of one level as a kernel sees it (Sec. 2.3.6).  OPEN uses the
// level's face array (layout of mg.h); FIXED uses `value`; the homogeneous
// counterpart of FIXED/OPEN is FIXED with value 0.  MIXED has a rule per face:
// bits 2q..2q+1 of `fk` hold the kind of face q (x-, x+, y-, y+, z-, z+:
// periodic, fixed or zero gradient) and the fixed faces' values are read from
// the face array, or are 0 where it is null (the homogeneous rule).
struct Bc {
  int kind;
  double value;
  const double* faces;
  int fk;
};

__host__ __device__ inline int face_kind(const Bc& b, int face) {
  return b.kind == BC_MIXED ? (b.fk >> (2 * face)) & 3 : b.kind;
}

// A MIXED rule whose six faces have one kind is that kind's rule (its fixed
// faces then hold 0: only homogeneous rules are collapsed).
inline Bc collapse_homogeneous(Bc h) {
  if (h.kind != BC_MIXED) return h;
  for (int q = 1; q < 6; ++q)
    if (face_kind(h, q) != face_kind(h, 0)) return h;
  return Bc{face_kind(h, 0), 0.0, nullptr, 0};
}

inline Bc homogeneous(const Bc& b) {
  Bc h{b.kind, 0.0, nullptr, b.fk};
  if (b.kind == BC_FIXED || b.kind == BC_OPEN) h.kind = BC_FIXED;
  return collapse_homogeneous(h);
}

inline size_t faces_count(const Grid& g) {
  return 2 * (size_t)(g.ny + 2) * (g.nz + 2) + 2 * (size_t)(g.nx + 2) * (g.nz + 2) +
         2 * (size_t)(g.nx + 2) * (g.ny + 2);
}

// mg_solve with rho and phi in host memory moved by copies on `s` (the copy
// engines) into the context's own device arrays and back, so that the SMs stay
// free for solves on other streams while the bytes cross the host link (the
// serving loop); mg_solve_host instead lets the solve's first and last passes
// read and write page-locked host memory themselves.
// copy_ms (may be null) receives the device time of the host-to-device copy
// of rho and of the device-to-host copy of phi, from events on `s`.
mg_status solve_host_copies(mg_ctx* c, const double* rho, double four_pi_G, double tol,
                            double* phi, double* hist, int hist_cap, int* n_hist,
                            cudaStream_t s, double* copy_ms = nullptr);

// Record the message mg_last_error(NULL) returns on this thread (entry points
// that have no context report their failures through it).
void set_last_error(const std::string& msg);

// Streaming multiprocessors of the current device (queried once per device).
int sm_count();

// Launch counter (per thread: a context is not thread-safe, so the driver
// resets and reads it around one solve on one thread).
extern thread_local long long g_launches;

// Number of blocks used by the deterministic two-stage reductions for an
// array of `n` elements; partial buffers need this many doubles.
int reduce_blocks(long long n);
constexpr int kMaxReduceBlocks = 1024;
// Doubles in a context's partial-sum buffer (reductions and moment partials).
constexpr int kPartials = 16384;

// ---------------------------------------------------------------------------
// Level kernels, T = float or double.  All return cudaGetLastError().

template <typename T>
cudaError_t launch_sor(T* u, const T* f, Grid g, double h, Bc bc, double omega, int colour,
                       cudaStream_t s);
// Red half-sweep from a zero initial value: writes red = (-omega h^2/6) f and
// black = 0 (Algorithm 1, coarse levels start from 0).
template <typename T>
cudaError_t launch_sor_red_zero(T* u, const T* f, Grid g, double h, double omega,
                                cudaStream_t s);
template <typename T>
cudaError_t launch_defect(const T* u, const T* f, T* d, Grid g, double h, Bc bc,
                          double* partials, cudaStream_t s);
template <typename T>
cudaError_t launch_defect_restrict(const T* u, const T* f, T* fc, Grid g, double h, Bc bc,
                                   cudaStream_t s);
template <typename T>
cudaError_t launch_restrict(const T* uf, T* uc, Grid gf, cudaStream_t s);
template <typename T>
cudaError_t launch_prolong(const T* uc, T* uf, Grid gf, Bc bc_coarse, int high_order, int add,
                           cudaStream_t s);
template <typename T>
// keep: a singular 1-cell level keeps u's start value (FAS) instead of 0.
cudaError_t launch_coarsest(const T* f, T* u, double h, Bc bc, cudaStream_t s, bool keep = false);
template <typename T>
cudaError_t launch_fill(T* u, long long n, T v, cudaStream_t s);

// FP64 source: f = four_pi_G * rho, partial sums of f into partials.
cudaError_t launch_source(const double* rho, double* f, long long n, double four_pi_G,
                          double* partials, cudaStream_t s);
// a[i] -= sum(partials[0..nb)) / n  (removes the mean; the sum is formed on
// the device in a fixed order into *total_slot, a device scalar).
cudaError_t launch_subtract_mean(double* a, long long n, const double* partials, int nb,
                                 double* total_slot, cudaStream_t s);
// Partial sums of a[i] (FP64) and of a[i]^2.
template <typename T>
cudaError_t launch_sum(const T* a, long long n, int squares, double* partials, cudaStream_t s);
// out[0] = sum(partials[0..nb)) in a fixed order.
cudaError_t launch_finish_sum(const double* partials, int nb, double* out, cudaStream_t s);
// FAS (Algorithm 3): f += L ur and u = ur (step 5); u -= ur (step 7).
cudaError_t launch_fas_rhs(const double* ur, double* f, double* u, Grid g, double h, Bc bc,
                           cudaStream_t s);
cudaError_t launch_sub(double* u, const double* ur, long long n, cudaStream_t s);
// g = -grad phi at cell centres (Sec. 3.2.3), g = [gx | gy | gz] (3 N doubles).
cudaError_t launch_gravity(const double* u, double* g, Grid gr, double h, Bc bc, cudaStream_t s);

// u += v (n cells).
cudaError_t launch_add_const(double* u, long long n, double v, cudaStream_t s);

// Mixed precision outer step (FP64 in, FP32 out): r32 = scale * (f - L_h u),
// partial sums of (f - L_h u)^2 in FP64.
cudaError_t launch_outer_residual(const double* u, const double* f, float* r32, Grid g, double h,
                                  Bc bc, double scale, double* partials, cudaStream_t s);
// b = (float)(scale * a).
cudaError_t launch_scale_to_f32(const double* a, float* b, long long n, double scale,
                               cudaStream_t s);
// u += inv_scale * e32 (FP64 correction update).
cudaError_t launch_correct(double* u, const float* e32, long long n, double inv_scale,
                           cudaStream_t s);

// ---------------------------------------------------------------------------
// Single-CTA bottom solver for the levels of at most 16^3 cells (levels
// 0 .. kBottomLevels-1): u, f, n, h, bc indexed by level (bc may be null when
// fmg is false).  fmg = false: one V-cycle on levels top .. 0 of the
// correction (u[top] starts at 0, f[top] holds the restricted defect);
// fmg = true: Algorithm 2 up to level `top` from f[top].
constexpr int kBottomLevels = 6;  // arrays of the bottom programs (levels up to 32^3)
constexpr int kBottomTopN = 16;   // the single-grid driver hands levels <= 16^3 to one CTA
template <typename T>
cudaError_t launch_bottom(T* const* u, T* const* f, const int* n, const double* h, const Bc* bc,
                          Bc hom, double omega, int pre, int post, int top, bool fmg,
                          cudaStream_t s);

// ---------------------------------------------------------------------------
// Fused FP32 V-cycle legs (homogeneous rules only).  Each reads u_in and
// writes u_out (distinct buffers).

// Launch shape of a z-marching kernel: tile width in cells (fused kernels:
// 32 or 64), z-planes per CTA and tile height (fused kernels: 16 or 32).  A
// zero field takes the built-in choice.
struct TileCfg {
  int tx = 0;
  int cz = 0;
  int ty = 0;  // tile height in rows (16 or 32; 0: 16)
};

// Whether the fused kernels handle this level (width >= 32, homogeneous rule).
bool fused_ok(Grid g, const Bc& bc);
// Whether cfg is a shape the fused kernels can run on g (zeros allowed).
bool fused_cfg_ok(Grid g, TileCfg cfg);
// One SMOOTH step from u_in (or 0) then fc = restriction of f - L u (Algorithm
// 1, steps 1-3).
cudaError_t launch_fused_down(const float* u_in, float* u_out, const float* f, float* fc, Grid g,
                              double h, Bc bc, double omega, bool zero_guess, cudaStream_t s,
                              TileCfg cfg = TileCfg{});
// u_in + trilinear(ec), then one SMOOTH step (Algorithm 1, steps 5-7).
cudaError_t launch_fused_up(const float* u_in, float* u_out, const float* f, const float* ec,
                            Grid g, double h, Bc bc, double omega, cudaStream_t s,
                            TileCfg cfg = TileCfg{});
// One SMOOTH step.
cudaError_t launch_fused_smooth(const float* u_in, float* u_out, const float* f, Grid g, double h,
                                Bc bc, double omega, bool zero_guess, cudaStream_t s,
                                TileCfg cfg = TileCfg{});

// The up leg of one V-cycle and the down leg of the next on the same level in
// one pass (Algorithm 1, steps 5-7 then 1-3): u_out = SMOOTH(SMOOTH(u_in +
// trilinear(ec))), fc = restriction of f - L u_out.  Levels with nx a multiple
// of 64, ny of 16 and nz >= 16 that fused_ok takes (updown_ok).
bool updown_ok(Grid g, const Bc& bc);
bool updown_cfg_ok(Grid g, TileCfg cfg);
cudaError_t launch_fused_updown(const float* u_in, float* u_out, const float* f, const float* ec,
                                float* fc, Grid g, double h, Bc bc, double omega, cudaStream_t s,
                                TileCfg cfg = TileCfg{});

// The periodic down leg with 64 x 32 tiles whose planes arrive by tensor copies
// (mg_fused_tma.cu); *err (device-visible) is set to 1 if a copy does not
// land in time.
bool down_tma_ok(Grid g, const Bc& bc);
cudaError_t launch_fused_down_tma(const float* u_in, float* u_out, const float* f, float* fc,
                                  Grid g, double h, double omega, bool zero_guess, int cz,
                                  int* err, cudaStream_t s);
// The periodic up leg with 64 x 16 tiles whose planes of u and f arrive by
// tensor copies (mg_fused_tma.cu); *err as for the down leg.
bool up_tma_ok(Grid g, const Bc& bc);
cudaError_t launch_fused_up_tma(const float* u_in, float* u_out, const float* f, const float* ec,
                                Grid g, double h, double omega, int cz, int* err, cudaStream_t s);
// A host-mapped flag (one per process, host and device share its address)
// for the leg-3 calls of mg_op_fused_leg; null if it cannot be had.
int* down_tma_op_flag();

// ---------------------------------------------------------------------------
// Exact 64-bit fixed-point outer residual (mg_fixed.cu).

// out[0] = max |a| (deterministic two-stage reduction through partials).
template <typename T>
cudaError_t launch_absmax(const T* a, long long n, double* partials, double* out, cudaStream_t s);
// In place: double -> round((a - mu) * c) as int64.  out = q * c - m as
// doubles (out may alias q), m = total[0] * cm when total is given.
cudaError_t launch_f64_to_fx(double* a, long long n, double mu, double c, cudaStream_t s);
// out[t] = (q[t] - *mean) 2^-S (mean may be null: 0); out may alias q.
cudaError_t launch_fx_to_f64(const long long* q, double* out, long long n, int S,
                             const long long* mean, cudaStream_t s);
// out[0] = sum rho, out[1] = max |rho| (n even; partials holds 2
// reduce_blocks(n / 2) doubles); reads rho only.
cudaError_t launch_convert(int kind, long long n, const void* in, void* out, cudaStream_t s);
// launch_rho_stats reading rho from (device-mapped) host memory and leaving
// its copy in dev.
cudaError_t launch_rho_stats_copy(const double* host_rho, double* dev, long long n,
                                  double* partials, double* out, cudaStream_t s);
cudaError_t launch_rho_stats(const double* rho, long long n, double* partials, double* out,
                             cudaStream_t s);
// out[0..3] = mu, scale, a, b of the source from the launch_rho_stats sums in
// st (on the device, so that no host round trip sits between the passes).
cudaError_t launch_source_scale(const double* st, long long n, double four_pi_G, bool has_mean,
                                double* out, cudaStream_t s);
// r32 = fl32(a rho - b); out[0] = sum r32^2, out[1] = max |r32|.  ab_dev: a
// and b from the device (launch_source_scale's out + 2) instead of the
// arguments.
cudaError_t launch_rho_to_r32(const double* rho, float* r32, long long n, double a, double b,
                              double* partials, double* out, cudaStream_t s,
                              const double* ab_dev = nullptr);
// q = round(a rho - b) as int64.
cudaError_t launch_rho_to_fx(const double* rho, long long* q, long long n, double a, double b,
                             cudaStream_t s);
// PHI += round(e * c); *flag |= 1 if |PHI| passes 2^60.
cudaError_t launch_fx_correct(long long* phi, const float* e, long long n, float c, int* flag,
                              cudaStream_t s);
// Fused outer step: PHI_out = PHI_in + round(e * c) (e must not be null; phi_in
// null means PHI_in = 0), then r32 = (F - (sum_nb PHI_out - 6 PHI_out)) *
// factor exactly in integers, one partial sum of r32^2 per block in partials
// (count in *nb_out, at most nb_max) and, when psum is given, the exact sum of
// PHI_out per block as a (hi 2^32, lo) pair of integers (2 nb_max entries).
// Requires nx % 32 == 0 and ny % 16 == 0 (fx_step_ok).
// cz = 0 takes the built-in planes per CTA; fx_step_blocks(g, 0) bounds the
// block count of every cz >= kFxMinCz.
constexpr int kFxMinCz = 4;
bool fx_step_ok(Grid g);
int fx_step_cz(Grid g, int cz);
int fx_step_blocks(Grid g, int cz);
cudaError_t launch_fx_step(const long long* phi_in, long long* phi_out, const float* e, float c,
                           const long long* F, float* r32, Grid g, const Bc& bc, double two_pow_S,
                           float factor, double* partials, int nb_max, int* flag, int* nb_out,
                           cudaStream_t s, int cz = 0, long long* psum = nullptr);
// phi = q 2^-S - m (m = total[0] * cm when total is given; phi must not alias
// q) and g = -grad phi at cell centres from the exact integer differences
// (Sec. 3.2.3), g = [gx | gy | gz].
cudaError_t launch_fx_finish_gravity(const long long* q, double* phi, double* g, Grid gr,
                                     const Bc& bc, double h, int S, const long long* mean,
                                     cudaStream_t s);
// out[0] = sum over nb blocks of the pairs launch_fx_step wrote, as a double;
// out[1] (as a long long) = that sum over n = 2^k cells, rounded to an integer.
cudaError_t launch_finish_fx_sum(const long long* psum, int nb, long long n, double* out,
                                 cudaStream_t s);

// ---------------------------------------------------------------------------
// Multipole boundary (App. A).

// Upload the polynomial tables to this device's constant memory (once per
// device; synchronous, so call it outside stream capture).
cudaError_t prepare_multipole();
// Raw moments sum rho x^a y^b z^c (a+b+c <= 4, 35 values) about the grid
// centre, written as per-block partials [nb][35]; returns nb via *nb_out.
cudaError_t launch_raw_moments(const double* rho, Grid g, double h, double* partials,
                               int* nb_out, cudaStream_t s);
// The same kernel on exactly nb blocks of 8 warps (one warp per row, rows
// strided over the nb * 8 warps); partials need nb * 35 doubles.
cudaError_t launch_raw_moments_blocks(const double* rho, Grid g, double h, double* partials,
                                      int nb, cudaStream_t s);
// Reduce the partials and form Q_lm (25) and the origin on the device:
// out[0..25) = Q, out[25..28) = origin, out[28] = total mass.
cudaError_t launch_moments_finish(const double* partials, int nb, double h, int lmax,
                                  int use_com, const double* origin_in, double* out,
                                  cudaStream_t s);
// Boundary values at every face point of a level from Q and the origin held
// in `qo` (layout of launch_moments_finish's output).
cudaError_t launch_open_faces(Grid g, double h, const double* qo, int lmax, double G,
                              double* faces, cudaStream_t s);
// A start value for phi under the open rule at every cell of level g: the
// monopole and dipole of the expansion in qo (as launch_open_faces reads it),
// -G (P_0 / r + P_1 / r^3) with r at least 1/8 of the shortest side.
cudaError_t launch_open_guess(double* phi, Grid g, double h, const double* qo, double G,
                              cudaStream_t s);

}  // namespace mg
