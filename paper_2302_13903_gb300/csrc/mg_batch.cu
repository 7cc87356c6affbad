// mg_batch.cu -- many independent grids solved by one persistent launch.
//
// Each grid is solved by the mixed-precision method of the single-grid path:
// an FP64 outer defect-correction loop (source, residual, correction and
// norms in FP64) around FP32 V(1,1) cycles on the correction equation
// (Algorithm 1 with the homogeneous rule on every level).  All grids advance
// together through a fixed list of phases; a phase is a set of independent
// work items (a tile of one grid's level, a chunk of one grid's finest level,
// or one whole grid) that the CTAs of a persistent cooperative kernel take
// from an atomic counter.  Phases are separated by a grid-wide barrier whose
// waits are bounded in time (on expiry the kernel records an error and every
// CTA returns).  Per grid, the stopping rule of the single-grid solve
// (||d||/||f|| < tol, stall, divergence, max_cycles) is applied after every
// outer iteration; a stopped grid's items become empty.
//
// Work items by phase:
//   source: f = 4 pi G rho, mean removal, ||f||     (chunks of 32768 cells)
//   first residual r = f - L(0), FP32 copy           (chunks)
//   per V-cycle: down legs on levels >= 64^3 (fused tiles), one CTA per grid
//     for the levels <= 32^3 (whole coarse cycle), up legs on levels >= 64^3
//   correction phi += e / scale, FP64 residual + norm (chunks), stopping rule
//     (one item per grid)
//   at the end: <phi> = 0 for periodic and zero-gradient grids (chunks)
// Partial sums live in per-chunk slots and are added in chunk order, so every
// result is independent of which CTA ran which item.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mg.h"
#include "mg_bottom.cuh"
#include "mg_convert.cuh"
#include "mg_device.cuh"
#include "mg_fused.cuh"
#include "mg_internal.h"

namespace mg {
namespace batch {

// The tile programs pad their shared rows (bank-conflict-free, as the
// single-grid kernels) at a cost of 9 KB per CTA of the shared memory the
// other phases could use as L1.
constexpr bool kPad = true;
constexpr int kThreads = fused::Shape<fused::kDown, 64, 16, 4, kPad>::NT;  // 216
constexpr size_t kSmem = fused::Shape<fused::kDown, 64, 16, 4, kPad>::SMEM;
static_assert(fused::Shape<fused::kUp, 64, 16, 4, kPad>::SMEM <= kSmem &&
                  fused::Shape<fused::kUp, 32, 16, 4, kPad>::SMEM <= kSmem,
              "an up-leg tile needs more shared memory than the CTA has");
constexpr int kMaxL = 16;
constexpr int kChunk = 32768;   // cells per chunk item
constexpr int kFusedMinN = 32;  // levels of at least 32^3 use the fused tiles
constexpr int kCz = 64;         // z-chunk of fused tiles
constexpr long long kBarrierCycles = 4000000000LL;  // ~2 s at 2 GHz

struct GridDev {
  int n, L, bc;
  double h, bcval, fpg, tol;
  const double* rho;
  double* phi;
  double* f64;
  float* u32[kMaxL];
  float* u32b[kMaxL];
  float* f32[kMaxL];
  int chunk0, nchunk;  // this grid's chunk items (same layout in every chunk phase)
  // state
  double mean, fnorm, rn, scale, prev, d0;
  int stalls, active, status, nh, cycles;
  int skip;  // this grid has no request in this solve: every phase passes it by
  // fixed-point outer loop: phi and h^2 f as integers scaled by two_S
  double maxf, two_S;
  int S;            // two_S = 2^S
  long long imean;  // PHI's mean rounded to an integer (periodic / zero gradient), else 0
  long long b2;  // FIXED: round(2 b 2^S), the integer ghost offset
  int in_fx, fxbad;
  long long* fx2;      // second integer buffer (the outer step writes the other one)
  int cur;             // which buffer holds PHI: 0 phi's own storage, 1 fx2
  int part0, ntile;    // this grid's tiles of the fixed-point step (partials in part3)
};

enum PhaseType : int {
  PH_SRC = 0,      // chunk: partial sum and maximum of rho
  PH_MEANFIN,      // grid: mean of f (periodic / zero gradient), the FP32 scale
  PH_R0,           // chunk: r = f - mean - L(0) -> r32 (scaled), sums of (f - mean)^2, r^2
  PH_R0FIN,        // grid: ||f||, rn
  PH_DOWN,         // tile: fused down leg on level size `n`
  PH_BOTTOM,       // grid: levels <= 32^3 of one V-cycle
  PH_UP,           // tile: fused up leg on level size `n`
  PH_EMAX,         // chunk: max |e| (first outer iteration)
  PH_SETFX,        // grid: the fixed-point scale 2^S
  PH_TOFX,         // chunk: F = round(h^2 f 2^S)
  PH_FXSTEP,       // tile: PHI' = PHI + round(e 2^S / scale), exact residual -> r32
  PH_FIN,          // grid: stopping rule, history
  PH_PSUM,         // chunk: partial sum phi (exact integer sum in fixed point)
  PH_PMEAN,        // grid: mean of phi
  PH_PSUB          // chunk: phi = PHI 2^-S - mean (fixed point) or phi -= mean
};

struct Phase {
  int type;
  int n;       // level size (DOWN / UP)
  int first;   // first item in the item list
  int count;   // items
  int cycle;   // inner cycle index within the outer iteration (DOWN / BOTTOM)
};

struct Item {
  int grid, a, b, c;
};

struct Ctl {
  const Phase* phases;
  const Item* items;
  GridDev* grids;
  double* part;        // one slot per chunk
  double* part2;       // a second slot per chunk (maxima)
  long long* ipart;    // two integer slots per chunk (exact sums of PHI: hi, lo)
  double* part3;       // one slot per tile of the fixed-point step
  double* hist;        // [ngrids][hist_cap]
  unsigned* counters;  // one per phase
  unsigned* bar_count;
  unsigned* bar_gen;
  int* err;
  int* active_left;    // grids still active, after each FIN phase (index = phase)
  unsigned long long* ptime;  // [nphases + 1]: end of each phase, [nphases] = start (ns)
  int nphases, ngrids, hist_cap;
  double omega;
  int max_cycles, inner_zero;
  double stall_ratio;
  long long bar_cycles;  // a barrier wait gives up after this many clock cycles
};

__device__ bool grid_barrier(const Ctl& c) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = c.bar_gen;
    const unsigned g0 = *gen;
    __threadfence();
    if (atomicAdd(c.bar_count, 1u) == gridDim.x - 1) {
      *c.bar_count = 0;
      __threadfence();
      atomicAdd(c.bar_gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g0) {
        if (clock64() - t0 > c.bar_cycles) {
          atomicOr(c.err, 1);
          break;
        }
        __nanosleep(256);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *((volatile int*)c.err) == 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int level_of(const GridDev& g, int n) {
  int l = g.L - 1, m = g.n;
  while (m > n) {
    m >>= 1;
    --l;
  }
  return l;
}

__device__ __forceinline__ Bc phys_bc(const GridDev& g) { return Bc{g.bc, g.bcval, nullptr}; }
__device__ __forceinline__ Bc hom_bc(const GridDev& g) {
  return Bc{g.bc == BC_FIXED ? BC_FIXED : g.bc, 0.0, nullptr};
}

// Reductions over the CTA (not a whole number of warps: the values are padded
// with the operation's identity to whole warps in shared memory); warp 0's
// lanes combine every 32nd value, then a shuffle tree.  A fixed order, so the
// results do not depend on timing; valid in thread 0.
constexpr int kPadThreads = (kThreads + 31) / 32 * 32;

template <typename T, typename Op>
__device__ __forceinline__ T block_reduce_pad(T v, T identity, Op op) {
  __shared__ T w[kPadThreads];
  w[threadIdx.x] = v;
  if (threadIdx.x < kPadThreads - (int)blockDim.x) w[blockDim.x + threadIdx.x] = identity;
  __syncthreads();
  T r = identity;
  if (threadIdx.x < 32) {
    for (int q = threadIdx.x; q < kPadThreads; q += 32) r = op(r, w[q]);
    for (int o = 16; o > 0; o >>= 1) r = op(r, __shfl_down_sync(0xffffffffu, r, o));
  }
  __syncthreads();
  return r;
}

__device__ double block_sum(double v) {
  return block_reduce_pad(v, 0.0, [](double a, double b) { return a + b; });
}
__device__ double block_max(double v) {
  return block_reduce_pad(v, 0.0, [](double a, double b) { return fmax(a, b); });
}
__device__ long long block_isum(long long v) {
  return block_reduce_pad(v, 0LL, [](long long a, long long b) { return a + b; });
}

// One chunk of the finest level: cells [c * kChunk, min(N, (c + 1) kChunk)).
// The grid's fields are read once into registers (the loop's stores could
// otherwise alias them).
template <int TYPE>
__device__ void chunk_item(const Ctl& c, GridDev& g, int chunk) {
  const int n = g.n, lg = g.L - 1;  // n = 2^lg
  const Grid gr{n, n, n};
  const int N = n * n * n;  // <= 1024^3 = 2^30
  const int lo = chunk * kChunk, hi = min(N, lo + kChunk);
  const int F = g.L - 1;
  double* phi = g.phi;
  // the integer potential: in phi's own storage or in the second buffer
  const long long* PHI = g.cur ? g.fx2 : reinterpret_cast<const long long*>(g.phi);  // may be phi
  long long* __restrict__ FX = reinterpret_cast<long long*>(g.f64);
  const double* __restrict__ rho = g.rho;
  float* __restrict__ r32 = g.f32[F];
  const float* __restrict__ e32 = g.u32[F];
  const double fpg = g.fpg, mean = g.mean, h = g.h;
  const double inv_h2 = 1.0 / (h * h), bcval = g.bcval;
  const int bc = g.bc;
  const bool fx = g.in_fx != 0;
  const double two_S = g.two_S;
  double acc = 0.0, mx = 0.0;
  long long s_hi = 0, s_lo = 0;
  // unrolled so that each thread has several independent loads in flight
  // f = 4 pi G rho is never stored: each pass forms what it needs from rho
  const double sc = g.scale;  // r32 = (f - mean - L(0)) sc
  const double a0 = fpg * sc, b0 = mean * sc;
  const float bt = (float)(2.0 * bcval * inv_h2 * sc);  // one fixed-value ghost term, scaled
  const double c2 = h * h * two_S;
  float af = 0.f, ar = 0.f;  // FP32 sums over at most 8 cells, then added in FP64
  double acc2 = 0.0;
  int nf = 0;
  unsigned long long mb = 0;  // largest |rho| bit pattern
  // two cells per step (16-byte loads) and the loop unrolled by eight, so that
  // each thread keeps several independent loads in flight: the CTA is small
  // (two per SM), and these passes are bound by memory latency
  const double2* __restrict__ rho2 = reinterpret_cast<const double2*>(rho);
  auto r0_cell = [&](int t, double v) {
    const float x = cvt::d2f_rn(fma(a0, v, -b0));  // (f - mean) sc
    float xs = x;
    if (bc == BC_FIXED && bcval != 0.0) {  // L_h(0): 2 b per fixed-value ghost
      const int i = t & (n - 1), j = (t >> lg) & (n - 1), k = t >> (2 * lg);
      const int faces = (i == 0) + (i == n - 1) + (j == 0) + (j == n - 1) + (k == 0) + (k == n - 1);
      xs = x - (float)faces * bt;
    }
    af = fmaf(x, x, af);
    ar = fmaf(xs, xs, ar);
    return xs;
  };
  if (TYPE == PH_TOFX || TYPE == PH_PSUB) {
    // pure streams: four 16-byte loads in flight per thread before their
    // stores (each element is read before it is written, so PHI may be phi)
    const double a = fpg * c2, b = mean * c2;
    auto tofx = [&](double2 v) {
      return make_longlong2(cvt::d2ll_rn(fma(a, v.x, -b)), cvt::d2ll_rn(fma(a, v.y, -b)));
    };
    auto psub = [&](longlong2 v) {
      return fx ? make_double2(cvt::ll2d_pow2_rn(v.x - g.imean, g.S),
                               cvt::ll2d_pow2_rn(v.y - g.imean, g.S))
                : make_double2(0.0, 0.0);
    };
    const int stride = blockDim.x, e2 = hi >> 1;
    int t2 = (lo >> 1) + threadIdx.x;
    for (; t2 + 3 * stride < e2; t2 += 4 * stride) {
      if (TYPE == PH_TOFX) {
        double2 v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = rho2[t2 + q * stride];
#pragma unroll
        for (int q = 0; q < 4; ++q) reinterpret_cast<longlong2*>(FX)[t2 + q * stride] = tofx(v[q]);
      } else {
        longlong2 v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = reinterpret_cast<const longlong2*>(PHI)[t2 + q * stride];
#pragma unroll
        for (int q = 0; q < 4; ++q) reinterpret_cast<double2*>(phi)[t2 + q * stride] = psub(v[q]);
      }
    }
    for (; t2 < e2; t2 += stride) {
      if (TYPE == PH_TOFX) reinterpret_cast<longlong2*>(FX)[t2] = tofx(rho2[t2]);
      else reinterpret_cast<double2*>(phi)[t2] = psub(reinterpret_cast<const longlong2*>(PHI)[t2]);
    }
    return;
  }
  // the first residual: each thread's cells in the same order as one at a
  // time, with four 16-byte loads in flight ahead of their use
  const int stride = blockDim.x, e2 = hi >> 1;
  auto r0_pair = [&](int t2, double2 v) {
    const int t = 2 * t2;  // cells t, t + 1 (lo, hi and N are even)
    const float x0 = r0_cell(t, v.x), x1 = r0_cell(t + 1, v.y);
    reinterpret_cast<float2*>(r32)[t2] = make_float2(x0, x1);
    if (++nf == 4) {  // FP32 sums over at most 8 cells, then added in FP64
      acc += af;
      acc2 += ar;
      af = ar = 0.f;
      nf = 0;
    }
  };
  if (TYPE == PH_R0) {
    int t2 = (lo >> 1) + threadIdx.x;
    for (; t2 + 3 * stride < e2; t2 += 4 * stride) {
      double2 v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = rho2[t2 + q * stride];
#pragma unroll
      for (int q = 0; q < 4; ++q) r0_pair(t2 + q * stride, v[q]);
    }
    for (; t2 < e2; t2 += stride) r0_pair(t2, rho2[t2]);
  }
#pragma unroll 8
  for (int t2 = (lo >> 1) + threadIdx.x; TYPE != PH_R0 && t2 < e2; t2 += stride) {
    if (TYPE == PH_SRC) {
      const double2 v = rho2[t2];
      acc += v.x + v.y;
      const unsigned long long b0 = (unsigned long long)__double_as_longlong(v.x) & 0x7fffffffffffffffULL;
      const unsigned long long b1 = (unsigned long long)__double_as_longlong(v.y) & 0x7fffffffffffffffULL;
      mb = b0 > mb ? b0 : mb;
      mb = b1 > mb ? b1 : mb;
    } else if (TYPE == PH_EMAX) {
      const float2 v = reinterpret_cast<const float2*>(e32)[t2];
      mx = fmax(mx, (double)fmaxf(fabsf(v.x), fabsf(v.y)));
    } else if (TYPE == PH_PSUM) {
      const longlong2 v = reinterpret_cast<const longlong2*>(PHI)[t2];
      s_hi += (v.x >> 32) + (v.y >> 32);
      s_lo += (v.x & 0xffffffffLL) + (v.y & 0xffffffffLL);
    }
  }
  if (TYPE == PH_R0) {
    acc += af;
    acc2 += ar;
  }
  if (TYPE == PH_SRC || TYPE == PH_R0) {
    const double b = block_sum(acc);
    if (threadIdx.x == 0) c.part[g.chunk0 + chunk] = b;
  }
  if (TYPE == PH_R0) {
    const double b = block_sum(acc2);
    if (threadIdx.x == 0) c.part2[g.chunk0 + chunk] = b;
  }
  if (TYPE == PH_SRC) mx = __longlong_as_double((long long)mb);
  if (TYPE == PH_SRC || TYPE == PH_EMAX) {
    const double b = block_max(mx);
    if (threadIdx.x == 0) c.part2[g.chunk0 + chunk] = b;
  }
  if (TYPE == PH_PSUM) {
    const long long bh = block_isum(s_hi), bl = block_isum(s_lo);
    if (threadIdx.x == 0) {
      c.ipart[2 * (g.chunk0 + chunk)] = bh;
      c.ipart[2 * (g.chunk0 + chunk) + 1] = bl;
    }
  }
}

__device__ double chunk_max(const Ctl& c, const GridDev& g) {
  double m = 0.0;
  for (int q = 0; q < g.nchunk; ++q) m = fmax(m, c.part2[g.chunk0 + q]);
  return m;
}

// The fixed-point scale of one grid after its first inner solve: 2^S the
// largest power of two keeping |PHI| < 2^55 and |h^2 f 2^S| < 2^58.
__device__ void setfx_item(const Ctl& c, GridDev& g) {
  const double mphi = chunk_max(c, g) / g.scale;  // phi = e / scale after this step
  const double mfh = g.maxf * g.h * g.h;
  double lim = 0.0;
  if (mphi > 0.0) lim = 36028797018963968.0 / mphi;                    // 2^55
  if (mfh > 0.0 && (lim == 0.0 || 288230376151711744.0 / mfh < lim))  // 2^58
    lim = 288230376151711744.0 / mfh;
  if (lim == 0.0) lim = 36028797018963968.0;
  int e2 = 0;
  frexp(lim, &e2);
  g.S = e2 - 1;
  g.two_S = ldexp(1.0, e2 - 1);
  g.b2 = g.bc == BC_FIXED ? __double2ll_rn(2.0 * g.bcval * g.two_S) : 0;
  g.in_fx = 1;
}

__device__ double chunk_total(const Ctl& c, const GridDev& g) {
  double s = 0.0;
  for (int q = 0; q < g.nchunk; ++q) s += c.part[g.chunk0 + q];
  return s;
}

// Tile sizes of the fixed-point step: TX x TY columns, FXCZ planes.
__host__ __device__ inline int fx_tx(int n) { return n < 32 ? n : 32; }
__host__ __device__ inline int fx_ty(int n) { return n < 16 ? n : 16; }
__host__ __device__ inline int fx_cz(int n) { return n < 32 ? n : 32; }
constexpr int kFxCols = 3;  // columns per thread (32 x 16 = 512 <= 3 x 216)

// One tile of the fused outer step on the integer grid (z-marching, as the
// single-grid kernel): PHI' = PHI + round(e 2^S / scale) (PHI = 0 on the
// first step), R = F - (sum_nb PHI' - 6 PHI') exactly, r32 = R / (rn h^2 2^S)
// with one partial sum of r32^2 per tile; PHI' goes to the other buffer.
// Each thread owns up to three columns, keeping PHI' of planes z-1, z, z+1 in
// registers; x / y neighbours come from the current plane in shared memory,
// whose halo the first threads load and correct.
// Asynchronous global -> shared copies of 8 or 4 bytes (src_bytes 0 fills
// zeros) for the outer step's staging ring.
__device__ __forceinline__ void ring_cp8(void* dst, const void* src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void ring_cp4(void* dst, const void* src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src),
               "r"(src_bytes)
               : "memory");
}

// Staging ring of the outer step in the CTA's dynamic shared memory, after
// the two halo planes: per plane, each thread's columns' PHI, F and e and its
// halo cell's PHI and e.  A thread reads back only what it copied itself.
constexpr int kRing = 4;
constexpr size_t kPlaneBytes = 2 * 18 * 34 * sizeof(long long);  // [2][TY+2][TX+2], TX, TY <= 32, 16
struct TileRing {
  long long p[kRing][kFxCols][kThreads];
  long long f[kRing][kFxCols][kThreads];
  float e[kRing][kFxCols][kThreads];
  long long hp[kRing][kThreads];
  float he[kRing][kThreads];
};
static_assert(kPlaneBytes + sizeof(TileRing) <= kSmem, "outer-step ring exceeds the CTA's smem");

__device__ void fx_tile_item(const Ctl& c, GridDev& g, const Item& I, bool zero_in,
                             float4* smem) {
  const int n = g.n, TX = fx_tx(n), TY = fx_ty(n), CZ = fx_cz(n);
  const int W = TX + 2, H = TY + 2, cols = TX * TY, nhalo = 2 * W + 2 * TY;
  const int x0 = I.a * TX, y0 = I.b * TY, z0 = I.c * CZ, z1 = z0 + CZ;
  const int F = g.L - 1;
  const bool per = g.bc == BC_PERIODIC;
  const long long* pin = g.cur ? g.fx2 : reinterpret_cast<const long long*>(g.phi);
  long long* __restrict__ pout = g.cur ? reinterpret_cast<long long*>(g.phi) : g.fx2;
  const long long* FX = reinterpret_cast<const long long*>(g.f64);
  const float* e = g.u32[F];
  float* __restrict__ r32 = g.f32[F];
  const float ce = (float)(g.two_S / g.scale);
  const float rfac = (float)(1.0 / (g.rn * g.h * g.h * g.two_S));
  const long long b2 = g.b2;
  const int bc = g.bc;
  const int tid = threadIdx.x;
  const size_t plane = (size_t)n * n;
  long long* P = reinterpret_cast<long long*>(smem);  // [2][H][W]
  TileRing& ring = *reinterpret_cast<TileRing*>(reinterpret_cast<char*>(smem) + kPlaneBytes);
  auto wrapq = [&](int q) { return q < 0 ? q + n : (q >= n ? q - n : q); };
  // this thread's columns
  int ci[kFxCols], cj[kFxCols];
  bool cact[kFxCols];
#pragma unroll
  for (int q = 0; q < kFxCols; ++q) {
    const int col = tid + q * kThreads;
    cact[q] = col < cols;
    ci[q] = x0 + (cact[q] ? col % TX : 0);
    cj[q] = y0 + (cact[q] ? col / TX : 0);
  }
  // this thread's halo cell (rows -1 and TY over the full width, columns -1
  // and TX over the tile's rows)
  const bool halo = tid < nhalo;
  int ha = 0, hb = 0;
  if (halo) {
    const int h = tid;
    if (h < W) { ha = h; hb = 0; }
    else if (h < 2 * W) { ha = h - W; hb = H - 1; }
    else if (h < 2 * W + TY) { ha = 0; hb = h - 2 * W + 1; }
    else { ha = W - 1; hb = h - 2 * W - TY + 1; }
  }
  int hx = x0 - 1 + ha, hy = y0 - 1 + hb;
  bool h_in = halo;
  if (per) {
    hx = wrapq(hx);
    hy = wrapq(hy);
  } else {
    h_in = h_in && hx >= 0 && hx < n && hy >= 0 && hy < n;
  }
  const size_t hcol = h_in ? (size_t)hy * n + hx : 0;
  auto slot = [&](int q) { return (q - z0 + 1) & (kRing - 1); };
  // copies for plane q: the columns' PHI and e (z0-1 <= q <= z1, zeros outside
  // a non-periodic grid), F and the halo cell (z0 <= q < z1)
  auto issue = [&](int q) {
    if (q <= z1) {
      const int sl = slot(q);
      const bool in = per || (q >= 0 && q < n);
      const int qw = per ? wrapq(q) : (in ? q : 0);
#pragma unroll
      for (int k = 0; k < kFxCols; ++k) {
        if (!cact[k]) continue;
        const size_t o = (size_t)qw * plane + (size_t)cj[k] * n + ci[k];
        if (!zero_in) ring_cp8(&ring.p[sl][k][tid], pin + o, in ? 8 : 0);
        ring_cp4(&ring.e[sl][k][tid], e + o, in ? 4 : 0);
        if (q >= z0 && q < z1)
          ring_cp8(&ring.f[sl][k][tid], FX + (size_t)q * plane + (size_t)cj[k] * n + ci[k], 8);
      }
      if (halo && q >= z0 && q < z1) {
        const size_t ho = (size_t)q * plane + hcol;
        if (!zero_in) ring_cp8(&ring.hp[sl][tid], pin + ho, h_in ? 8 : 0);
        ring_cp4(&ring.he[sl][tid], e + ho, h_in ? 4 : 0);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  auto own_at = [&](int k, int q) -> long long {
    const int sl = slot(q);
    const long long v = zero_in ? 0 : ring.p[sl][k][tid];
    return v + __float2ll_rn(ring.e[sl][k][tid] * ce);
  };
  issue(z0 - 1);
  issue(z0);
  issue(z0 + 1);
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // planes z0 - 1, z0 landed
  long long zm[kFxCols], self[kFxCols];
#pragma unroll
  for (int k = 0; k < kFxCols; ++k) {
    zm[k] = cact[k] ? own_at(k, z0 - 1) : 0;
    self[k] = cact[k] ? own_at(k, z0) : 0;
  }
  float acc = 0.f;
  bool bad = false;
  for (int z = z0; z < z1; ++z) {
    issue(z + 2);
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // every plane up to z + 1
    const int sl = slot(z);
    const int buf = (z - z0) & 1;
    long long* Pb = P + (size_t)buf * H * W;
#pragma unroll
    for (int k = 0; k < kFxCols; ++k) {
      if (!cact[k]) continue;
      Pb[(cj[k] - y0 + 1) * W + (ci[k] - x0 + 1)] = self[k];
      pout[(size_t)z * plane + (size_t)cj[k] * n + ci[k]] = self[k];
      bad |= (self[k] > (1LL << 60)) || (self[k] < -(1LL << 60));
    }
    if (halo) {
      const long long hv = (zero_in ? 0 : ring.hp[sl][tid]) + __float2ll_rn(ring.he[sl][tid] * ce);
      Pb[hb * W + ha] = h_in ? hv : 0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kFxCols; ++k) {
      if (!cact[k]) continue;
      const int i = ci[k], j = cj[k], a = i - x0 + 1, bb = j - y0 + 1;
      const long long sv = self[k];
      const long long zp = own_at(k, z + 1);
      long long xm = Pb[bb * W + a - 1], xp = Pb[bb * W + a + 1];
      long long ym = Pb[(bb - 1) * W + a], yp = Pb[(bb + 1) * W + a];
      long long zmv = zm[k], zpv = zp;
      if (!per) {
        const long long gh = bc == BC_ZEROGRAD ? sv : b2 - sv;
        if (i == 0) xm = gh;
        if (i == n - 1) xp = gh;
        if (j == 0) ym = gh;
        if (j == n - 1) yp = gh;
        if (z == 0) zmv = gh;
        if (z == n - 1) zpv = gh;
      }
      const size_t o = (size_t)z * plane + (size_t)j * n + i;
      const long long R = ring.f[sl][k][tid] - (((xm + xp) + (ym + yp)) + (zmv + zpv) - 6 * sv);
      const float r = __ll2float_rn(R) * rfac;
      r32[o] = r;
      acc = fmaf(r, r, acc);
      zm[k] = sv;
      self[k] = zp;
    }
    // the next plane writes the other half of P; this one is rewritten two
    // planes on, after every thread has passed the next barrier
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  if (bad) atomicOr(&g.fxbad, 1);
  const double b = block_sum((double)acc);
  if (threadIdx.x == 0) c.part3[g.part0 + (I.c * (n / TY) + I.b) * (n / TX) + I.a] = b;
}

// Stopping rule of the single-grid solve, after one outer iteration.
__device__ void fin_item(const Ctl& c, GridDev& g, int gi) {
  const double N = (double)g.n * g.n * g.n;
  // the outer step summed the squares of r32 = r / rn_previous, per tile
  double tot = 0.0;
  for (int q = 0; q < g.ntile; ++q) tot += c.part3[g.part0 + q];
  const double rn = sqrt(tot / N) * g.rn;
  g.cur ^= 1;  // the step wrote the other integer buffer
  double r = rn / g.fnorm;
  if (g.fxbad) r = NAN;  // the integers passed 2^60: the solve diverged
  g.scale = 1.0 / g.rn;  // the scale the residual just written used
  g.rn = rn;
  if (g.nh < c.hist_cap) c.hist[(size_t)gi * c.hist_cap + g.nh] = r;
  g.nh++;
  g.cycles++;
  if (g.prev >= 0.0) g.stalls = (r > c.stall_ratio * g.prev) ? g.stalls + 1 : 0;
  g.prev = r;
  if (g.d0 < 0.0) g.d0 = r;
  int st = -1;
  if (isnan(r) || isinf(r) || r > 10.0 * g.d0) st = MG_ERR_DIVERGED;
  else if (r < g.tol) st = MG_OK;
  else if (g.stalls >= 2) st = g.tol == 0.0 ? MG_OK : MG_ERR_NOT_CONVERGED;
  else if (g.cycles >= c.max_cycles || g.nh >= c.hist_cap) st = MG_ERR_NOT_CONVERGED;
  if (st >= 0) {
    g.status = st;
    g.active = 0;
  }
}

// One tile item of a fused leg on level l: tiles TX x 16 cells, the chunk's
// planes; the down leg starts from zero on coarse levels and, when asked, on
// the finest.
template <int TX>
__device__ __forceinline__ void tile_leg(bool down, bool per, const GridDev& g, int l,
                                         bool zero_finest, const fused::FusedParams& fp,
                                         const Item& I, float4* smem) {
  if (down) {
    const bool zg = (l < g.L - 1) || zero_finest;
    if (zg) {
      if (per)
        fused::fused_tile<fused::kDown, true, 7, TX, 16, 4, kPad, kThreads>(
            g.u32[l], g.u32b[l], g.f32[l], nullptr, g.f32[l - 1], fp, I.a, I.b, I.c, smem);
      else
        fused::fused_tile<fused::kDown, true, 0, TX, 16, 4, kPad, kThreads>(
            g.u32[l], g.u32b[l], g.f32[l], nullptr, g.f32[l - 1], fp, I.a, I.b, I.c, smem);
    } else {
      if (per)
        fused::fused_tile<fused::kDown, false, 7, TX, 16, 4, kPad, kThreads>(
            g.u32[l], g.u32b[l], g.f32[l], nullptr, g.f32[l - 1], fp, I.a, I.b, I.c, smem);
      else
        fused::fused_tile<fused::kDown, false, 0, TX, 16, 4, kPad, kThreads>(
            g.u32[l], g.u32b[l], g.f32[l], nullptr, g.f32[l - 1], fp, I.a, I.b, I.c, smem);
    }
  } else {
    if (per)
      fused::fused_tile<fused::kUp, false, 7, TX, 16, 4, kPad, kThreads>(
          g.u32b[l], g.u32[l], g.f32[l], g.u32[l - 1], nullptr, fp, I.a, I.b, I.c, smem);
    else
      fused::fused_tile<fused::kUp, false, 0, TX, 16, 4, kPad, kThreads>(
          g.u32b[l], g.u32[l], g.f32[l], g.u32[l - 1], nullptr, fp, I.a, I.b, I.c, smem);
  }
}

__global__ void __launch_bounds__(kThreads, 2) k_batch(Ctl c) {
  extern __shared__ float4 smem[];
  if (blockIdx.x == 0 && threadIdx.x == 0) c.ptime[c.nphases] = global_ns();
  for (int ph = 0; ph < c.nphases; ++ph) {
    const Phase P = c.phases[ph];
    __shared__ int s_item;
    for (;;) {
      if (threadIdx.x == 0) s_item = (int)atomicAdd(&c.counters[ph], 1u);
      __syncthreads();
      const int it = s_item;
      __syncthreads();
      if (it >= P.count) break;
      const Item I = c.items[P.first + it];
      GridDev& g = c.grids[I.grid];
      const bool has_mean = g.bc == BC_PERIODIC || g.bc == BC_ZEROGRAD;
      const bool run =
          !g.skip && (P.type == PH_PSUM ? has_mean : (P.type > PH_PSUM || g.active));
      if (!run) continue;
      switch (P.type) {
        case PH_SRC: chunk_item<PH_SRC>(c, g, I.a); break;
        case PH_R0: chunk_item<PH_R0>(c, g, I.a); break;
        case PH_EMAX: chunk_item<PH_EMAX>(c, g, I.a); break;
        case PH_TOFX: chunk_item<PH_TOFX>(c, g, I.a); break;
        case PH_SETFX:
          if (threadIdx.x == 0) setfx_item(c, g);
          break;
        case PH_FXSTEP:
          fx_tile_item(c, g, I, P.cycle != 0, smem);
          break;
        case PH_PSUM: chunk_item<PH_PSUM>(c, g, I.a); break;
        case PH_PSUB: chunk_item<PH_PSUB>(c, g, I.a); break;
        case PH_MEANFIN:
          if (threadIdx.x == 0) {
            const double N = (double)g.n * g.n * g.n;
            g.mean = (g.bc == BC_PERIODIC || g.bc == BC_ZEROGRAD) ? g.fpg * (chunk_total(c, g) / N)
                                                                  : 0.0;
            // max |f - mean| <= |4 pi G| max |rho| + |mean|: the scale of r32 and of 2^S
            g.maxf = fabs(g.fpg) * chunk_max(c, g) + fabs(g.mean);
            g.scale = g.maxf > 0.0 ? 1.0 / g.maxf : 1.0;
          }
          break;
        case PH_PMEAN:
          if (threadIdx.x == 0) {
            const double N = (double)g.n * g.n * g.n;
            double m = 0.0;
            if (g.bc == BC_PERIODIC || g.bc == BC_ZEROGRAD) {
              if (g.in_fx) {  // exact integer total, independent of the chunking
                long long th = 0, tl = 0;
                for (int q = 0; q < g.nchunk; ++q) {
                  th += c.ipart[2 * (g.chunk0 + q)];
                  tl += c.ipart[2 * (g.chunk0 + q) + 1];
                }
                m = ((double)th * 4294967296.0 + (double)tl) / (N * g.two_S);
                // the same mean as an integer, exactly: the 128-bit sum th 2^32 + tl
                // over N = 2^(3 lg) cells, rounded (ties up)
                const int k = 3 * (g.L - 1);
                const unsigned long long t = (unsigned long long)th << 32;
                unsigned long long lo = t + (unsigned long long)tl;
                long long hi = (th >> 32) + (tl < 0 ? -1 : 0) + (lo < t ? 1 : 0);
                if (k > 0) {
                  const unsigned long long lo2 = lo + (1ULL << (k - 1));
                  hi += lo2 < lo ? 1 : 0;
                  g.imean = (long long)((lo2 >> k) | ((unsigned long long)hi << (64 - k)));
                } else {
                  g.imean = (long long)lo;
                }
              }  // otherwise phi = 0 exactly (the grid stopped at its first residual)
            }
            g.mean = m;
          }
          break;
        case PH_R0FIN:
          if (threadIdx.x == 0) {
            const double N = (double)g.n * g.n * g.n;
            double fs = 0.0, rs = 0.0;  // sums of ((f - mean) sc)^2 and (r0 sc)^2
            for (int q = 0; q < g.nchunk; ++q) {
              fs += c.part[g.chunk0 + q];
              rs += c.part2[g.chunk0 + q];
            }
            g.fnorm = sqrt(fs / N) / g.scale;
            g.rn = sqrt(rs / N) / g.scale;
            if (g.fnorm == 0.0) g.fnorm = g.rn > 0.0 ? g.rn : 1.0;
            if (g.rn == 0.0) {  // phi = 0 is exact
              g.active = 0;
              g.status = MG_OK;
              if (c.hist_cap > 0) c.hist[(size_t)I.grid * c.hist_cap] = 0.0;
              g.nh = 1;
            }
          }
          break;
        case PH_FIN:
          if (threadIdx.x == 0) {
            fin_item(c, g, I.grid);
            if (g.active) atomicAdd(&c.active_left[ph], 1);
          }
          break;
        case PH_BOTTOM: {
          // the arguments in shared memory: their per-level arrays are indexed
          // by a run-time level, which in each thread's own copy would put
          // them in local memory
          __shared__ bottom::BottomArgs<float> a;
          const int top = level_of(g, min(g.n, kFusedMinN / 2));
          if (threadIdx.x == 0) {
            for (int l = 0; l < kBottomLevels; ++l) {
              const bool used = l <= top;
              a.u[l] = used ? g.u32[l] : nullptr;
              a.f[l] = used ? g.f32[l] : nullptr;
              a.n[l] = used ? (g.n >> (g.L - 1 - l)) : 0;
              a.h[l] = used ? g.h * (double)(1 << (g.L - 1 - l)) : 0.0;
              a.bc[l] = hom_bc(g);
            }
            a.hom = hom_bc(g);
            a.omega = c.omega;
            a.pre = 1;
            a.post = 1;
            a.top = top;
            a.fmg = 0;
            bottom::set_coefficients(a);
          }
          __syncthreads();
          const bool zg = (top < g.L - 1) || (P.cycle == 0 && c.inner_zero);
          bottom::vcycle<float, false>(a, top, a.hom, zg);
          break;
        }
        case PH_DOWN:
        case PH_UP: {
          const int l = level_of(g, P.n);
          const double hl = g.h * (double)(1 << (g.L - 1 - l));
          fused::FusedParams fp;
          fp.nx = fp.ny = fp.nz = P.n;
          fp.sx0 = fp.sx1 = fp.sy0 = fp.sy1 = fp.sz0 = fp.sz1 = g.bc == BC_ZEROGRAD ? 1.f : -1.f;
          fp.cu = (float)(1.0 - c.omega);
          fp.cs = (float)(c.omega / 6.0);
          fp.cf = (float)(-c.omega * hl * hl / 6.0);
          fp.inv_h2 = (float)(1.0 / (hl * hl));
          fp.cz = kCz < P.n ? kCz : P.n;
          const bool per = g.bc == BC_PERIODIC;
          if (P.n >= 64)
            tile_leg<64>(P.type == PH_DOWN, per, g, l, P.cycle == 0 && c.inner_zero, fp, I, smem);
          else
            tile_leg<32>(P.type == PH_DOWN, per, g, l, P.cycle == 0 && c.inner_zero, fp, I, smem);
          break;
        }
      }
      __syncthreads();
    }
    if (!grid_barrier(c)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) c.ptime[ph] = global_ns();
    if (P.type == PH_FIN && *((volatile int*)&c.active_left[ph]) == 0) {
      // every grid has stopped: go to the final mean removal
      int q = ph + 1;
      while (q < c.nphases && c.phases[q].type < PH_PSUM) ++q;
      ph = q - 1;
    }
  }
}

}  // namespace batch
}  // namespace mg

using namespace mg;
using namespace mg::batch;

struct mg_batch {
  int ngrids = 0;
  mg_opts opts{};
  int device = 0;
  std::vector<GridDev> host_grids;  // pointers and sizes (state fields reset per solve)
  GridDev* d_grids = nullptr;
  GridDev* h_grids = nullptr;  // pinned staging
  Phase* d_phases = nullptr;
  Item* d_items = nullptr;
  double* d_part = nullptr;
  double* d_part2 = nullptr;
  long long* d_ipart = nullptr;
  double* d_part3 = nullptr;
  double* d_hist = nullptr;
  double* h_hist = nullptr;  // pinned
  unsigned* d_counters = nullptr;
  unsigned* d_bar = nullptr;
  int* d_err = nullptr;
  int* d_active = nullptr;
  unsigned long long* d_ptime = nullptr;
  std::vector<Phase> host_phases;
  int* h_err = nullptr;
  int nphases = 0, nitems = 0, nchunks = 0, ntiles = 0, hist_cap = 64;
  int blocks = 0, max_blocks = 0;  // CTAs of the persistent launch; all that fit at once
  long long cells = 0;
  // the per-solve work captured once as a CUDA graph and replayed
  bool graph_tried = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  std::vector<void*> allocs;
  size_t bytes = 0;
  std::string err;
  long long bar_cycles = kBarrierCycles;  // limit of one grid-wide barrier wait
};

namespace {

thread_local std::string g_batch_err;

bool pow2(int n) { return n >= 2 && (n & (n - 1)) == 0; }

template <typename T>
T* balloc(mg_batch* b, size_t count) {
  void* p = nullptr;
  if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  b->allocs.push_back(p);
  b->bytes += count * sizeof(T);
  return static_cast<T*>(p);
}

void free_batch(mg_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (void* p : b->allocs) cudaFree(p);
  if (b->h_grids) cudaFreeHost(b->h_grids);
  if (b->h_hist) cudaFreeHost(b->h_hist);
  if (b->h_err) cudaFreeHost(b->h_err);
  delete b;
}

// The phase list: source, first residual, max_cycles outer iterations of
// (1 + inner_cycles V-cycles, outer step, stopping rule), mean removal.
void build_phases(mg_batch* b, std::vector<Phase>& phases, std::vector<Item>& items) {
  const int G = b->ngrids;
  auto add_chunk_phase = [&](int type) {
    Phase p{type, 0, (int)items.size(), 0, 0};
    for (int g = 0; g < G; ++g)
      for (int q = 0; q < b->host_grids[g].nchunk; ++q) items.push_back(Item{g, q, 0, 0});
    p.count = (int)items.size() - p.first;
    phases.push_back(p);
  };
  auto add_grid_phase = [&](int type, int cycle) {
    Phase p{type, 0, (int)items.size(), 0, cycle};
    for (int g = 0; g < G; ++g) items.push_back(Item{g, 0, 0, 0});
    p.count = G;
    phases.push_back(p);
  };
  int nmax = 0;
  for (const GridDev& g : b->host_grids) nmax = std::max(nmax, g.n);
  auto add_tile_phase = [&](int type, int n, int cycle) {
    Phase p{type, n, (int)items.size(), 0, cycle};
    // largest tiles first: grids in the order given, tiles of this level
    for (int g = 0; g < G; ++g) {
      if (b->host_grids[g].n < n) continue;
      const int cz = std::min(kCz, n), tx = n >= 64 ? 64 : 32;
      for (int z = 0; z < n / cz; ++z)
        for (int y = 0; y < n / 16; ++y)
          for (int x = 0; x < n / tx; ++x) items.push_back(Item{g, x, y, z});
    }
    p.count = (int)items.size() - p.first;
    if (p.count > 0) phases.push_back(p);
  };
  auto add_fx_phase = [&](int zero_in) {
    Phase p{PH_FXSTEP, 0, (int)items.size(), 0, zero_in};
    for (int g = 0; g < G; ++g) {
      const int n = b->host_grids[g].n, tx = fx_tx(n), ty = fx_ty(n), cz = fx_cz(n);
      for (int z = 0; z < n / cz; ++z)
        for (int y = 0; y < n / ty; ++y)
          for (int x = 0; x < n / tx; ++x) items.push_back(Item{g, x, y, z});
    }
    p.count = (int)items.size() - p.first;
    phases.push_back(p);
  };
  add_chunk_phase(PH_SRC);
  add_grid_phase(PH_MEANFIN, 0);
  add_chunk_phase(PH_R0);
  add_grid_phase(PH_R0FIN, 0);
  // one V-cycle from a zero correction, then inner_cycles more (as mg_solve;
  // first_cycles in all in the first outer iteration when given)
  for (int o = 0; o < b->opts.max_cycles; ++o) {
    const int inner =
        (o == 0 && b->opts.first_cycles > 0) ? b->opts.first_cycles : 1 + b->opts.inner_cycles;
    for (int k = 0; k < inner; ++k) {
      for (int n = nmax; n >= kFusedMinN; n >>= 1) add_tile_phase(PH_DOWN, n, k);
      add_grid_phase(PH_BOTTOM, k);
      for (int n = kFusedMinN; n <= nmax; n <<= 1) add_tile_phase(PH_UP, n, k);
    }
    if (o == 0) {
      add_chunk_phase(PH_EMAX);
      add_grid_phase(PH_SETFX, 0);
      add_chunk_phase(PH_TOFX);
    }
    add_fx_phase(o == 0 ? 1 : 0);  // the first step starts from PHI = 0
    add_grid_phase(PH_FIN, 0);
  }
  add_chunk_phase(PH_PSUM);
  add_grid_phase(PH_PMEAN, 0);
  add_chunk_phase(PH_PSUB);
}

// The device work of one solve, in stream order.
cudaError_t enqueue_solve(mg_batch* b, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(b->d_grids, b->h_grids, sizeof(GridDev) * b->ngrids,
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counters, 0, sizeof(unsigned) * b->nphases, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_bar, 0, sizeof(unsigned) * 2, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_active, 0, sizeof(int) * b->nphases, s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(b->d_ptime, 0, sizeof(unsigned long long) * (b->nphases + 1), s);
  Ctl c;
  c.phases = b->d_phases;
  c.items = b->d_items;
  c.grids = b->d_grids;
  c.part = b->d_part;
  c.part2 = b->d_part2;
  c.ipart = b->d_ipart;
  c.part3 = b->d_part3;
  c.hist = b->d_hist;
  c.counters = b->d_counters;
  c.bar_count = b->d_bar;
  c.bar_gen = b->d_bar + 1;
  c.err = b->d_err;
  c.active_left = b->d_active;
  c.ptime = b->d_ptime;
  c.nphases = b->nphases;
  c.ngrids = b->ngrids;
  c.hist_cap = b->hist_cap;
  c.omega = b->opts.omega;
  c.max_cycles = b->opts.max_cycles;
  c.inner_zero = b->opts.inner_fmg ? 0 : 1;
  c.stall_ratio = b->opts.stall_ratio;
  c.bar_cycles = b->bar_cycles;
  if (e == cudaSuccess) {
    void* args[] = {&c};
    e = cudaLaunchCooperativeKernel((const void*)k_batch, dim3(b->blocks), dim3(kThreads), args,
                                    kSmem, s);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->h_grids, b->d_grids, sizeof(GridDev) * b->ngrids,
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->h_hist, b->d_hist, sizeof(double) * b->ngrids * b->hist_cap,
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  return e;
}

}  // namespace

extern "C" {

mg_status mg_batch_create(int n, const int* dims, const double* dx, const mg_bc* bcs,
                          const double* fixed_values, const mg_opts* opts, mg_batch** out) {
  if (!out || n < 1 || !dims || !dx || !bcs) {
    g_batch_err = "mg_batch_create: invalid argument";
    return MG_ERR_ARG;
  }
  *out = nullptr;
  mg_opts o;
  if (opts) o = *opts;
  else mg_opts_init(&o);
  if (o.prec != MG_MIXED || o.pre != 1 || o.post != 1 || !o.mode_fmg || o.inner_fmg ||
      o.max_cycles < 1 || o.max_cycles > 64 || o.inner_cycles < 0 || o.inner_cycles > 16 ||
      o.first_cycles < 0 || o.first_cycles > 17 || o.coarse_literal) {
    g_batch_err = "mg_batch_create: the batched solve runs MG_MIXED, V(1,1), FMG mode, inner "
                  "V-cycles from a zero correction (inner_fmg = 0), 1..64 outer iterations "
                  "of at most 17 V-cycles, homogeneous coarse rules (coarse_literal = 0)";
    return MG_ERR_ARG;
  }
  for (int g = 0; g < n; ++g) {
    const int nx = dims[3 * g], ny = dims[3 * g + 1], nz = dims[3 * g + 2];
    if (!pow2(nx) || nx != ny || nx != nz || nx > 1024 || !(dx[g] > 0.0) ||
        (bcs[g] != MG_BC_PERIODIC && bcs[g] != MG_BC_FIXED && bcs[g] != MG_BC_ZEROGRAD)) {
      g_batch_err = "mg_batch_create: grids must be cubic powers of two 2..1024 with a "
                    "periodic, fixed or zero-gradient rule";
      return MG_ERR_ARG;
    }
  }
  mg_batch* b = new mg_batch;
  b->ngrids = n;
  b->opts = o;
  cudaGetDevice(&b->device);
  b->host_grids.resize(n);
  int chunk0 = 0, tile0 = 0;
  bool ok = true;
  for (int g = 0; g < n && ok; ++g) {
    GridDev& d = b->host_grids[g];
    std::memset(&d, 0, sizeof d);
    d.n = dims[3 * g];
    int L = 1;
    while ((d.n >> (L - 1)) > 1) ++L;
    d.L = L;
    d.bc = (int)bcs[g];
    d.h = dx[g];
    d.bcval = (bcs[g] == MG_BC_FIXED && fixed_values) ? fixed_values[g] : 0.0;
    const long long N = (long long)d.n * d.n * d.n;
    b->cells += N;
    d.f64 = balloc<double>(b, N);
    ok = ok && d.f64;
    for (int l = 0; l < L && ok; ++l) {
      const long long c = 1LL << (3 * l);
      d.u32[l] = balloc<float>(b, c);
      d.f32[l] = balloc<float>(b, c);
      ok = ok && d.u32[l] && d.f32[l];
      if ((1 << l) >= kFusedMinN) {
        d.u32b[l] = balloc<float>(b, c);
        ok = ok && d.u32b[l];
      }
    }
    d.chunk0 = chunk0;
    d.nchunk = (int)((N + kChunk - 1) / kChunk);
    chunk0 += d.nchunk;
    d.fx2 = balloc<long long>(b, N);
    ok = ok && d.fx2;
    d.part0 = tile0;
    d.ntile = (d.n / fx_tx(d.n)) * (d.n / fx_ty(d.n)) * (d.n / fx_cz(d.n));
    tile0 += d.ntile;
  }
  b->nchunks = chunk0;
  b->ntiles = tile0;
  std::vector<Phase> phases;
  std::vector<Item> items;
  if (ok) build_phases(b, phases, items);
  b->nphases = (int)phases.size();
  b->nitems = (int)items.size();
  if (ok) {
    b->d_grids = balloc<GridDev>(b, n);
    b->d_phases = balloc<Phase>(b, phases.size());
    b->d_items = balloc<Item>(b, items.size());
    b->d_part = balloc<double>(b, b->nchunks);
    b->d_part2 = balloc<double>(b, b->nchunks);
    b->d_ipart = balloc<long long>(b, 2 * (size_t)b->nchunks);
    b->d_part3 = balloc<double>(b, b->ntiles);
    b->d_hist = balloc<double>(b, (size_t)n * b->hist_cap);
    b->d_counters = balloc<unsigned>(b, b->nphases);
    b->d_bar = balloc<unsigned>(b, 2);
    b->d_err = balloc<int>(b, 1);
    b->d_active = balloc<int>(b, b->nphases);
    b->d_ptime = balloc<unsigned long long>(b, b->nphases + 1);
    ok = b->d_grids && b->d_phases && b->d_items && b->d_part && b->d_part2 && b->d_ipart &&
         b->d_part3 &&
         b->d_hist && b->d_counters &&
         b->d_bar && b->d_err && b->d_active && b->d_ptime;
    b->host_phases = phases;
  }
  if (ok) {
    ok = cudaMallocHost(&b->h_grids, sizeof(GridDev) * n) == cudaSuccess &&
         cudaMallocHost(&b->h_hist, sizeof(double) * n * b->hist_cap) == cudaSuccess &&
         cudaMallocHost(&b->h_err, sizeof(int) * 4) == cudaSuccess;
  }
  if (ok) {
    ok = cudaMemcpy(b->d_phases, phases.data(), sizeof(Phase) * phases.size(),
                    cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(b->d_items, items.data(), sizeof(Item) * items.size(),
                    cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem) ==
             cudaSuccess;
  }
  int per_sm = 0, sms = 0;
  if (ok) {
    ok = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, kThreads, kSmem) ==
             cudaSuccess &&
         cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device) == cudaSuccess &&
         per_sm > 0;
  }
  if (!ok) {
    cudaGetLastError();
    g_batch_err = "mg_batch_create: device allocation or set-up failed";
    free_batch(b);
    return MG_ERR_OOM;
  }
  b->blocks = b->max_blocks = per_sm * sms;
  *out = b;
  return MG_OK;
}

mg_status mg_batch_solve(mg_batch* b, const double* const* rho, const double* four_pi_G,
                         const double* tol, double* const* phi, double* hist, int hist_cap,
                         int* n_hist, mg_status* status, void* stream) {
  if (!b || !rho || !four_pi_G || !tol || !phi) {
    g_batch_err = "mg_batch_solve: invalid argument";
    return MG_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int used = 0;
  for (int g = 0; g < b->ngrids; ++g) {
    if (!rho[g]) continue;  // a slot without a grid this time
    ++used;
    if (!phi[g] || !(tol[g] >= 0.0)) {
      g_batch_err = "mg_batch_solve: invalid per-grid argument";
      return MG_ERR_ARG;
    }
  }
  if (used == 0) {
    g_batch_err = "mg_batch_solve: no grid to solve";
    return MG_ERR_ARG;
  }
  for (int g = 0; g < b->ngrids; ++g) {
    GridDev d = b->host_grids[g];
    d.rho = rho[g];
    d.phi = rho[g] ? phi[g] : nullptr;
    d.fpg = rho[g] ? four_pi_G[g] : 0.0;
    d.tol = rho[g] ? tol[g] : 0.0;
    d.mean = 0.0;
    d.fnorm = d.rn = 0.0;
    d.scale = 1.0;
    d.prev = -1.0;
    d.d0 = -1.0;
    d.stalls = 0;
    d.active = 1;
    d.status = MG_ERR_NOT_CONVERGED;
    d.nh = 0;
    d.cycles = 0;
    d.maxf = 0.0;
    d.two_S = 1.0;
    d.S = 0;
    d.imean = 0;
    d.b2 = 0;
    d.in_fx = 0;
    d.fxbad = 0;
    d.cur = 0;
    d.skip = rho[g] ? 0 : 1;
    if (d.skip) {
      d.active = 0;
      d.status = MG_OK;
    }
    b->h_grids[g] = d;
  }
  cudaError_t e = cudaSuccess;
  if (!b->graph_tried) {
    // Capture the whole solve (upload of the per-grid arguments, counter
    // resets, the persistent kernel, download of the results) once.
    b->graph_tried = true;
    cudaError_t ce = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
      const cudaError_t ee = enqueue_solve(b, b->cap);
      cudaGraph_t gph = nullptr;
      ce = cudaStreamEndCapture(b->cap, &gph);
      if (ee == cudaSuccess && ce == cudaSuccess && gph) {
        b->graph = gph;
        if (cudaGraphInstantiate(&b->exec, gph, 0) != cudaSuccess) b->exec = nullptr;
      } else if (gph) {
        cudaGraphDestroy(gph);
      }
    }
    cudaGetLastError();  // a failed capture leaves the direct launch path
  }
  ++g_launches;
  if (b->exec) e = cudaGraphLaunch(b->exec, s);
  else e = enqueue_solve(b, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    b->err = std::string("mg_batch_solve: ") + cudaGetErrorString(e);
    g_batch_err = b->err;
    return MG_ERR_CUDA;
  }
  if (*b->h_err) {
    b->err = "mg_batch_solve: a grid-wide barrier timed out";
    g_batch_err = b->err;
    return MG_ERR_TIMEOUT;
  }
  mg_status worst = MG_OK;
  for (int g = 0; g < b->ngrids; ++g) {
    const GridDev& d = b->h_grids[g];
    const int nh = std::min(d.nh, std::min(hist_cap, b->hist_cap));
    if (hist && hist_cap > 0)
      for (int q = 0; q < nh; ++q) hist[(size_t)g * hist_cap + q] = b->h_hist[(size_t)g * b->hist_cap + q];
    if (n_hist) n_hist[g] = nh;
    if (status) status[g] = (mg_status)d.status;
    if (d.status != MG_OK && worst == MG_OK) worst = (mg_status)d.status;
  }
  return worst;
}

mg_status mg_batch_destroy(mg_batch* b) {
  if (b) free_batch(b);
  return MG_OK;
}

long long mg_batch_cells(const mg_batch* b) { return b ? b->cells : 0; }

int mg_batch_graph(const mg_batch* b) { return b && b->exec ? 1 : 0; }

mg_status mg_batch_phase_ms(mg_batch* b, double* ms_by_type, int n_types) {
  if (!b || !ms_by_type || n_types < 1) return MG_ERR_ARG;
  std::vector<unsigned long long> t((size_t)b->nphases + 1);
  if (cudaMemcpy(t.data(), b->d_ptime, sizeof(unsigned long long) * t.size(),
                 cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return MG_ERR_CUDA;
  }
  for (int k = 0; k < n_types; ++k) ms_by_type[k] = 0.0;
  unsigned long long last = t[(size_t)b->nphases];
  for (int ph = 0; ph < b->nphases; ++ph) {
    if (!t[(size_t)ph] || !last) continue;  // skipped after every grid stopped
    const int ty = b->host_phases[(size_t)ph].type;
    if (ty < n_types) ms_by_type[ty] += (double)(t[(size_t)ph] - last) * 1e-6;
    last = t[(size_t)ph];
  }
  return MG_OK;
}

mg_status mg_batch_set_blocks(mg_batch* b, int blocks) {
  if (!b || blocks < 0) {
    g_batch_err = "mg_batch_set_blocks: invalid argument";
    return MG_ERR_ARG;
  }
  const int cap = b->max_blocks;
  b->blocks = blocks == 0 || blocks > cap ? cap : blocks;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->graph_tried = false;
  return MG_OK;
}

mg_status mg_batch_set_barrier_limit(mg_batch* b, long long cycles) {
  if (!b || cycles < 0) {
    g_batch_err = "mg_batch_set_barrier_limit: invalid argument";
    return MG_ERR_ARG;
  }
  b->bar_cycles = cycles;
  // the limit is a kernel argument: the captured solve is captured again
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->graph_tried = false;
  return MG_OK;
}

const char* mg_batch_last_error(const mg_batch* b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

}  // extern "C"
