// mg_fixed.cu -- exact 64-bit fixed-point outer residual of the mixed solve.
//
// The outer loop of the mixed-precision solve needs r = f - L_h phi to FP64
// accuracy.  On this GPU FP64 arithmetic (and every FP64 <-> integer / FP32
// conversion) runs at 1/58 of the FP32 rate, so an FP64 residual sweep is
// bound by the FP64 pipe, not by memory.  Here phi and h^2 f are held as
// 64-bit integers scaled by 2^S (S chosen per solve so that |phi| < 2^55):
//   R = F - (sum of the six neighbours of PHI - 6 PHI)
// is then exact integer arithmetic (no rounding at all, and 2^-55 max|phi|
// resolution against 2^-53 relative for doubles), and r = R 2^-S / h^2 is
// rounded once when it is converted for the FP32 inner solve.  The FP64 pipe
// is used once per cell per pass (the conversion), integer adds do the rest.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <type_traits>

#include "mg_convert.cuh"
#include "mg_device.cuh"
#include "mg_internal.h"

namespace mg {
namespace {

constexpr int kThreads = 256;

int grid_for(long long work) {
  long long b = (work + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  if (b > sm_count() * 64LL) b = sm_count() * 64LL;
  return (int)b;
}

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <bool MAX>
__device__ __forceinline__ double block_reduce(double v) {
  __shared__ double ws[kThreads / 32];
  v = MAX ? warp_max(v) : warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) ws[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = lane < kThreads / 32 ? ws[lane] : 0.0;
    r = MAX ? warp_max(r) : warp_sum(r);
  }
  __syncthreads();
  return r;
}

// max |a| in the array's own precision (no FP64 work for FP32 data)
// VEC (FP32, 16-byte aligned): four values per 16-byte load, four loads in
// flight per thread.
template <typename T, bool VEC = false>
__global__ void k_absmax(const T* __restrict__ a, long long n, double* __restrict__ partials) {
  T m = T(0);
  auto take = [&](T x) {
    const T v = x < T(0) ? -x : x;
    m = v > m ? v : m;
  };
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if constexpr (VEC) {
    const long long n4 = n >> 2;
    const float4* a4 = reinterpret_cast<const float4*>(a);
    for (; t + 3 * stride < n4; t += 4 * stride) {
      float4 v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = a4[t + k * stride];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        take(v[k].x);
        take(v[k].y);
        take(v[k].z);
        take(v[k].w);
      }
    }
    for (; t < n4; t += stride) {
      const float4 v = a4[t];
      take(v.x);
      take(v.y);
      take(v.z);
      take(v.w);
    }
    for (long long i = 4 * n4 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += stride)
      take(a[i]);
  } else {
    for (; t < n; t += stride) take(a[t]);
  }
  const double r = block_reduce<true>((double)m);
  if (threadIdx.x == 0) partials[blockIdx.x] = r;
}

__global__ void k_finish_max(const double* __restrict__ partials, int nb, double* out) {
  double m = 0.0;
  for (int t = threadIdx.x; t < nb; t += blockDim.x) m = fmax(m, partials[t]);
  m = block_reduce<true>(m);
  if (threadIdx.x == 0) out[0] = m;
}

// In place: the double a[t] becomes the integer round((a[t] - mu) * c).
__global__ void k_f64_to_fx(double* a, long long n, double mu, double c) {
  long long* q = reinterpret_cast<long long*>(a);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    q[t] = cvt::d2ll_rn((a[t] - mu) * c);
}

// out[t] = (q[t] - M) 2^-S as a double (out may alias q), M = *mean (the
// integers' rounded mean) when given, else 0.  Integer arithmetic only.
// out[i] = op(in[i]) over n 8-byte elements.  PAIRS: both arrays are 16-byte
// aligned, so a thread moves two elements per 16-byte load and store, with
// four such loads in flight before their results are stored (each element is
// read before it is written, so in == out is allowed).
template <bool PAIRS, typename Op>
__device__ __forceinline__ void stream8(const unsigned long long* in, unsigned long long* out,
                                        long long n, Op op) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if constexpr (!PAIRS) {
    for (; t < n; t += stride) out[t] = op(in[t]);
    return;
  }
  const long long n2 = n >> 1;
  const ulonglong2* in2 = reinterpret_cast<const ulonglong2*>(in);
  ulonglong2* out2 = reinterpret_cast<ulonglong2*>(out);
  for (; t + 3 * stride < n2; t += 4 * stride) {
    ulonglong2 v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = in2[t + k * stride];
#pragma unroll
    for (int k = 0; k < 4; ++k) out2[t + k * stride] = make_ulonglong2(op(v[k].x), op(v[k].y));
  }
  for (; t < n2; t += stride) {
    const ulonglong2 v = in2[t];
    out2[t] = make_ulonglong2(op(v.x), op(v.y));
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) out[n - 1] = op(in[n - 1]);
}

inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

template <bool PAIRS>
__global__ void k_fx_to_f64(const long long* q, double* out, long long n, int S,
                            const long long* __restrict__ mean) {
  const long long M = mean ? mean[0] : 0;
  stream8<PAIRS>(reinterpret_cast<const unsigned long long*>(q),
                 reinterpret_cast<unsigned long long*>(out), n, [&](unsigned long long v) {
                   return (unsigned long long)__double_as_longlong(
                       cvt::ll2d_pow2_rn((long long)v - M, S));
                 });
}

// |x| as an unsigned integer: for non-negative doubles (and floats) the order
// of the bit patterns is the order of the values, so maxima need no FP64 work.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
}

// Exact sum of a thread's doubles in integer arithmetic: A (two's-complement
// 128-bit, hi:lo) counts units of 2^B, with B = 60 below the binary exponent
// of the largest significand unit seen so far.  A double m 2^k (m < 2^53) adds
// m 2^(k - B) < 2^113, so a thread may add up to 2^14 values without
// overflow; bits below 2^B (2^-112 of the largest value, and values below
// 2^-1022) are dropped.  No FP64 arithmetic per value: that pipe, not memory,
// would bound the pass.
struct ExactSum {
  unsigned long long lo = 0;
  long long hi = 0;
  int B = -100000;  // no value yet
};

__device__ __forceinline__ void exact_add(ExactSum& a, double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned uh = (unsigned)(u >> 32), ul = (unsigned)u;
  const int e = (int)((uh >> 20) & 0x7ff);
  if (e == 0) return;
  const int k = e - 1075;  // x = +-m 2^k, m = mh 2^32 + ul
  if (k - a.B > 60) {  // a new largest exponent: A >>= d (arithmetic), B += d
    const int d = k - 60 - a.B;
    if (d >= 128) {
      a.lo = (unsigned long long)(a.hi >> 63);
      a.hi >>= 63;
    } else if (d >= 64) {
      a.lo = (unsigned long long)(a.hi >> (d - 64));
      a.hi >>= 63;
    } else {
      a.lo = (a.lo >> d) | ((unsigned long long)a.hi << (64 - d));
      a.hi >>= d;
    }
    a.B = k - 60;
  }
  const int sh = k - a.B;  // <= 60
  unsigned long long tlo, thi;
  if (sh >= 0) {
    // m << sh as four 32-bit words: shift by sh mod 32 with funnel shifts,
    // then up one word when sh >= 32 (m < 2^53, sh <= 60: 113 bits at most)
    const unsigned mh = (uh & 0xFFFFFu) | 0x100000u;
    const unsigned r = (unsigned)sh & 31u;
    const unsigned x0 = ul << r, x1 = __funnelshift_l(ul, mh, r), x2 = __funnelshift_l(mh, 0u, r);
    const bool up = sh >= 32;
    tlo = ((unsigned long long)(up ? x0 : x1) << 32) | (up ? 0u : x0);
    thi = ((unsigned long long)(up ? x2 : 0u) << 32) | (up ? x1 : x2);
  } else if (sh > -64) {
    const unsigned long long m = (u & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
    tlo = m >> -sh;
    thi = 0;
  } else {
    return;
  }
  // A -= T or A += T with the carry chained through the two words
  unsigned long long hi = (unsigned long long)a.hi;
  if (uh >> 31)
    asm("sub.cc.u64 %0, %0, %2;\n\tsubc.u64 %1, %1, %3;" : "+l"(a.lo), "+l"(hi) : "l"(tlo), "l"(thi));
  else
    asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(a.lo), "+l"(hi) : "l"(tlo), "l"(thi));
  a.hi = (long long)hi;
}

// The thread's sum as a double (rounded in the conversions of its two words).
__device__ __forceinline__ double exact_value(const ExactSum& a) {
  if (a.B == -100000) return 0.0;
  return ldexp(fma((double)a.hi, 18446744073709551616.0, __ull2double_rn(a.lo)), a.B);
}

// Per-block partial sums of rho (sum[]) and maxima of |rho| (mx[], as the
// double whose bits are the largest |rho| pattern); two cells per step.
// With `copy`, rho is read from host memory and each value is also stored
// into copy (the device array the later passes read).
__global__ void k_rho_stats(const double2* __restrict__ rho, long long n2,
                            double* __restrict__ sum, double* __restrict__ mx,
                            double2* __restrict__ copy) {
  ExactSum acc;
  unsigned long long m = 0;
  auto take = [&](const double2 r) {
    exact_add(acc, r.x);
    exact_add(acc, r.y);
    const unsigned long long a = abs_bits(r.x), b = abs_bits(r.y);
    m = a > m ? a : m;
    m = b > m ? b : m;
  };
  // four loads in flight before the (branchy) exact adds use them; the same
  // order of values per thread as one at a time
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; t + 3 * stride < n2; t += 4 * stride) {
    double2 r[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) r[k] = rho[t + k * stride];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (copy) copy[t + k * stride] = r[k];
      take(r[k]);
    }
  }
  for (; t < n2; t += stride) {
    const double2 r = rho[t];
    if (copy) copy[t] = r;
    take(r);
  }
  const double bs = block_reduce<false>(exact_value(acc));
  const double bm = block_reduce<true>(__longlong_as_double((long long)m));
  if (threadIdx.x == 0) {
    sum[blockIdx.x] = bs;
    mx[blockIdx.x] = bm;
  }
}

// r32 = a rho - b in FP32 arithmetic (a = 4 pi G scale, b = mean scale, so
// |a rho|, |b| <= 1 + |b| and the error is a few FP32 ulps of 1: this is only
// the right-hand side of the first FP32 inner solve, whose exact residual the
// fixed-point step recomputes); per-block partial sums of r32^2 (FP32 per
// thread) and maxima of |r32|.  No FP64 arithmetic: rho reaches FP32 by the
// integer conversion.
// From the device: a and b (as doubles holding FP32 values) in ab[0], ab[1]
// when ab is given, else the arguments.
__global__ void k_rho_to_r32(const double2* __restrict__ rho, float2* __restrict__ r32,
                             long long n2, float a_arg, float b_arg, const double* __restrict__ ab,
                             double* __restrict__ sum, double* __restrict__ mx) {
  const float a = ab ? (float)ab[0] : a_arg, b = ab ? (float)ab[1] : b_arg;
  float acc = 0.f, m = 0.f;
#pragma unroll 4
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n2;
       t += (long long)gridDim.x * blockDim.x) {
    const double2 r = rho[t];
    const float x = fmaf(a, cvt::d2f_rn(r.x), -b), y = fmaf(a, cvt::d2f_rn(r.y), -b);
    r32[t] = make_float2(x, y);
    acc = fmaf(x, x, fmaf(y, y, acc));
    m = fmaxf(m, fmaxf(fabsf(x), fabsf(y)));
  }
  const double bs = block_reduce<false>((double)acc);
  const double bm = block_reduce<true>((double)m);
  if (threadIdx.x == 0) {
    sum[blockIdx.x] = bs;
    mx[blockIdx.x] = bm;
  }
}

// In place into the integer array q: round(a rho - b) (the fixed-point h^2 f).
template <bool PAIRS>
__global__ void k_rho_to_fx(const double* __restrict__ rho, long long* __restrict__ q, long long n,
                            double a, double b) {
  stream8<PAIRS>(reinterpret_cast<const unsigned long long*>(rho),
                 reinterpret_cast<unsigned long long*>(q), n, [&](unsigned long long v) {
                   return (unsigned long long)cvt::d2ll_rn(fma(a, __longlong_as_double(v), -b));
                 });
}

__global__ void k_finish_sum_max(const double* __restrict__ sum, const double* __restrict__ mx,
                                 int nb, double* __restrict__ out) {
  double a = 0.0, m = 0.0;
  for (int t = threadIdx.x; t < nb; t += blockDim.x) {
    a += sum[t];
    m = fmax(m, mx[t]);
  }
  a = block_reduce<false>(a);
  m = block_reduce<true>(m);
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = m;
  }
}

// PHI += round(e * c) (the FP32 correction on the fixed-point grid); flags a
// value above 2^60, past which neighbour sums could overflow.
__global__ void k_fx_correct(long long* __restrict__ phi, const float* __restrict__ e, long long n,
                             float c, int* __restrict__ flag) {
  bool bad = false;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const long long v = phi[t] + __float2ll_rn(e[t] * c);
    phi[t] = v;
    bad |= (v > (1LL << 60)) || (v < -(1LL << 60));
  }
  if (bad) atomicOr(flag, 1);
}

// The rule on the integer grid.  A MIXED rule (kinds per face in fk, as in
// Bc) takes its fixed faces' values from the face array like OPEN, or 0
// where there is none (the homogeneous rule).
struct FxBc {
  int kind;
  int fk;                // MIXED: bits 2q..2q+1 the kind of face q
  long long b2;          // FIXED: round(2 b 2^S)
  const double* faces;   // OPEN / MIXED: boundary values (doubles), scaled by c2 = 2^(S+1)
  double c2;
};

__device__ __forceinline__ int fx_face_kind(const FxBc& bc, int face) {
  return bc.kind == BC_MIXED ? (bc.fk >> (2 * face)) & 3 : bc.kind;
}

// One outer step on the integer grid, fused and z-marching:
//   PHI' = PHI_in + round(e * c)          (the pending FP32 correction, never
//                                           null; ZERO_IN: PHI_in is all zero)
//   R    = F - (sum_nb PHI' - 6 PHI')      (exact)
//   r32  = R * factor, partial sums of r32^2 (and of PHI' when psum is given),
//   PHI_out = PHI' (a different buffer: neighbouring tiles read PHI_in as
//   their halo and correct it themselves).
// A 32 x 16 tile of columns marches up a chunk of planes.  Each thread keeps
// PHI' of its own column at planes z-1, z, z+1 in registers (the z
// neighbours); the x / y neighbours come from the current plane in shared
// memory (double-buffered, one barrier per plane), whose 100 halo cells the
// first 100 threads load and correct.
constexpr int FX_TX = 32, FX_TY = 16, FX_W = FX_TX + 2, FX_H = FX_TY + 2;
constexpr int FX_HALO = 2 * FX_W + 2 * FX_TY;  // 100

// The ghost across face (axis, hi) of a non-periodic axis.
__device__ __forceinline__ long long fx_face_ghost(const FxBc& bc, const Grid& g, long long self,
                                                   int i, int j, int k, int axis, int hi) {
  if (fx_face_kind(bc, 2 * axis + hi) == BC_ZEROGRAD) return self;
  long long b2 = bc.b2;
  if (bc.kind == BC_MIXED && !bc.faces) b2 = 0;
  if ((bc.kind == BC_OPEN || bc.kind == BC_MIXED) && bc.faces) {
    size_t off;
    const size_t fx = (size_t)(g.ny + 2) * (g.nz + 2), fy = (size_t)(g.nx + 2) * (g.nz + 2),
                 fz = (size_t)(g.nx + 2) * (g.ny + 2);
    if (axis == 0) off = hi * fx + (size_t)(k + 1) * (g.ny + 2) + (j + 1);
    else if (axis == 1) off = 2 * fx + hi * fy + (size_t)(k + 1) * (g.nx + 2) + (i + 1);
    else off = 2 * fx + 2 * fy + hi * fz + (size_t)(j + 1) * (g.nx + 2) + (i + 1);
    b2 = __double2ll_rn(bc.faces[off] * bc.c2);
  }
  return b2 - self;
}

// Integer neighbour along `axis` (side hi) of cell (i, j, k) holding `self`:
// the stored value inside the grid, else the rule's ghost.
__device__ __forceinline__ long long fx_nb_lite(const long long* __restrict__ q, const FxBc& bc,
                                                const Grid& g, long long self, bool inside,
                                                long long o, int i, int j, int k, int axis,
                                                int hi) {
  if (inside) return q[o];
  if (fx_face_kind(bc, 2 * axis + hi) == BC_PERIODIC) {
    const long long sy = g.nx, sz = (long long)g.nx * g.ny;
    const long long t = ((long long)k * g.ny + j) * g.nx + i;
    if (axis == 0) return q[hi ? t - (g.nx - 1) : t + (g.nx - 1)];
    if (axis == 1) return q[hi ? t - (long long)(g.ny - 1) * sy : t + (long long)(g.ny - 1) * sy];
    return q[hi ? t - (long long)(g.nz - 1) * sz : t + (long long)(g.nz - 1) * sz];
  }
  return fx_face_ghost(bc, g, self, i, j, k, axis, hi);
}

// Asynchronous global -> shared copies of 8 or 4 bytes (src_bytes 0 fills
// zeros), and the wait for all but the newest N groups.
__device__ __forceinline__ void cp_async8(void* dst, const void* src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Per-thread staging ring of the fixed-point step: for each of FX_RING planes,
// this thread's own PHI_in, e and F, and its halo cell's PHI_in and e.  Each
// thread reads back only what it copied itself, so the ring needs no barrier.
constexpr int FX_RING = 4;
constexpr int FX_NT = FX_TX * FX_TY;
struct FxRing {
  long long p[FX_RING][FX_NT];
  long long f[FX_RING][FX_NT];
  float e[FX_RING][FX_NT];
  long long hp[FX_RING][128];
  float he[FX_RING][128];
};
constexpr size_t kFxSmem = sizeof(FxRing);

// CTAs per SM the step's registers are sized for: three (at most 40
// registers), except for the masks whose ghosts need more (0: no periodic
// axis, 1: only x, 2: only y), which spilled at 40 and run 11 % faster at two
// CTAs per SM without spills (256 x 256 x 512 box).
template <int PM>
constexpr int fx_min_blocks() {
  return (PM == 0 || PM == 1 || PM == 2) ? 2 : 3;
}

// PM: the periodic axes (bit 0 x, 1 y, 2 z).
template <int PM, bool ZERO_IN>
__global__ void __launch_bounds__(FX_TX* FX_TY, fx_min_blocks<PM>())
    k_fx_step(const long long* __restrict__ phi_in, long long* __restrict__ phi_out,
              const float* __restrict__ e, float c, const long long* __restrict__ F,
              float* __restrict__ r32, Grid g, FxBc bc, float factor, int cz,
              double* __restrict__ partials, long long* __restrict__ psum,
              int* __restrict__ flag) {
  __shared__ long long P[2][FX_H][FX_W];
  extern __shared__ long long fx_dyn[];
  FxRing& ring = *reinterpret_cast<FxRing*>(fx_dyn);
  const int tid = threadIdx.x;
  const int tx = tid % FX_TX, ty = tid / FX_TX;
  const int x0 = blockIdx.x * FX_TX, y0 = blockIdx.y * FX_TY, z0 = blockIdx.z * cz;
  const int z1 = min(z0 + cz, g.nz);
  const int i = x0 + tx, j = y0 + ty;  // this thread's column
  const unsigned plane = (unsigned)g.nx * (unsigned)g.ny;  // 32-bit offsets (fx_step_ok)
  const unsigned col = (unsigned)j * g.nx + i;
  // the halo cell this thread loads (threads < FX_HALO): rows -1 and 16 over
  // the full width, columns -1 and 32 over the tile's rows
  int ha = 0, hb = 0;
  const bool halo = tid < FX_HALO;
  if (halo) {
    const int h = tid;
    if (h < FX_W) { ha = h; hb = 0; }
    else if (h < 2 * FX_W) { ha = h - FX_W; hb = FX_H - 1; }
    else if (h < 2 * FX_W + FX_TY) { ha = 0; hb = h - 2 * FX_W + 1; }
    else { ha = FX_W - 1; hb = h - 2 * FX_W - FX_TY + 1; }
  }
  constexpr bool PX = (PM & 1) != 0, PY = (PM & 2) != 0, PZ = (PM & 4) != 0;
  int hx = x0 - 1 + ha, hy = y0 - 1 + hb;
  bool h_in = halo;
  if (PX) hx = hx < 0 ? hx + g.nx : (hx >= g.nx ? hx - g.nx : hx);
  else h_in = h_in && hx >= 0 && hx < g.nx;
  if (PY) hy = hy < 0 ? hy + g.ny : (hy >= g.ny ? hy - g.ny : hy);
  else h_in = h_in && hy >= 0 && hy < g.ny;
  const unsigned hcol = h_in ? (unsigned)hy * g.nx + hx : 0u;
  // Ring slot of plane q is (q - z0 + 1) mod 4; the z-march below is unrolled
  // by four, so every slot (and the plane buffer of P) is a compile-time
  // constant.
  auto issue = [&](auto SLc, int q) {
    constexpr int sl = decltype(SLc)::value;
    if (q <= z1) {
      const bool in = PZ || (q >= 0 && q < g.nz);
      const int qw = PZ ? (q < 0 ? q + g.nz : (q >= g.nz ? q - g.nz : q)) : (in ? q : 0);
      const unsigned o = (unsigned)qw * plane + col;
      if (!ZERO_IN) cp_async8(&ring.p[sl][tid], phi_in + o, in ? 8 : 0);
      cp_async4(&ring.e[sl][tid], e + o, in ? 4 : 0);
      if (q >= z0 && q < z1) {
        cp_async8(&ring.f[sl][tid], F + ((unsigned)q * plane + col), 8);
        if (halo) {
          const unsigned ho = (unsigned)q * plane + hcol;
          if (!ZERO_IN) cp_async8(&ring.hp[sl][tid], phi_in + ho, h_in ? 8 : 0);
          cp_async4(&ring.he[sl][tid], e + ho, h_in ? 4 : 0);
        }
      }
    }
    cp_commit();
  };
  // PHI' of this column in slot SL.  The correction's rounding to an integer
  // is done in integer arithmetic (exact, as the hardware's): with it and the
  // residual's conversion both on the FP64 pipe, that pipe bounds the step,
  // and with both in integer arithmetic, the issue rate does.
  auto own_at = [&](auto SLc) -> long long {
    constexpr int sl = decltype(SLc)::value;
    const long long v = ZERO_IN ? 0 : ring.p[sl][tid];
    return v + cvt::f2ll_rn(ring.e[sl][tid] * c);
  };
  using I0 = std::integral_constant<int, 0>;
  using I1 = std::integral_constant<int, 1>;
  using I2 = std::integral_constant<int, 2>;
  issue(I0{}, z0 - 1);
  issue(I1{}, z0);
  issue(I2{}, z0 + 1);
  cp_wait<1>();  // planes z0 - 1 and z0 have landed
  long long zm = own_at(I0{}), self = own_at(I1{});
  float acc = 0.f;
  // exact sum of this column's PHI' (|PHI'| <= 2^60 and at most 128 planes per
  // CTA, so no overflow); split into hi 2^32 + lo for the block sums
  long long csum = 0;
  bool bad = false;
  // plane z = z0 + J (mod 4): its slot is J + 1, z + 1's is J + 2, z + 2's J + 3
  auto step = [&](auto Jc, int z) {
    constexpr int J = decltype(Jc)::value;
    issue(std::integral_constant<int, (J + 3) & 3>{}, z + 2);
    cp_wait<1>();  // every plane up to z + 1 has landed
    constexpr int sl = (J + 1) & 3, buf = J & 1;
    const unsigned o = (unsigned)z * plane + col;
    const long long Fo = ring.f[sl][tid];
    const long long zp = own_at(std::integral_constant<int, (J + 2) & 3>{});
    P[buf][ty + 1][tx + 1] = self;
    if (halo) {
      const long long hv = (ZERO_IN ? 0 : ring.hp[sl][tid]) + __float2ll_rn(ring.he[sl][tid] * c);
      P[buf][hb][ha] = h_in ? hv : 0;
    }
    phi_out[o] = self;
    csum += self;
    bad |= (unsigned long long)(self + (1LL << 60)) > (2ULL << 60);  // |PHI'| > 2^60
    __syncthreads();
    long long xm = P[buf][ty + 1][tx], xp = P[buf][ty + 1][tx + 2];
    long long ym = P[buf][ty][tx + 1], yp = P[buf][ty + 2][tx + 1];
    long long zmv = zm, zpv = zp;
    if (!PX) {
      if (i == 0) xm = fx_face_ghost(bc, g, self, i, j, z, 0, 0);
      if (i == g.nx - 1) xp = fx_face_ghost(bc, g, self, i, j, z, 0, 1);
    }
    if (!PY) {
      if (j == 0) ym = fx_face_ghost(bc, g, self, i, j, z, 1, 0);
      if (j == g.ny - 1) yp = fx_face_ghost(bc, g, self, i, j, z, 1, 1);
    }
    if (!PZ) {
      if (z == 0) zmv = fx_face_ghost(bc, g, self, i, j, z, 2, 0);
      if (z == g.nz - 1) zpv = fx_face_ghost(bc, g, self, i, j, z, 2, 1);
    }
    const long long R = Fo - (((xm + xp) + (ym + yp)) + (zmv + zpv) - 6 * self);
    const float r = __ll2float_rn(R) * factor;
    r32[o] = r;
    acc = fmaf(r, r, acc);
    zm = self;
    self = zp;
    // the next plane writes the other half of P; this one is rewritten two
    // planes on, after every thread has passed the next barrier
  };
  for (int z = z0; z < z1; z += 4) {
    step(I0{}, z);
    if (z + 1 >= z1) break;
    step(I1{}, z + 1);
    if (z + 2 >= z1) break;
    step(I2{}, z + 2);
    if (z + 3 >= z1) break;
    step(std::integral_constant<int, 3>{}, z + 3);
  }
  cp_wait<0>();
  if (bad) atomicOr(flag, 1);
  // deterministic block sums, then one partial per block (blocks in launch
  // order); the sums of PHI' stay exact integers, so their total does not
  // depend on the blocking
  __shared__ double ws[FX_TX * FX_TY / 32];
  __shared__ long long wh[FX_TX * FX_TY / 32], wl[FX_TX * FX_TY / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const double v = warp_sum((double)acc);
  long long sum_hi = csum >> 32, sum_lo = csum & 0xffffffffLL;
  if (psum) {
    for (int o = 16; o > 0; o >>= 1) {
      sum_hi += __shfl_down_sync(0xffffffffu, sum_hi, o);
      sum_lo += __shfl_down_sync(0xffffffffu, sum_lo, o);
    }
  }
  if (lane == 0) {
    ws[w] = v;
    wh[w] = sum_hi;
    wl[w] = sum_lo;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    long long th = 0, tl = 0;
    for (int q = 0; q < FX_TX * FX_TY / 32; ++q) {
      t += ws[q];
      th += wh[q];
      tl += wl[q];
    }
    const size_t b = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    partials[b] = t;
    if (psum) {
      psum[2 * b] = th;
      psum[2 * b + 1] = tl;
    }
  }
}

// out[0] = the total of the (hi, lo) pairs as a double, summed exactly.
// The integers' sum from the per-block (hi, lo) partials (value = hi 2^32 +
// lo) and their mean rounded to an integer, exactly: N = 2^log2n cells, so the
// mean is the 128-bit sum shifted right with rounding (ties up).  out[0]: the
// sum as a double; out[1]: the mean's bits as a long long.
__global__ void k_finish_fx_sum(const long long* __restrict__ psum, int nb, int log2n,
                                double* __restrict__ out) {
  __shared__ long long sh[kThreads], sl[kThreads];
  long long h = 0, l = 0;
  for (int t = threadIdx.x; t < nb; t += blockDim.x) {
    h += psum[2 * t];
    l += psum[2 * t + 1];
  }
  sh[threadIdx.x] = h;
  sl[threadIdx.x] = l;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)blockDim.x; ++q) {
      h += sh[q];
      l += sl[q];
    }
    out[0] = (double)h * 4294967296.0 + (double)l;
    // 128-bit sum: h 2^32 + l
    const long long shi = h >> 32;
    const unsigned long long t = (unsigned long long)h << 32;
    unsigned long long slo = t + (unsigned long long)l;
    long long sh2 = shi + (l < 0 ? -1 : 0) + (slo < t ? 1 : 0);
    // + 2^(log2n - 1), then an arithmetic shift right by log2n (0 <= log2n < 64)
    long long mean = 0;
    if (log2n == 0) {
      mean = (long long)slo;
    } else {
      const unsigned long long half = 1ULL << (log2n - 1);
      const unsigned long long lo2 = slo + half;
      sh2 += lo2 < slo ? 1 : 0;
      mean = (long long)((lo2 >> log2n) | ((unsigned long long)sh2 << (64 - log2n)));
    }
    reinterpret_cast<long long*>(out)[1] = mean;
  }
}

// The last conversion of the fixed-point outer loop with the acceleration
// (Sec. 3.2.3) fused in: phi = PHI 2^-S - m and, per axis, the average of the
// two face accelerations, which on the integer grid is the exact difference
// -(PHI_{i+1} - PHI_{i-1}) rounded once and scaled by 2^-S / (2 h).
// Writes phi (as doubles, into a different buffer than q) and g = [gx|gy|gz].
__global__ void k_fx_finish_gravity(const long long* __restrict__ q, double* __restrict__ phi,
                                    double* __restrict__ g, Grid gr, FxBc bc, int S,
                                    double cg, const long long* __restrict__ mean) {
  const long long M = mean ? mean[0] : 0;
  const long long N = gr.cells();
  const dev::Split sp(gr.nx, gr.ny);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N;
       t += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    sp(t, i, j, k);
    const long long self = q[t];
    phi[t] = cvt::ll2d_pow2_rn(self - M, S);
    const long long sy = gr.nx, sz = (long long)gr.nx * gr.ny;
    const long long xm = fx_nb_lite(q, bc, gr, self, i > 0, t - 1, i, j, k, 0, 0);
    const long long xp = fx_nb_lite(q, bc, gr, self, i < gr.nx - 1, t + 1, i, j, k, 0, 1);
    const long long ym = fx_nb_lite(q, bc, gr, self, j > 0, t - sy, i, j, k, 1, 0);
    const long long yp = fx_nb_lite(q, bc, gr, self, j < gr.ny - 1, t + sy, i, j, k, 1, 1);
    const long long zm = fx_nb_lite(q, bc, gr, self, k > 0, t - sz, i, j, k, 2, 0);
    const long long zp = fx_nb_lite(q, bc, gr, self, k < gr.nz - 1, t + sz, i, j, k, 2, 1);
    g[t] = -cvt::ll2d_rn(xp - xm) * cg;
    g[N + t] = -cvt::ll2d_rn(yp - ym) * cg;
    g[2 * N + t] = -cvt::ll2d_rn(zp - zm) * cg;
  }
}

}  // namespace

template <typename T>
cudaError_t launch_absmax(const T* a, long long n, double* partials, double* out, cudaStream_t s) {
  const int nb = reduce_blocks(n);
  ++g_launches;
  if (sizeof(T) == 4 && aligned16(a))
    k_absmax<T, sizeof(T) == 4><<<nb, kThreads, 0, s>>>(a, n, partials);
  else
    k_absmax<T><<<nb, kThreads, 0, s>>>(a, n, partials);
  ++g_launches;
  k_finish_max<<<1, kThreads, 0, s>>>(partials, nb, out);
  return cudaGetLastError();
}
template cudaError_t launch_absmax<double>(const double*, long long, double*, double*, cudaStream_t);
template cudaError_t launch_absmax<float>(const float*, long long, double*, double*, cudaStream_t);

cudaError_t launch_f64_to_fx(double* a, long long n, double mu, double c, cudaStream_t s) {
  ++g_launches;
  k_f64_to_fx<<<grid_for(n), kThreads, 0, s>>>(a, n, mu, c);
  return cudaGetLastError();
}

cudaError_t launch_fx_to_f64(const long long* q, double* out, long long n, int S,
                             const long long* mean, cudaStream_t s) {
  ++g_launches;
  if (aligned16(q) && aligned16(out))
    k_fx_to_f64<true><<<grid_for(n / 8), kThreads, 0, s>>>(q, out, n, S, mean);
  else
    k_fx_to_f64<false><<<grid_for(n), kThreads, 0, s>>>(q, out, n, S, mean);
  return cudaGetLastError();
}

template <int KIND>
__global__ void k_convert(const void* __restrict__ in, void* __restrict__ out, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    if (KIND == 0) static_cast<long long*>(out)[t] = cvt::d2ll_rn(static_cast<const double*>(in)[t]);
    if (KIND == 1) static_cast<double*>(out)[t] = cvt::ll2d_rn(static_cast<const long long*>(in)[t]);
    if (KIND == 2) static_cast<float*>(out)[t] = cvt::d2f_rn(static_cast<const double*>(in)[t]);
    if (KIND == 3) static_cast<long long*>(out)[t] = cvt::f2ll_rn(static_cast<const float*>(in)[t]);
    if (KIND == 4) static_cast<float*>(out)[t] = cvt::ll2f_rn(static_cast<const long long*>(in)[t]);
  }
}

cudaError_t launch_convert(int kind, long long n, const void* in, void* out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  ++g_launches;
  switch (kind) {
    case 0: k_convert<0><<<grid_for(n), kThreads, 0, s>>>(in, out, n); break;
    case 1: k_convert<1><<<grid_for(n), kThreads, 0, s>>>(in, out, n); break;
    case 2: k_convert<2><<<grid_for(n), kThreads, 0, s>>>(in, out, n); break;
    case 3: k_convert<3><<<grid_for(n), kThreads, 0, s>>>(in, out, n); break;
    case 4: k_convert<4><<<grid_for(n), kThreads, 0, s>>>(in, out, n); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_rho_stats(const double* rho, long long n, double* partials, double* out,
                             cudaStream_t s) {
  if (n % 2) return cudaErrorInvalidValue;
  const int nb = reduce_blocks(n / 2);
  // at most 2^14 values per thread in the exact sums (2^32 cells, 34 GB of rho)
  if (n > (long long)nb * kThreads * 16384) return cudaErrorInvalidValue;
  ++g_launches;
  k_rho_stats<<<nb, kThreads, 0, s>>>(reinterpret_cast<const double2*>(rho), n / 2, partials,
                                      partials + nb, nullptr);
  ++g_launches;
  k_finish_sum_max<<<1, kThreads, 0, s>>>(partials, partials + nb, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_rho_stats_copy(const double* host_rho, double* dev, long long n,
                                  double* partials, double* out, cudaStream_t s) {
  if (n % 2) return cudaErrorInvalidValue;
  const int nb = reduce_blocks(n / 2);
  if (n > (long long)nb * kThreads * 16384) return cudaErrorInvalidValue;
  ++g_launches;
  k_rho_stats<<<nb, kThreads, 0, s>>>(reinterpret_cast<const double2*>(host_rho), n / 2, partials,
                                      partials + nb, reinterpret_cast<double2*>(dev));
  ++g_launches;
  k_finish_sum_max<<<1, kThreads, 0, s>>>(partials, partials + nb, nb, out);
  return cudaGetLastError();
}

// The source's scale on the device, from the sums of launch_rho_stats in
// st[0] (sum rho) and st[1] (max |rho|): out[0] = mu (the mean of f, or 0),
// out[1] = scale = 1 / (|4 pi G| max|rho| + |mu|), out[2], out[3] = the FP32
// a = 4 pi G scale and b = mu scale of launch_rho_to_r32 -- each one IEEE
// operation in the order the host would take them.
__global__ void k_source_scale(const double* __restrict__ st, long long n, double four_pi_G,
                               int has_mean, double* __restrict__ out) {
  const double mu = has_mean ? __dmul_rn(four_pi_G, __ddiv_rn(st[0], (double)n)) : 0.0;
  const double bound = __dadd_rn(__dmul_rn(fabs(four_pi_G), st[1]), fabs(mu));
  const double scale = bound > 0.0 ? __ddiv_rn(1.0, bound) : 1.0;
  out[0] = mu;
  out[1] = scale;
  out[2] = (double)__double2float_rn(__dmul_rn(four_pi_G, scale));
  out[3] = (double)__double2float_rn(__dmul_rn(mu, scale));
}

cudaError_t launch_source_scale(const double* st, long long n, double four_pi_G, bool has_mean,
                                double* out, cudaStream_t s) {
  ++g_launches;
  k_source_scale<<<1, 1, 0, s>>>(st, n, four_pi_G, has_mean ? 1 : 0, out);
  return cudaGetLastError();
}

cudaError_t launch_rho_to_r32(const double* rho, float* r32, long long n, double a, double b,
                              double* partials, double* out, cudaStream_t s,
                              const double* ab_dev) {
  if (n % 2) return cudaErrorInvalidValue;
  const int nb = reduce_blocks(n / 2);
  ++g_launches;
  k_rho_to_r32<<<nb, kThreads, 0, s>>>(reinterpret_cast<const double2*>(rho),
                                       reinterpret_cast<float2*>(r32), n / 2, (float)a, (float)b,
                                       ab_dev, partials, partials + nb);
  ++g_launches;
  k_finish_sum_max<<<1, kThreads, 0, s>>>(partials, partials + nb, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_rho_to_fx(const double* rho, long long* q, long long n, double a, double b,
                             cudaStream_t s) {
  ++g_launches;
  if (aligned16(rho) && aligned16(q))
    k_rho_to_fx<true><<<grid_for(n / 8), kThreads, 0, s>>>(rho, q, n, a, b);
  else
    k_rho_to_fx<false><<<grid_for(n), kThreads, 0, s>>>(rho, q, n, a, b);
  return cudaGetLastError();
}

cudaError_t launch_fx_correct(long long* phi, const float* e, long long n, float c, int* flag,
                              cudaStream_t s) {
  ++g_launches;
  k_fx_correct<<<grid_for(n), kThreads, 0, s>>>(phi, e, n, c, flag);
  return cudaGetLastError();
}

// 32-bit element offsets: fewer than 2^32 cells
bool fx_step_ok(Grid g) {
  return g.nx % FX_TX == 0 && g.ny % FX_TY == 0 && g.cells() < (1LL << 32);
}

// Planes per CTA: the given cz, else the largest of 64 .. 4 that still
// gives four CTAs per SM; at most 128 (a thread's exact sum of its column's
// integers, each below 2^55, must stay below 2^63).
int fx_step_cz(Grid g, int cz) {
  const long long cols = (long long)(g.nx / FX_TX) * (g.ny / FX_TY);
  if (cz <= 0) {
    cz = 64;
    while (cz > kFxMinCz && cols * ((g.nz + cz - 1) / cz) < 4LL * sm_count()) cz /= 2;
  }
  if (cz > 128) cz = 128;
  return cz > g.nz ? g.nz : cz;
}

// Blocks of a launch with `cz` planes per CTA; cz = 0: the most any allowed
// cz (>= kFxMinCz) gives, to size the partial sums.
int fx_step_blocks(Grid g, int cz) {
  const long long cols = (long long)(g.nx / FX_TX) * (g.ny / FX_TY);
  const int z = cz > 0 ? fx_step_cz(g, cz) : (g.nz < kFxMinCz ? g.nz : kFxMinCz);
  return (int)(cols * ((g.nz + z - 1) / z));
}

namespace {

FxBc fx_bc(const Bc& bc, double two_pow_S) {
  FxBc b;
  b.kind = bc.kind;
  b.fk = bc.fk;
  b.c2 = 2.0 * two_pow_S;
  b.b2 = bc.kind == BC_FIXED ? (long long)std::llrint(bc.value * b.c2) : 0;
  b.faces = bc.faces;
  return b;
}

int fx_periodic_mask(const Bc& bc) {
  int m = 0;
  for (int a = 0; a < 3; ++a)
    if (face_kind(bc, 2 * a) == BC_PERIODIC) m |= 1 << a;
  return m;
}

}  // namespace

cudaError_t launch_fx_step(const long long* phi_in, long long* phi_out, const float* e, float c,
                           const long long* F, float* r32, Grid g, const Bc& bc, double two_pow_S,
                           float factor, double* partials, int nb_max, int* flag, int* nb_out,
                           cudaStream_t s, int cz_req, long long* psum) {
  // The ghost 2 b - phi on the fixed-point grid: 2 b 2^S rounded once.
  const FxBc b = fx_bc(bc, two_pow_S);
  const int pm = fx_periodic_mask(bc);
  if (cz_req != 0 && cz_req < kFxMinCz) return cudaErrorInvalidValue;
  if (!e || !F || !phi_out || !r32 || !partials || !flag) return cudaErrorInvalidValue;
  const int cz = fx_step_cz(g, cz_req);
  dim3 grid(g.nx / FX_TX, g.ny / FX_TY, (g.nz + cz - 1) / cz);
  const int nb = (int)(grid.x * grid.y * grid.z);
  if (nb > nb_max) return cudaErrorInvalidValue;
  *nb_out = nb;
  ++g_launches;
  const bool zero_in = phi_in == nullptr;
  static std::atomic<int> configured[64];
  int dev = 0;
  cudaGetDevice(&dev);
  // the step's kernels by periodic-axis mask (0..7) and zero start
  using Kf = void (*)(const long long*, long long*, const float*, float, const long long*,
                      float*, Grid, FxBc, float, int, double*, long long*, int*);
  static const Kf kfs[8][2] = {
      {k_fx_step<0, false>, k_fx_step<0, true>}, {k_fx_step<1, false>, k_fx_step<1, true>},
      {k_fx_step<2, false>, k_fx_step<2, true>}, {k_fx_step<3, false>, k_fx_step<3, true>},
      {k_fx_step<4, false>, k_fx_step<4, true>}, {k_fx_step<5, false>, k_fx_step<5, true>},
      {k_fx_step<6, false>, k_fx_step<6, true>}, {k_fx_step<7, false>, k_fx_step<7, true>}};
  if (dev >= 0 && dev < 64 && !configured[dev].load()) {
    for (const auto& pair : kfs)
      for (Kf kf : pair) {
        const cudaError_t e2 =
            cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFxSmem);
        if (e2 != cudaSuccess) return e2;
      }
    configured[dev].store(1);
  }
  const Kf kf = kfs[pm][zero_in ? 1 : 0];
  kf<<<grid, FX_TX * FX_TY, kFxSmem, s>>>(phi_in, phi_out, e, c, F, r32, g, b, factor, cz,
                                          partials, psum, flag);
  return cudaGetLastError();
}

cudaError_t launch_fx_finish_gravity(const long long* q, double* phi, double* g, Grid gr,
                                     const Bc& bc, double h, int S, const long long* mean,
                                     cudaStream_t s) {
  const double two_pow_S = std::ldexp(1.0, S);
  const FxBc b = fx_bc(bc, two_pow_S);
  ++g_launches;
  k_fx_finish_gravity<<<grid_for(gr.cells()), kThreads, 0, s>>>(
      q, phi, g, gr, b, S, 1.0 / (2.0 * h * two_pow_S), mean);
  return cudaGetLastError();
}

cudaError_t launch_finish_fx_sum(const long long* psum, int nb, long long n, double* out,
                                 cudaStream_t s) {
  int log2n = 0;
  while ((1LL << log2n) < n) ++log2n;
  if ((1LL << log2n) != n) return cudaErrorInvalidValue;  // levels have 2^k cells
  ++g_launches;
  k_finish_fx_sum<<<1, kThreads, 0, s>>>(psum, nb, log2n, out);
  return cudaGetLastError();
}

}  // namespace mg
