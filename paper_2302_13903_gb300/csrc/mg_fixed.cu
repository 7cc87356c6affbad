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

#include <cmath>

#include "mg_device.cuh"
#include "mg_internal.h"

namespace mg {
namespace {

constexpr int kThreads = 256;

int grid_for(long long work) {
  long long b = (work + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  if (b > 152LL * 64) b = 152LL * 64;
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
template <typename T>
__global__ void k_absmax(const T* __restrict__ a, long long n, double* __restrict__ partials) {
  T m = T(0);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const T v = a[t] < T(0) ? -a[t] : a[t];
    m = v > m ? v : m;
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

// In place: the double a[t] becomes the integer round(a[t] * c).
__global__ void k_f64_to_fx(double* a, long long n, double c) {
  long long* q = reinterpret_cast<long long*>(a);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    q[t] = __double2ll_rn(a[t] * c);
}

// out[t] = q[t] * c as a double (out may alias q).
__global__ void k_fx_to_f64(const long long* q, double* out, long long n, double c) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    out[t] = __ll2double_rn(q[t]) * c;
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

struct FxBc {
  int kind;
  long long b2;          // FIXED: 2 round(b 2^S)
  const double* faces;   // OPEN: boundary values (doubles), scaled by c2 = 2^(S+1)
  double c2;
};

// One outer step on the integer grid, fused and z-marching:
//   PHI' = PHI_in + round(e * c)          (the pending FP32 correction; e may be null)
//   R    = F - (sum_nb PHI' - 6 PHI')      (exact)
//   r32  = R * factor, partial sums of r32^2, PHI_out = PHI' (a different buffer:
//   neighbouring tiles read PHI_in as their halo).
// A 32 x 16 tile of columns marches through a chunk of planes with a ring of
// three corrected planes (halo of one cell) in shared memory.
constexpr int FX_TX = 32, FX_TY = 16, FX_W = FX_TX + 2, FX_H = FX_TY + 2;

__device__ __forceinline__ long long fx_face_ghost(const FxBc& bc, const Grid& g, long long self,
                                                   int i, int j, int k, int axis, int hi) {
  if (bc.kind == BC_ZEROGRAD) return self;
  long long b2 = bc.b2;
  if (bc.kind == BC_OPEN) {
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

__global__ void __launch_bounds__(FX_TX* FX_TY)
    k_fx_step(const long long* __restrict__ phi_in, long long* __restrict__ phi_out,
              const float* __restrict__ e, float c, const long long* __restrict__ F,
              float* __restrict__ r32, Grid g, FxBc bc, float factor, int cz,
              double* __restrict__ partials, int* __restrict__ flag) {
  __shared__ long long P[3][FX_H][FX_W];
  const bool per = bc.kind == BC_PERIODIC;
  const int tx = threadIdx.x % FX_TX, ty = threadIdx.x / FX_TX;
  const int x0 = blockIdx.x * FX_TX, y0 = blockIdx.y * FX_TY, z0 = blockIdx.z * cz;
  const int z1 = min(z0 + cz, g.nz);
  const int i = x0 + tx, j = y0 + ty;  // this thread's interior column
  const size_t plane = (size_t)g.nx * g.ny;
  float acc = 0.f;
  bool bad = false;
  for (int q = z0 - 1; q <= z1; ++q) {
    const int slot = (q - z0 + 1) % 3;
    __syncthreads();  // the slot being refilled was read two planes ago
    const bool q_in = per || (q >= 0 && q < g.nz);
    const int qw = per ? (q < 0 ? q + g.nz : (q >= g.nz ? q - g.nz : q)) : q;
    for (int idx = threadIdx.x; idx < FX_W * FX_H; idx += blockDim.x) {
      const int a = idx % FX_W, b = idx / FX_W;
      int gx = x0 - 1 + a, gy = y0 - 1 + b;
      long long v = 0;
      bool in = q_in;
      if (per) {
        gx = gx < 0 ? gx + g.nx : (gx >= g.nx ? gx - g.nx : gx);
        gy = gy < 0 ? gy + g.ny : (gy >= g.ny ? gy - g.ny : gy);
      } else {
        in = in && gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny;
      }
      if (in) {
        const size_t o = (size_t)qw * plane + (size_t)gy * g.nx + gx;
        v = phi_in[o];
        if (e) v += __float2ll_rn(e[o] * c);
        // the owner of an interior cell of this tile stores it
        if (a >= 1 && a <= FX_TX && b >= 1 && b <= FX_TY && q >= z0 && q < z1) {
          phi_out[o] = v;
          bad |= (v > (1LL << 60)) || (v < -(1LL << 60));
        }
      }
      P[slot][b][a] = v;
    }
    __syncthreads();
    const int pz = q - 1;  // residual of the plane below, now that q is in
    if (pz >= z0 && pz < z1) {
      const int sm = (slot + 1) % 3, s0 = (slot + 2) % 3;  // planes pz-1, pz
      const long long self = P[s0][ty + 1][tx + 1];
      long long xm = P[s0][ty + 1][tx], xp = P[s0][ty + 1][tx + 2];
      long long ym = P[s0][ty][tx + 1], yp = P[s0][ty + 2][tx + 1];
      long long zm = P[sm][ty + 1][tx + 1], zp = P[slot][ty + 1][tx + 1];
      if (!per) {
        if (i == 0) xm = fx_face_ghost(bc, g, self, i, j, pz, 0, 0);
        if (i == g.nx - 1) xp = fx_face_ghost(bc, g, self, i, j, pz, 0, 1);
        if (j == 0) ym = fx_face_ghost(bc, g, self, i, j, pz, 1, 0);
        if (j == g.ny - 1) yp = fx_face_ghost(bc, g, self, i, j, pz, 1, 1);
        if (pz == 0) zm = fx_face_ghost(bc, g, self, i, j, pz, 2, 0);
        if (pz == g.nz - 1) zp = fx_face_ghost(bc, g, self, i, j, pz, 2, 1);
      }
      const size_t o = (size_t)pz * plane + (size_t)j * g.nx + i;
      const long long R = F[o] - (((xm + xp) + (ym + yp)) + (zm + zp) - 6 * self);
      const float r = __ll2float_rn(R) * factor;
      r32[o] = r;
      acc = fmaf(r, r, acc);
    }
  }
  if (bad) atomicOr(flag, 1);
  // deterministic block sum, then one partial per block (blocks in launch order)
  __shared__ double ws[FX_TX * FX_TY / 32];
  double v = warp_sum((double)acc);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) ws[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < FX_TX * FX_TY / 32; ++q) t += ws[q];
    partials[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
  }
}

}  // namespace

template <typename T>
cudaError_t launch_absmax(const T* a, long long n, double* partials, double* out, cudaStream_t s) {
  const int nb = reduce_blocks(n);
  ++g_launches;
  k_absmax<T><<<nb, kThreads, 0, s>>>(a, n, partials);
  ++g_launches;
  k_finish_max<<<1, kThreads, 0, s>>>(partials, nb, out);
  return cudaGetLastError();
}
template cudaError_t launch_absmax<double>(const double*, long long, double*, double*, cudaStream_t);
template cudaError_t launch_absmax<float>(const float*, long long, double*, double*, cudaStream_t);

cudaError_t launch_f64_to_fx(double* a, long long n, double c, cudaStream_t s) {
  ++g_launches;
  k_f64_to_fx<<<grid_for(n), kThreads, 0, s>>>(a, n, c);
  return cudaGetLastError();
}

cudaError_t launch_fx_to_f64(const long long* q, double* out, long long n, double c,
                             cudaStream_t s) {
  ++g_launches;
  k_fx_to_f64<<<grid_for(n), kThreads, 0, s>>>(q, out, n, c);
  return cudaGetLastError();
}

cudaError_t launch_fx_correct(long long* phi, const float* e, long long n, float c, int* flag,
                              cudaStream_t s) {
  ++g_launches;
  k_fx_correct<<<grid_for(n), kThreads, 0, s>>>(phi, e, n, c, flag);
  return cudaGetLastError();
}

bool fx_step_ok(Grid g) { return g.nx % FX_TX == 0 && g.ny % FX_TY == 0; }

// Planes per CTA: the given cz, else the largest of 64 .. 4 that still
// gives four CTAs per SM.
int fx_step_cz(Grid g, int cz) {
  const long long cols = (long long)(g.nx / FX_TX) * (g.ny / FX_TY);
  if (cz <= 0) {
    cz = 64;
    while (cz > kFxMinCz && cols * ((g.nz + cz - 1) / cz) < 4 * 152) cz /= 2;
  }
  return cz > g.nz ? g.nz : cz;
}

// Blocks of a launch with `cz` planes per CTA; cz = 0: the most any allowed
// cz (>= kFxMinCz) gives, to size the partial sums.
int fx_step_blocks(Grid g, int cz) {
  const long long cols = (long long)(g.nx / FX_TX) * (g.ny / FX_TY);
  const int z = cz > 0 ? fx_step_cz(g, cz) : (g.nz < kFxMinCz ? g.nz : kFxMinCz);
  return (int)(cols * ((g.nz + z - 1) / z));
}

cudaError_t launch_fx_step(const long long* phi_in, long long* phi_out, const float* e, float c,
                           const long long* F, float* r32, Grid g, const Bc& bc, double two_pow_S,
                           float factor, double* partials, int nb_max, int* flag, int* nb_out,
                           cudaStream_t s, int cz_req) {
  // The ghost 2 b - phi on the fixed-point grid: 2 b 2^S rounded once.
  FxBc b;
  b.kind = bc.kind;
  b.c2 = 2.0 * two_pow_S;
  b.b2 = bc.kind == BC_FIXED ? (long long)std::llrint(bc.value * b.c2) : 0;
  b.faces = bc.faces;
  if (cz_req != 0 && cz_req < kFxMinCz) return cudaErrorInvalidValue;
  const int cz = fx_step_cz(g, cz_req);
  dim3 grid(g.nx / FX_TX, g.ny / FX_TY, (g.nz + cz - 1) / cz);
  const int nb = (int)(grid.x * grid.y * grid.z);
  if (nb > nb_max) return cudaErrorInvalidValue;
  *nb_out = nb;
  ++g_launches;
  k_fx_step<<<grid, FX_TX * FX_TY, 0, s>>>(phi_in, phi_out, e, c, F, r32, g, b, factor, cz,
                                           partials, flag);
  return cudaGetLastError();
}

}  // namespace mg
