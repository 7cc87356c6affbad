// mg_bottom.cu -- the coarse end of a V-cycle or of the FMG ladder in one CTA.
//
// The levels at or below 16^3 cells hold at most 4681 cells together, too few
// to fill a GPU: as separate launches they cost one launch latency per smoothing
// half-step.  Here one CTA of 512 threads runs all of them in order, each step
// a block-strided loop over the level followed by __syncthreads (global
// memory written by the CTA is visible to the whole CTA after the barrier).
//   VCYCLE: levels top .. 1 as corrections from 0 (Algorithm 1 steps 1-3),
//           COARSEST on level 0, then steps 5-7 back up to `top`.
//   FMG:    Algorithm 2 up to level `top` (restrict f down, COARSEST, then
//           I' prolongation and one V-cycle per level), every level with its
//           physical rule and the homogeneous rule below the top of a cycle.
#include <cuda_runtime.h>

#include "mg_device.cuh"
#include "mg_internal.h"

namespace mg {
namespace {

constexpr int kBottomThreads = 512;

template <typename T>
struct BottomArgs {
  T* u[kBottomLevels];
  T* f[kBottomLevels];
  int n[kBottomLevels];
  double h[kBottomLevels];
  Bc bc[kBottomLevels];  // physical rule of each level (FMG)
  Bc hom;                // homogeneous rule (corrections)
  double omega;
  int pre, post;
  int top;
  int fmg;
};

template <typename T>
__device__ void smooth_level(const BottomArgs<T>& a, int l, const Bc& bc, int steps,
                             bool zero_guess) {
  const Grid g{a.n[l], a.n[l], a.n[l]};
  const double h = a.h[l], om = a.omega;
  const T cu = (T)(1.0 - om), cs = (T)(om / 6.0), cf = (T)(-om * h * h / 6.0);
  if (zero_guess && steps == 0) {
    for (long long t = threadIdx.x; t < g.cells(); t += blockDim.x) a.u[l][t] = T(0);
    __syncthreads();
    return;
  }
  for (int q = 0; q < steps; ++q) {
    if (q == 0 && zero_guess)
      dev::sor_red_zero_range(a.u[l], a.f[l], g, cf, threadIdx.x, blockDim.x);
    else
      dev::sor_range(a.u[l], a.f[l], g, bc, cu, cs, cf, 0, threadIdx.x, blockDim.x);
    __syncthreads();
    dev::sor_range(a.u[l], a.f[l], g, bc, cu, cs, cf, 1, threadIdx.x, blockDim.x);
    __syncthreads();
  }
}

// One V-cycle on levels top .. 0 with rule bc_top on level `top`.
template <typename T>
__device__ void vcycle(const BottomArgs<T>& a, int top, const Bc& bc_top, bool zero_guess) {
  for (int l = top; l >= 1; --l) {
    const Bc& bc = (l == top) ? bc_top : a.hom;
    smooth_level(a, l, bc, a.pre, l < top || zero_guess);
    const Grid g{a.n[l], a.n[l], a.n[l]};
    dev::defect_restrict_range(a.u[l], a.f[l], a.f[l - 1], g, bc, (T)(1.0 / (a.h[l] * a.h[l])),
                               threadIdx.x, blockDim.x);
    __syncthreads();
  }
  if (threadIdx.x == 0) dev::coarsest_one(a.f[0], a.u[0], a.h[0], top == 0 ? bc_top : a.hom);
  __syncthreads();
  for (int l = 1; l <= top; ++l) {
    const Bc& bc = (l == top) ? bc_top : a.hom;
    const Grid g{a.n[l], a.n[l], a.n[l]};
    dev::prolong_range<T, false>(a.u[l - 1], a.u[l], g, a.hom, 1, threadIdx.x, blockDim.x);
    __syncthreads();
    smooth_level(a, l, bc, a.post, false);
  }
}

template <typename T>
__global__ void __launch_bounds__(kBottomThreads) k_bottom(BottomArgs<T> a) {
  if (!a.fmg) {
    vcycle(a, a.top, a.hom, true);
    return;
  }
  for (int l = a.top; l >= 1; --l) {
    const Grid g{a.n[l], a.n[l], a.n[l]};
    dev::restrict_range(a.f[l], a.f[l - 1], g, threadIdx.x, blockDim.x);
    __syncthreads();
  }
  if (threadIdx.x == 0) dev::coarsest_one(a.f[0], a.u[0], a.h[0], a.bc[0]);
  __syncthreads();
  for (int l = 1; l <= a.top; ++l) {
    const Grid g{a.n[l], a.n[l], a.n[l]};
    dev::prolong_range<T, true>(a.u[l - 1], a.u[l], g, a.bc[l - 1], 0, threadIdx.x, blockDim.x);
    __syncthreads();
    vcycle(a, l, a.bc[l], false);
  }
}

}  // namespace

template <typename T>
cudaError_t launch_bottom(T* const* u, T* const* f, const int* n, const double* h, const Bc* bc,
                          Bc hom, double omega, int pre, int post, int top, bool fmg,
                          cudaStream_t s) {
  if (top < 0 || top >= kBottomLevels) return cudaErrorInvalidValue;
  BottomArgs<T> a;
  for (int l = 0; l < kBottomLevels; ++l) {
    const bool used = l <= top;
    a.u[l] = used ? u[l] : nullptr;
    a.f[l] = used ? f[l] : nullptr;
    a.n[l] = used ? n[l] : 0;
    a.h[l] = used ? h[l] : 0.0;
    a.bc[l] = used && bc ? bc[l] : hom;
  }
  a.hom = hom;
  a.omega = omega;
  a.pre = pre;
  a.post = post;
  a.top = top;
  a.fmg = fmg ? 1 : 0;
  ++g_launches;
  k_bottom<T><<<1, kBottomThreads, 0, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_bottom<float>(float* const*, float* const*, const int*, const double*,
                                          const Bc*, Bc, double, int, int, int, bool,
                                          cudaStream_t);
template cudaError_t launch_bottom<double>(double* const*, double* const*, const int*,
                                           const double*, const Bc*, Bc, double, int, int, int,
                                           bool, cudaStream_t);

}  // namespace mg
