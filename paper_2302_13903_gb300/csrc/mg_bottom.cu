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

#include <atomic>

#include "mg_bottom.cuh"
#include "mg_device.cuh"
#include "mg_internal.h"

namespace mg {
namespace {

constexpr int kBottomThreads = 512;
using bottom::BottomArgs;
using bottom::vcycle;

template <typename T>
__global__ void __launch_bounds__(kBottomThreads) k_bottom(BottomArgs<T> a) {
  extern __shared__ double bottom_smem[];
  T* sm = reinterpret_cast<T*>(bottom_smem);
  if (!a.fmg) {
    bottom::in_shared(a, sm, false, [&](const BottomArgs<T>& b) { vcycle(b, b.top, b.hom, true); });
    return;
  }
  bottom::in_shared(a, sm, false, [&](const BottomArgs<T>& b) {
    for (int l = b.top; l >= 1; --l) {
      const Grid g{b.n[l], b.n[l], b.n[l]};
      dev::restrict_range(b.f[l], b.f[l - 1], g, threadIdx.x, blockDim.x);
      __syncthreads();
    }
    if (threadIdx.x == 0) dev::coarsest_one(b.f[0], b.u[0], b.h[0], b.bc[0]);
    __syncthreads();
    for (int l = 1; l <= b.top; ++l) {
      const Grid g{b.n[l], b.n[l], b.n[l]};
      dev::prolong_range<T, true>(b.u[l - 1], b.u[l], g, b.bc[l - 1], 0, threadIdx.x, blockDim.x);
      __syncthreads();
      vcycle(b, l, b.bc[l], false);
    }
  });
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
  bottom::set_coefficients(a);
  const size_t smem = 2 * (size_t)bottom::cells_upto(a) * sizeof(T);
  static std::atomic<int> configured[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !configured[dev].load()) {
    // room for the largest case: levels up to 16^3 in FP64 (75 KB)
    const cudaError_t e = cudaFuncSetAttribute(k_bottom<T>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(2 * 4681 * sizeof(double)));
    if (e != cudaSuccess) return e;
    configured[dev].store(1);
  }
  ++g_launches;
  k_bottom<T><<<1, kBottomThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_bottom<float>(float* const*, float* const*, const int*, const double*,
                                          const Bc*, Bc, double, int, int, int, bool,
                                          cudaStream_t);
template cudaError_t launch_bottom<double>(double* const*, double* const*, const int*,
                                           const double*, const Bc*, Bc, double, int, int, int,
                                           bool, cudaStream_t);

}  // namespace mg
