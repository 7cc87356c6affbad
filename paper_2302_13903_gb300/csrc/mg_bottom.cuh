// mg_bottom.cuh -- block-level programs for the coarse end of a V-cycle
// (device code shared by the single-CTA bottom kernel and the batched solver).
// Each step is a block-strided loop over one level followed by __syncthreads;
// global memory written by the CTA is visible to the whole CTA after the
// barrier.
#pragma once

#include <cuda_runtime.h>

#include "mg_device.cuh"
#include "mg_internal.h"

namespace mg {
namespace bottom {

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

// Cells of levels 0 .. top together.
template <typename T>
__host__ __device__ inline int cells_upto(const BottomArgs<T>& a) {
  int total = 0;
  for (int l = 0; l <= a.top; ++l) total += a.n[l] * a.n[l] * a.n[l];
  return total;
}

// Runs `body` on copies of levels 0 .. top held in shared memory `smem` (room
// for 2 cells_upto(a) values of T): the levels' f and u then have the latency
// of shared memory, not of L2.  f[top] is copied in, and u[top] when its start
// value is used (load_u); u[top] is copied back out.  Lower levels are
// scratch of the cycle (their f comes from restriction, their u starts at 0).
template <typename T, typename Body>
__device__ void in_shared(const BottomArgs<T>& a, T* smem, bool load_u, Body body) {
  BottomArgs<T> b = a;
  const int total = cells_upto(a);
  int off = 0;
  for (int l = 0; l <= a.top; ++l) {
    b.u[l] = smem + off;
    b.f[l] = smem + total + off;
    off += a.n[l] * a.n[l] * a.n[l];
  }
  const int top = a.top, ct = a.n[top] * a.n[top] * a.n[top];
  for (int t = threadIdx.x; t < ct; t += blockDim.x) {
    b.f[top][t] = a.f[top][t];
    if (load_u) b.u[top][t] = a.u[top][t];
  }
  __syncthreads();
  body(b);
  __syncthreads();
  for (int t = threadIdx.x; t < ct; t += blockDim.x) a.u[top][t] = b.u[top][t];
  __syncthreads();
}

}  // namespace bottom
}  // namespace mg
