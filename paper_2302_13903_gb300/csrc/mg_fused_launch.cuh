// mg_fused_launch.cuh -- host-side launch templates of the fused FP32
// V-cycle-leg kernels, shared by the translation units that instantiate them
// (mg_fused.cu: the periodic-axis masks 0, 3, 7; mg_fused_masks_a.cu and
// mg_fused_masks_b.cu: the others, compiled in parallel).
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include "mg_fused.cuh"
#include "mg_internal.h"

namespace mg {
namespace fused {


template <int MODE, bool ZERO, int PM, int TX, int TY>
inline cudaError_t launch_t(const float* ui, float* uo, const float* f, const float* ec, float* fc,
                     const FusedParams& p, cudaStream_t s) {
  using S_ = Shape<MODE, TX, TY>;
  static std::atomic<int> configured[64];  // zero-initialised (static storage)
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !configured[dev].load()) {
    cudaError_t e = cudaFuncSetAttribute(k_fused<MODE, ZERO, PM, TX, TY>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)S_::SMEM);
    if (e != cudaSuccess) return e;
    configured[dev].store(1);
  }
  dim3 grid(p.nx / TX, p.ny / TY, (p.nz + p.cz - 1) / p.cz);
  ++g_launches;
  k_fused<MODE, ZERO, PM, TX, TY><<<grid, S_::NT, S_::SMEM, s>>>(ui, uo, f, ec, fc, p);
  return cudaGetLastError();
}

// Built-in shape: tiles of 64 x 16 for levels >= 64 cells wide, 32 x 16 for
// 32 (32 rows when asked); the z-chunk is the largest of 64, 32, 16, 8 planes that still gives two
// CTAs per SM.  A nonzero cfg field (checked by fused_cfg_ok) replaces it.
template <int MODE, bool ZERO, int PM>
inline cudaError_t dispatch_t(const float* ui, float* uo, const float* f, const float* ec, float* fc,
                       FusedParams p, TileCfg cfg, cudaStream_t s) {
  const int tx = cfg.tx ? cfg.tx : (p.nx >= 64 ? 64 : 32), ty = cfg.ty ? cfg.ty : 16;
  p.cz = chunk_planes(p, tx, ty, cfg.cz);
  if (ty == 32) {
    if (tx == 64) return launch_t<MODE, ZERO, PM, 64, 32>(ui, uo, f, ec, fc, p, s);
    return launch_t<MODE, ZERO, PM, 32, 32>(ui, uo, f, ec, fc, p, s);
  }
  if (tx == 64) return launch_t<MODE, ZERO, PM, 64, 16>(ui, uo, f, ec, fc, p, s);
  return launch_t<MODE, ZERO, PM, 32, 16>(ui, uo, f, ec, fc, p, s);
}

// The legs for periodic-axis masks 1, 2, 4 (mg_fused_masks_a.cu) and 5, 6
// (mg_fused_masks_b.cu).
cudaError_t dispatch_mask_124(int pm, int mode, bool zero, const float* ui, float* uo,
                              const float* f, const float* ec, float* fc, FusedParams p,
                              TileCfg cfg, cudaStream_t s);
cudaError_t dispatch_mask_56(int pm, int mode, bool zero, const float* ui, float* uo,
                             const float* f, const float* ec, float* fc, FusedParams p,
                             TileCfg cfg, cudaStream_t s);

}  // namespace fused
}  // namespace mg
