// mg_fused_ud_launch.cuh -- host-side launch template of the fused up-down
// kernel (mg_fused_ud.cuh), shared by the translation units that instantiate
// it for the periodic-axis masks (compiled in parallel).
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include "mg_fused_ud.cuh"
#include "mg_internal.h"

namespace mg {
namespace fused {

template <int PM, int TX, int TY>
inline cudaError_t launch_ud_t(const float* ui, float* uo, const float* f, const float* ec,
                               float* fc, const FusedParams& p, cudaStream_t s) {
  using S_ = ShapeUD<TX, TY>;
  static std::atomic<int> configured[64];  // zero-initialised (static storage)
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !configured[dev].load()) {
    cudaError_t e = cudaFuncSetAttribute(k_updown<PM, TX, TY>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)S_::SMEM);
    if (e != cudaSuccess) return e;
    configured[dev].store(1);
  }
  dim3 grid(p.nx / TX, p.ny / TY, (p.nz + p.cz - 1) / p.cz);
  ++g_launches;
  k_updown<PM, TX, TY><<<grid, S_::NT, S_::SMEM, s>>>(ui, uo, f, ec, fc, p);
  return cudaGetLastError();
}

// Tiles of 64 cells by 32 rows (16 when the level has rows in 16s only); the
// z-chunk is the largest of 128 .. 8 planes that still gives four CTAs per SM
// over the grid.  Nonzero cfg fields (checked by updown_cfg_ok) replace it.
template <int PM>
inline cudaError_t dispatch_ud_t(const float* ui, float* uo, const float* f, const float* ec,
                                 float* fc, FusedParams p, TileCfg cfg, cudaStream_t s) {
  const long long sms = sm_count();
  const int ty = cfg.ty ? cfg.ty : (p.ny % 32 == 0 ? 32 : 16);
  const long long cols = (long long)(p.nx / 64) * (p.ny / ty);
  int cz = 128;
  while (cz > 8 && cols * ((p.nz + cz - 1) / cz) < 4 * sms) cz /= 2;
  if (cfg.cz) cz = cfg.cz;
  p.cz = cz < p.nz ? cz : p.nz;
  if (ty == 32) return launch_ud_t<PM, 64, 32>(ui, uo, f, ec, fc, p, s);
  return launch_ud_t<PM, 64, 16>(ui, uo, f, ec, fc, p, s);
}

// Masks 1, 2, 4, 5, 6 (mg_fused_ud_masks.cu).
cudaError_t dispatch_ud_other(int pm, const float* ui, float* uo, const float* f, const float* ec,
                              float* fc, FusedParams p, TileCfg cfg, cudaStream_t s);

}  // namespace fused
}  // namespace mg
