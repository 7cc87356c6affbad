// mg_fused_ud_masks.cu -- the fused up-down kernel for rules per face whose
// periodic axes are x only, y only, z only, x and z, or y and z (masks 1, 2,
// 4, 5, 6); mg_fused_ud.cu has masks 0, 3 and 7.  A separate translation unit,
// compiled in parallel.
#include "mg_fused_ud_launch.cuh"

namespace mg {
namespace fused {

cudaError_t dispatch_ud_other(int pm, const float* ui, float* uo, const float* f, const float* ec,
                              float* fc, FusedParams p, TileCfg cfg, cudaStream_t s) {
  switch (pm) {
    case 1: return dispatch_ud_t<1>(ui, uo, f, ec, fc, p, cfg, s);
    case 2: return dispatch_ud_t<2>(ui, uo, f, ec, fc, p, cfg, s);
    case 4: return dispatch_ud_t<4>(ui, uo, f, ec, fc, p, cfg, s);
    case 5: return dispatch_ud_t<5>(ui, uo, f, ec, fc, p, cfg, s);
    case 6: return dispatch_ud_t<6>(ui, uo, f, ec, fc, p, cfg, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fused
}  // namespace mg
