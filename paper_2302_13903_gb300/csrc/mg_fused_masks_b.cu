// mg_fused_masks_b.cu -- the fused FP32 V-cycle legs for rules per face whose
// periodic axes are x and z or y and z (masks 5, 6); mg_fused.cu has
// masks 0, 3 and 7.  Separate translation units, so that the build compiles
// them in parallel.
#include "mg_fused_launch.cuh"

namespace mg {
namespace fused {

namespace {

template <int MODE, bool ZERO>
cudaError_t by_mask(int pm, const float* ui, float* uo, const float* f, const float* ec,
                    float* fc, const FusedParams& p, TileCfg cfg, cudaStream_t s) {
  switch (pm) {
    case 5: return dispatch_t<MODE, ZERO, 5>(ui, uo, f, ec, fc, p, cfg, s);
    case 6: return dispatch_t<MODE, ZERO, 6>(ui, uo, f, ec, fc, p, cfg, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t dispatch_mask_56(int pm, int mode, bool zero, const float* ui, float* uo,
                                const float* f, const float* ec, float* fc, FusedParams p,
                                TileCfg cfg, cudaStream_t s) {
  if (mode == kDown)
    return zero ? by_mask<kDown, true>(pm, ui, uo, f, ec, fc, p, cfg, s)
                : by_mask<kDown, false>(pm, ui, uo, f, ec, fc, p, cfg, s);
  if (mode == kUp) return by_mask<kUp, false>(pm, ui, uo, f, ec, fc, p, cfg, s);
  return zero ? by_mask<kPlain, true>(pm, ui, uo, f, ec, fc, p, cfg, s)
              : by_mask<kPlain, false>(pm, ui, uo, f, ec, fc, p, cfg, s);
}

}  // namespace fused
}  // namespace mg
