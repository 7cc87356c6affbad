// mg_fused.cu -- launchers of the fused FP32 V-cycle-leg kernels (the
// programs themselves are in mg_fused.cuh).
#include <cuda_runtime.h>

#include "mg_fused_launch.cuh"

namespace mg {
namespace fused {
namespace {

// Periodic axes of a rule: bit 0 x, 1 y, 2 z.
int periodic_mask(const Bc& bc) {
  int m = 0;
  for (int a = 0; a < 3; ++a)
    if (face_kind(bc, 2 * a) == BC_PERIODIC) m |= 1 << a;
  return m;
}

template <int MODE, bool ZERO>
cudaError_t dispatch(const float* ui, float* uo, const float* f, const float* ec, float* fc,
                     FusedParams p, const Bc& bc, TileCfg cfg, cudaStream_t s) {
  const int pm = periodic_mask(bc);
  switch (pm) {
    case 7: return dispatch_t<MODE, ZERO, 7>(ui, uo, f, ec, fc, p, cfg, s);
    case 3: return dispatch_t<MODE, ZERO, 3>(ui, uo, f, ec, fc, p, cfg, s);
    case 0: return dispatch_t<MODE, ZERO, 0>(ui, uo, f, ec, fc, p, cfg, s);
    case 5:
    case 6: return dispatch_mask_56(pm, MODE, ZERO, ui, uo, f, ec, fc, p, cfg, s);
    default: return dispatch_mask_124(pm, MODE, ZERO, ui, uo, f, ec, fc, p, cfg, s);
  }
}

}  // namespace
}  // namespace fused

using fused::FusedParams;
using fused::kDown;
using fused::kUp;
using fused::kPlain;
using fused::dispatch;
using fused::params;

bool fused_ok(Grid g, const Bc& bc) {
  // homogeneous: no open face, fixed faces at 0 (a MIXED rule without face
  // values); any periodic axes
  bool hom = bc.kind != BC_OPEN;
  if (bc.kind == BC_FIXED) hom = hom && bc.value == 0.0;
  if (bc.kind == BC_MIXED) hom = hom && bc.faces == nullptr;
  // widths the 64- or 32-wide tiles divide, rows in 16s, planes in 8s;
  // element offsets of 32 bits
  return hom && g.nx >= 32 && g.ny >= 32 && g.nz >= 32 && g.nx % 32 == 0 && g.ny % 16 == 0 &&
         g.nz % 8 == 0 && (g.nx < 64 || g.nx % 64 == 0) && g.cells() < (1LL << 32);
}

bool fused_cfg_ok(Grid g, TileCfg cfg) {
  const bool tx_ok = cfg.tx == 0 || (cfg.tx == 32 && g.nx % 32 == 0) ||
                     (cfg.tx == 64 && g.nx % 64 == 0);
  const bool cz_ok = cfg.cz == 0 || (cfg.cz >= 4 && cfg.cz % 4 == 0 && cfg.cz <= 1024);
  const bool ty_ok = cfg.ty == 0 || cfg.ty == 16 || (cfg.ty == 32 && g.ny % 32 == 0);
  return tx_ok && cz_ok && ty_ok;
}

cudaError_t launch_fused_down(const float* u_in, float* u_out, const float* f, float* fc, Grid g,
                              double h, Bc bc, double omega, bool zero_guess, cudaStream_t s,
                              TileCfg cfg) {
  if (!fused_cfg_ok(g, cfg)) return cudaErrorInvalidValue;
  const FusedParams p = params(g, h, bc, omega);
  return zero_guess ? dispatch<kDown, true>(u_in, u_out, f, nullptr, fc, p, bc, cfg, s)
                    : dispatch<kDown, false>(u_in, u_out, f, nullptr, fc, p, bc, cfg, s);
}

cudaError_t launch_fused_up(const float* u_in, float* u_out, const float* f, const float* ec,
                            Grid g, double h, Bc bc, double omega, cudaStream_t s, TileCfg cfg) {
  if (!fused_cfg_ok(g, cfg)) return cudaErrorInvalidValue;
  return dispatch<kUp, false>(u_in, u_out, f, ec, nullptr, params(g, h, bc, omega), bc, cfg, s);
}

cudaError_t launch_fused_smooth(const float* u_in, float* u_out, const float* f, Grid g, double h,
                                Bc bc, double omega, bool zero_guess, cudaStream_t s,
                                TileCfg cfg) {
  if (!fused_cfg_ok(g, cfg)) return cudaErrorInvalidValue;
  const FusedParams p = params(g, h, bc, omega);
  return zero_guess ? dispatch<kPlain, true>(u_in, u_out, f, nullptr, nullptr, p, bc, cfg, s)
                    : dispatch<kPlain, false>(u_in, u_out, f, nullptr, nullptr, p, bc, cfg, s);
}

}  // namespace mg
