// mg_fused_ud.cu -- launcher of the fused up-down kernel (the up leg of one
// V-cycle and the down leg of the next on one FP32 level; mg_fused_ud.cuh).
#include <cuda_runtime.h>

#include "mg_fused_ud_launch.cuh"

namespace mg {

bool updown_ok(Grid g, const Bc& bc) {
  // the fused legs' conditions, 64-cell tiles, rows in 16s, at least two
  // z-chunks' worth of planes
  return fused_ok(g, bc) && g.nx % 64 == 0 && g.ny % 16 == 0 && g.nz >= 16;
}

bool updown_cfg_ok(Grid g, TileCfg cfg) {
  return (cfg.tx == 0 || cfg.tx == 64) && (cfg.ty == 0 || cfg.ty == 16 ||
                                           (cfg.ty == 32 && g.ny % 32 == 0)) &&
         (cfg.cz == 0 || (cfg.cz >= 8 && cfg.cz % 8 == 0 && cfg.cz <= 1024));
}

cudaError_t launch_fused_updown(const float* u_in, float* u_out, const float* f, const float* ec,
                                float* fc, Grid g, double h, Bc bc, double omega, cudaStream_t s,
                                TileCfg cfg) {
  if (!updown_ok(g, bc) || !updown_cfg_ok(g, cfg)) return cudaErrorInvalidValue;
  fused::FusedParams p;
  p.nx = g.nx; p.ny = g.ny; p.nz = g.nz;
  float sg[6];
  int pm = 0;
  for (int q = 0; q < 6; ++q) sg[q] = face_kind(bc, q) == BC_ZEROGRAD ? 1.f : -1.f;
  for (int a = 0; a < 3; ++a)
    if (face_kind(bc, 2 * a) == BC_PERIODIC) pm |= 1 << a;
  p.sx0 = sg[0]; p.sx1 = sg[1]; p.sy0 = sg[2]; p.sy1 = sg[3]; p.sz0 = sg[4]; p.sz1 = sg[5];
  p.cu = (float)(1.0 - omega);
  p.cs = (float)(omega / 6.0);
  p.cf = (float)(-omega * h * h / 6.0);
  p.inv_h2 = (float)(1.0 / (h * h));
  p.cz = 8;
  switch (pm) {
    case 7: return fused::dispatch_ud_t<7>(u_in, u_out, f, ec, fc, p, cfg, s);
    case 3: return fused::dispatch_ud_t<3>(u_in, u_out, f, ec, fc, p, cfg, s);
    case 0: return fused::dispatch_ud_t<0>(u_in, u_out, f, ec, fc, p, cfg, s);
    default: return fused::dispatch_ud_other(pm, u_in, u_out, f, ec, fc, p, cfg, s);
  }
}

}  // namespace mg
