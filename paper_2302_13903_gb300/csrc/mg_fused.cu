// mg_fused.cu -- launchers of the fused FP32 V-cycle-leg kernels (the
// programs themselves are in mg_fused.cuh).
#include <cuda_runtime.h>

#include <atomic>

#include "mg_fused.cuh"
#include "mg_internal.h"

namespace mg {
namespace fused {
namespace {

template <int MODE, bool ZERO, int PM, int TX, int TY>
cudaError_t launch_t(const float* ui, float* uo, const float* f, const float* ec, float* fc,
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
cudaError_t dispatch_t(const float* ui, float* uo, const float* f, const float* ec, float* fc,
                       FusedParams p, TileCfg cfg, cudaStream_t s) {
  const long long sms = 152;
  const int tx = cfg.tx ? cfg.tx : (p.nx >= 64 ? 64 : 32), ty = cfg.ty ? cfg.ty : 16;
  const long long cols = (long long)(p.nx / tx) * (p.ny / ty);
  int cz = 64;
  while (cz > 8 && cols * ((p.nz + cz - 1) / cz) < 2 * sms) cz /= 2;
  if (cfg.cz) cz = cfg.cz;
  p.cz = cz < p.nz ? cz : p.nz;
  if (ty == 32) {
    if (tx == 64) return launch_t<MODE, ZERO, PM, 64, 32>(ui, uo, f, ec, fc, p, s);
    return launch_t<MODE, ZERO, PM, 32, 32>(ui, uo, f, ec, fc, p, s);
  }
  if (tx == 64) return launch_t<MODE, ZERO, PM, 64, 16>(ui, uo, f, ec, fc, p, s);
  return launch_t<MODE, ZERO, PM, 32, 16>(ui, uo, f, ec, fc, p, s);
}

// Periodic axes of a rule: bit 0 x, 1 y, 2 z.
int periodic_mask(const Bc& bc) {
  int m = 0;
  for (int a = 0; a < 3; ++a)
    if (face_kind(bc, 2 * a) == BC_PERIODIC) m |= 1 << a;
  return m;
}

// The masks with kernels: none, the x-y slab, all.
bool mask_built(int pm) { return pm == 0 || pm == 3 || pm == 7; }

template <int MODE, bool ZERO>
cudaError_t dispatch(const float* ui, float* uo, const float* f, const float* ec, float* fc,
                     FusedParams p, const Bc& bc, TileCfg cfg, cudaStream_t s) {
  switch (periodic_mask(bc)) {
    case 7: return dispatch_t<MODE, ZERO, 7>(ui, uo, f, ec, fc, p, cfg, s);
    case 3: return dispatch_t<MODE, ZERO, 3>(ui, uo, f, ec, fc, p, cfg, s);
    case 0: return dispatch_t<MODE, ZERO, 0>(ui, uo, f, ec, fc, p, cfg, s);
    default: return cudaErrorInvalidValue;
  }
}

FusedParams params(Grid g, double h, const Bc& bc, double omega) {
  FusedParams p;
  p.nx = g.nx; p.ny = g.ny; p.nz = g.nz;
  float sg[6];
  for (int q = 0; q < 6; ++q) sg[q] = face_kind(bc, q) == BC_ZEROGRAD ? 1.f : -1.f;
  p.sx0 = sg[0]; p.sx1 = sg[1]; p.sy0 = sg[2]; p.sy1 = sg[3]; p.sz0 = sg[4]; p.sz1 = sg[5];
  p.cu = (float)(1.0 - omega);
  p.cs = (float)(omega / 6.0);
  p.cf = (float)(-omega * h * h / 6.0);
  p.inv_h2 = (float)(1.0 / (h * h));
  p.cz = 8;
  return p;
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
  // values); periodic axes none, x and y, or all
  bool hom = bc.kind != BC_OPEN && fused::mask_built(fused::periodic_mask(bc));
  if (bc.kind == BC_FIXED) hom = hom && bc.value == 0.0;
  if (bc.kind == BC_MIXED) hom = hom && bc.faces == nullptr;
  // widths the 64- or 32-wide tiles divide, rows in 16s, planes in chunks of 8;
  // element offsets of 32 bits
  return hom && g.nx >= 32 && g.ny >= 32 && g.nz >= 32 && g.nx % 32 == 0 && g.ny % 16 == 0 &&
         g.nz % 8 == 0 && (g.nx < 64 || g.nx % 64 == 0) && g.cells() < (1LL << 32);
}

bool fused_cfg_ok(Grid g, TileCfg cfg) {
  const bool tx_ok = cfg.tx == 0 || (cfg.tx == 32 && g.nx % 32 == 0) ||
                     (cfg.tx == 64 && g.nx % 64 == 0);
  const bool cz_ok = cfg.cz == 0 || (cfg.cz >= 8 && cfg.cz % 8 == 0 && cfg.cz <= 1024);
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
