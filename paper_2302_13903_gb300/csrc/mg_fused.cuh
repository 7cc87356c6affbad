// mg_fused.cuh -- the fused z-marching FP32 V-cycle-leg programs (device code
// shared by the standalone kernels of mg_fused.cu and the batched solver).
//
// One kernel per leg of Algorithm 1 on an FP32 level with a homogeneous rule
// (periodic, zero fixed or zero gradient -- the rules of the correction
// equation):
//   down:  [u = 0 or u_in] -> SMOOTH (red, then black) -> d = f - L u ->
//          f_{l-1} = I_l^{l-1} d                          (steps 1-3)
//   up:    u_in + I_{l-1}^l e_{l-1} -> SMOOTH             (steps 5-7)
//   plain: one SMOOTH step (extra steps of V(2,.) / V(.,2) cycles)
//
// A CTA owns a TX x TY tile of (x, y) columns and marches along z through a
// chunk of planes.  Each thread owns a 4 x 2 patch (four consecutive x cells
// of an even row and of the odd row after it) and keeps its patch of the last
// few planes in registers.  Per plane step the pipeline is:
//   copy plane q+2 of u and plane q+1 of f into shared memory (cp.async),
//   [A] load plane q of u (up leg: add the prolonged correction),
//   [B] red half-step on plane q-1, [C] black half-step on plane q-2 (down
//   leg: with the black cells' defects), write plane q-2,
//   [D] down leg: the red cells' defect of plane q-3 and, every second plane,
//   the 2x2x2 restriction.
// A half-step needs of its own plane only the other colour's cells in the
// neighbouring patches; they come from colour-pair planes in shared memory
// (each thread's two cells of one colour per row, as a float2), written when
// that colour was last updated: the black cells of u at [A], the red cells at
// [B], the final black cells at [C].  One __syncthreads separates plane steps.
// Because the patch spans an even and an odd row and the z-loop is unrolled by
// four, the colour of every cell is known at compile time; the two cells of
// one colour in a row are updated together with packed FP32x2 arithmetic.
//
// Kernels read u_in and write u_out (different buffers): neighbouring tiles
// recompute this tile's border cells as their halo (a ring of 2 cells around
// the smoothed region, 3 when the defect follows; 4 in x to keep 16-byte
// alignment, 4 in y to keep row pairs) and must see the values from before
// the step.
//
// Boundaries: along a periodic axis (bit a of the compile-time mask PM) halo
// cells are real cells at wrapped indices and are updated like any other;
// across a non-periodic face a neighbour outside the level is s * (the cell
// itself), with the face's own s = -1 (zero fixed) or +1 (zero gradient) --
// the ghost value of Sec. 2.3.6 at the moment it is read.  PM = 7 is the
// periodic rule, 0 the zero-fixed / zero-gradient ones (one s on every face
// or one per face), 3 a slab periodic in x and y.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "mg_internal.h"

namespace mg {
namespace fused {

struct FusedParams {
  int nx, ny, nz;
  // ghost sign of each non-periodic face: -1 zero fixed, +1 zero gradient
  float sx0, sx1, sy0, sy1, sz0, sz1;
  float cu, cs, cf;  // SOR: u <- cu u + cs sum_nb + cf f
  float inv_h2;
  int cz;            // planes per CTA (multiple of 4, or nz)
};

// The kernels' constants for level g (spacing h, SOR factor omega, face
// rules bc); cz is set by the launch.
inline FusedParams params(Grid g, double h, const Bc& bc, double omega) {
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

// Planes per CTA: cz_cfg when nonzero, else the largest of 64, 32, 16, 8, 4
// that still gives two CTAs per SM on tiles of tx x ty; at most nz.
inline int chunk_planes(const FusedParams& p, int tx, int ty, int cz_cfg) {
  const long long sms = sm_count();
  const long long cols = (long long)(p.nx / tx) * (p.ny / ty);
  int cz = 64;
  while (cz > 4 && cols * ((p.nz + cz - 1) / cz) < 2 * sms) cz /= 2;
  if (cz_cfg) cz = cz_cfg;
  return cz < p.nz ? cz : p.nz;
}

enum Mode : int { kPlain = 0, kDown = 1, kUp = 2 };

__device__ __forceinline__ int wrap(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// Periodic axes of a mask PM.
template <int PM>
struct Per {
  static constexpr bool X = (PM & 1) != 0, Y = (PM & 2) != 0, Z = (PM & 4) != 0;
};

// ---------------------------------------------------------------------------
// Packed helpers.  A row of four cells is kept as e = (c0, c2), o = (c1, c3).

struct Row {
  float2 e, o;
};
struct Patch {
  Row a, b;  // a: even row, b: odd row
};

// A float4 of a level (or of its copy in a shared plane) holds four
// consecutive cells c0..c3; a Row keeps them as the colour pairs (c0, c2) and
// (c1, c3).
__device__ __forceinline__ Row unpack(const float4 v) {
  return Row{make_float2(v.x, v.z), make_float2(v.y, v.w)};
}
__device__ __forceinline__ float4 pack(const Row r) { return make_float4(r.e.x, r.o.x, r.e.y, r.o.y); }
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ Patch zero_patch() {
  const float2 z = make_float2(0.f, 0.f);
  return Patch{Row{z, z}, Row{z, z}};
}

// u <- cu u + cs (xm + xp + ym + yp + zm + zp) + cf f on two cells at once;
// `sum` receives the neighbour sum.
__device__ __forceinline__ float2 sor2(float2 self, float2 xm, float2 xp, float2 ym, float2 yp,
                                       float2 zm, float2 zp, float2 f, const FusedParams& p,
                                       float2& sum) {
  sum = add2(add2(add2(xm, xp), add2(ym, yp)), add2(zm, zp));
  float2 t = __fmul2_rn(make_float2(p.cf, p.cf), f);
  t = __ffma2_rn(make_float2(p.cu, p.cu), self, t);
  return __ffma2_rn(make_float2(p.cs, p.cs), sum, t);
}

// d = f - (sum - 6 u) / h^2 from a neighbour sum.
__device__ __forceinline__ float2 defect_from_sum(float2 self, float2 sum, float2 f,
                                                  const FusedParams& p) {
  const float2 lap = __ffma2_rn(make_float2(-6.f, -6.f), self, sum);
  return __ffma2_rn(make_float2(-p.inv_h2, -p.inv_h2), lap, f);
}

// d = f - (sum_nb - 6 u) / h^2 on two cells at once.
__device__ __forceinline__ float2 defect2(float2 self, float2 xm, float2 xp, float2 ym, float2 yp,
                                          float2 zm, float2 zp, float2 f, const FusedParams& p) {
  const float2 sum = add2(add2(add2(xm, xp), add2(ym, yp)), add2(zm, zp));
  const float2 lap = __ffma2_rn(make_float2(-6.f, -6.f), self, sum);
  return __ffma2_rn(make_float2(-p.inv_h2, -p.inv_h2), lap, f);
}

// Boundary flags of a thread's patch at non-periodic faces.
struct Flags {
  bool xlo, xhi, ylo, yhi;
};

__device__ __forceinline__ float2 sub_if(bool flag, float s, float2 self, float2 v) {
  return flag ? make_float2(s * self.x, s * self.y) : v;
}

template <bool E>
__device__ __forceinline__ float2 part(const Row& r) {
  return E ? r.e : r.o;
}
template <bool E>
__device__ __forceinline__ void set_part(Row& r, float2 v) {
  if (E) r.e = v;
  else r.o = v;
}

// x neighbours of one row's e cells (E) or o cells (!E); `sidev` is the
// neighbouring thread's cell next to them: its c3 on the left for e, its c0 on
// the right for o.
template <int PM, bool E>
__device__ __forceinline__ void x_nb(const Row& r, float sidev, float2 self, float2& xm,
                                     float2& xp, const FusedParams& p, const Flags& fl) {
  if (E) {
    xm = f2(sidev, r.o.x);
    xp = r.o;
    if (!Per<PM>::X && fl.xlo) xm.x = p.sx0 * self.x;
  } else {
    xm = r.e;
    xp = f2(r.e.y, sidev);
    if (!Per<PM>::X && fl.xhi) xp.y = p.sx1 * self.y;
  }
}

// The y / z neighbours of a row's cells with the ghosts of non-periodic faces
// applied (yout: the neighbours in the adjacent row pair, on the low side for
// row a, ROWB = false, on the high side for row b).
template <int PM, bool ROWB>
__device__ __forceinline__ void yz_ghosts(float2 self, float2& yout, float2& zmv, float2& zpv,
                                          const FusedParams& p, const Flags& fl, bool zlo,
                                          bool zhi) {
  if (!Per<PM>::Y) yout = sub_if(ROWB ? fl.yhi : fl.ylo, ROWB ? p.sy1 : p.sy0, self, yout);
  if (!Per<PM>::Z) {
    zmv = sub_if(zlo, p.sz0, self, zmv);
    zpv = sub_if(zhi, p.sz1, self, zpv);
  }
}

// SOR update of one row's E cells.  yout: their neighbours in the adjacent
// row pair (the row above for row a, ROWB = false; below for row b); `other`:
// the patch's other row; sidev as in x_nb.  DEF: *d receives the updated
// cells' defects from the update's own neighbour sum (plus, for the
// non-periodic rules, the change of their ghost neighbours s u).
template <int PM, bool E, bool ROWB, bool DEF>
__device__ __forceinline__ void sor_row(Row& r, const Row& other, float2 yout, float sidev,
                                        const Row& rzm, const Row& rzp, const Row& rf,
                                        const FusedParams& p, const Flags& fl, bool zlo, bool zhi,
                                        float2* d) {
  const float2 self = part<E>(r);
  float2 xm, xp;
  x_nb<PM, E>(r, sidev, self, xm, xp, p, fl);
  const float2 yin = part<E>(other);
  float2 zmv = part<E>(rzm), zpv = part<E>(rzp);
  yz_ghosts<PM, ROWB>(self, yout, zmv, zpv, p, fl, zlo, zhi);
  float2 sum;
  const float2 un = ROWB ? sor2(self, xm, xp, yin, yout, zmv, zpv, part<E>(rf), p, sum)
                         : sor2(self, xm, xp, yout, yin, zmv, zpv, part<E>(rf), p, sum);
  set_part<E>(r, un);
  if (DEF) {
    float2 dd = defect_from_sum(un, sum, part<E>(rf), p);
    if (PM != 7) {
      // each ghost neighbour s u moved with u: its share of the finished
      // sweep's sum is s (un - self) more than the update used
      float sg = 0.f;
      if (!Per<PM>::Y && (ROWB ? fl.yhi : fl.ylo)) sg += ROWB ? p.sy1 : p.sy0;
      if (!Per<PM>::Z && zlo) sg += p.sz0;
      if (!Per<PM>::Z && zhi) sg += p.sz1;
      const float sgx = sg + ((!Per<PM>::X && E && fl.xlo) ? p.sx0 : 0.f);
      const float sgy = sg + ((!Per<PM>::X && !E && fl.xhi) ? p.sx1 : 0.f);
      const float2 kng = make_float2(-p.inv_h2 * sgx, -p.inv_h2 * sgy);
      dd = __ffma2_rn(kng, add2(un, make_float2(-self.x, -self.y)), dd);
    }
    *d = dd;
  }
}

// Defect of one row's E cells (arguments as in sor_row).
template <int PM, bool E, bool ROWB>
__device__ __forceinline__ float2 defect_row(const Row& r, const Row& other, float2 yout,
                                             float sidev, const Row& rzm, const Row& rzp,
                                             const Row& rf, const FusedParams& p,
                                             const Flags& fl, bool zlo, bool zhi) {
  const float2 self = part<E>(r);
  float2 xm, xp;
  x_nb<PM, E>(r, sidev, self, xm, xp, p, fl);
  const float2 yin = part<E>(other);
  float2 zmv = part<E>(rzm), zpv = part<E>(rzp);
  yz_ghosts<PM, ROWB>(self, yout, zmv, zpv, p, fl, zlo, zhi);
  return ROWB ? defect2(self, xm, xp, yin, yout, zmv, zpv, part<E>(rf), p)
              : defect2(self, xm, xp, yout, yin, zmv, zpv, part<E>(rf), p);
}

// A pair plane holds, for every row of a plane and every thread, the two cells
// of that row's patch of one colour (the colour whose values a later
// half-step needs as neighbours) as a float2; rows are RS2 float2 apart.  A
// cell's y neighbours in the adjacent rows have the same x, so the pair of the
// adjacent row is exactly the yout of sor_row; the x neighbour across a patch
// edge is the pair's .y (left thread, its c3) or .x (right thread, its c0).
__device__ __forceinline__ float side_of(const float2* SP, int idx, int offL, int offR, bool e) {
  const float* SF = reinterpret_cast<const float*>(SP);
  return e ? SF[2 * (idx + offL) + 1] : SF[2 * (idx + offR)];
}

// One SOR half-step on the patch: row a updates its e cells if AE (else o),
// row b the cells of the other parity (the same colour one row down), with
// the other colour's cells of this plane in the pair plane SP (offsets in
// float2); zm, zp: the patch in the planes below / above.  DEF: dsum receives
// the updated cells' defects summed over both rows (sor_row).
template <int PM, bool AE, bool DEF = false>
__device__ __forceinline__ void sor_pairs(Patch& u, const float2* __restrict__ SP, int pa, int pb,
                                          int offL, int offR, int offU, int offD, const Patch& zm,
                                          const Patch& zp, const Patch& f, const FusedParams& p,
                                          const Flags& fl, bool zlo, bool zhi,
                                          float2* dsum = nullptr) {
  constexpr bool BE = !AE;
  float2 da, db;
  sor_row<PM, AE, false, DEF>(u.a, u.b, SP[pa + offU], side_of(SP, pa, offL, offR, AE), zm.a,
                              zp.a, f.a, p, fl, zlo, zhi, &da);
  sor_row<PM, BE, true, DEF>(u.b, u.a, SP[pb + offD], side_of(SP, pb, offL, offR, BE), zm.b,
                             zp.b, f.b, p, fl, zlo, zhi, &db);
  if (DEF) *dsum = add2(da, db);
}

// Defect of the red cells of a patch (row a's e cells if AE, row b's of the
// other parity) from a pair plane of the final black cells, summed over both
// rows.
template <int PM, bool AE>
__device__ __forceinline__ float2 defect_red(const Patch& u, const float2* __restrict__ SP, int pa,
                                             int pb, int RS2, const Patch& zm, const Patch& zp,
                                             const Patch& f, const FusedParams& p,
                                             const Flags& fl, bool zlo, bool zhi) {
  const float2 da = defect_row<PM, AE, false>(u.a, u.b, SP[pa - RS2], side_of(SP, pa, -1, 1, AE),
                                              zm.a, zp.a, f.a, p, fl, zlo, zhi);
  const float2 db = defect_row<PM, !AE, true>(u.b, u.a, SP[pb + RS2], side_of(SP, pb, -1, 1, !AE),
                                              zm.b, zp.b, f.b, p, fl, zlo, zhi);
  return add2(da, db);
}

// Asynchronous 16-byte global -> shared copy; src_bytes = 0 fills zeros.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Tensor-memory-accelerator copies of whole plane tiles (one thread issues,
// an mbarrier in shared memory counts the bytes that land).
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of the barrier; gives up after 2^22 tries (each
// suspends the thread for at most a few microseconds), raising *err and
// returning false, so that a copy that never lands cannot hang the GPU.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int* err) {
  for (int k = 0; k < (1 << 22); ++k)
    if (mbar_try_wait(bar, parity)) return true;
  if (err) *reinterpret_cast<volatile int*>(err) = 1;  // a flag: a plain store suffices
  return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_addr(dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void tma_prefetch_3d(const void* tmap, int x, int y, int z) {
  asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];\n" ::"l"(tmap),
               "r"(x), "r"(y), "r"(z)
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// (x, y) part of the trilinear prolongation of one coarse plane at a patch:
// rows gyA (even: coarse rows Y-1, Y) and gyA+1 (odd: Y, Y+1), Y = gyA/2;
// four fine x cells from coarse x X0-1 .. X0+2, X0 = gx4/2.  The up leg
// stages the coarse cells under its tile in shared memory, one plane at a
// time: CX columns from x0/2 - 4 and CY rows from y0/2 - HY/2 - 1, wrapped
// along periodic axes, zero-filled outside the level along the others.  A
// thread's 3 x 4 block then starts at tile row tp, column 1 + 2 tr; along a
// non-periodic axis its indices are clamped to the level's edge cells and
// carry that face's ghost sign s (CoarseIdx).  Patches outside the level read
// clamped indices; their values are unused.
struct Coarse12 {
  float c[3][4];
};

struct CoarseIdx {
  int col[4];  // tile column
  int row[3];  // tile row
  float sx[4], sy[3];  // ghost signs (1 inside)
};

// Along a periodic axis the tile index is the plain one (the staged tile is
// wrapped) and the sign 1.
template <int PM>
__device__ __forceinline__ CoarseIdx coarse_idx(const FusedParams& p, int gx4, int gyA, int cx0,
                                                int cy0) {
  const int cnx = p.nx >> 1, cny = p.ny >> 1;
  const int X0 = gx4 >> 1, Y = gyA >> 1;
  CoarseIdx ci;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int Xc = X0 - 1 + a;
    ci.sx[a] = Per<PM>::X ? 1.f : (Xc < 0 ? p.sx0 : (Xc >= cnx ? p.sx1 : 1.f));
    ci.col[a] = (Per<PM>::X ? Xc : (Xc < 0 ? 0 : (Xc >= cnx ? cnx - 1 : Xc))) - cx0;
  }
#pragma unroll
  for (int yy = 0; yy < 3; ++yy) {
    const int Yc = Y - 1 + yy;
    ci.sy[yy] = Per<PM>::Y ? 1.f : (Yc < 0 ? p.sy0 : (Yc >= cny ? p.sy1 : 1.f));
    ci.row[yy] = (Per<PM>::Y ? Yc : (Yc < 0 ? 0 : (Yc >= cny ? cny - 1 : Yc))) - cy0;
  }
  return ci;
}

// The 3 x 4 coarse values of a staged plane S (sz: the ghost sign of a plane
// outside a level with z walls, else 1), ghosts applied.  C0: the tile column
// of thread tr = 0's first coarse cell.
template <int PM, int CX, int C0 = 1>
__device__ __forceinline__ Coarse12 xy_read(const float* S, const CoarseIdx& ci, int tr, int tp,
                                            float sz) {
  Coarse12 r;
  if (Per<PM>::X && Per<PM>::Y) {
    const float* b = S + tp * CX + C0 + 2 * tr;
#pragma unroll
    for (int yy = 0; yy < 3; ++yy)
#pragma unroll
      for (int a = 0; a < 4; ++a) r.c[yy][a] = Per<PM>::Z ? b[yy * CX + a] : sz * b[yy * CX + a];
  } else {
#pragma unroll
    for (int yy = 0; yy < 3; ++yy)
#pragma unroll
      for (int a = 0; a < 4; ++a)
        r.c[yy][a] = sz * (ci.sy[yy] * (ci.sx[a] * S[ci.row[yy] * CX + ci.col[a]]));
  }
  return r;
}

__device__ __forceinline__ Patch xy_combine(const Coarse12& r) {
  float xr[3][4];
#pragma unroll
  for (int yy = 0; yy < 3; ++yy) {
    const float* c = r.c[yy];
    xr[yy][0] = 0.25f * c[0] + 0.75f * c[1];
    xr[yy][1] = 0.75f * c[1] + 0.25f * c[2];
    xr[yy][2] = 0.25f * c[1] + 0.75f * c[2];
    xr[yy][3] = 0.75f * c[2] + 0.25f * c[3];
  }
  Patch P;
  P.a.e = f2(0.25f * xr[0][0] + 0.75f * xr[1][0], 0.25f * xr[0][2] + 0.75f * xr[1][2]);
  P.a.o = f2(0.25f * xr[0][1] + 0.75f * xr[1][1], 0.25f * xr[0][3] + 0.75f * xr[1][3]);
  P.b.e = f2(0.75f * xr[1][0] + 0.25f * xr[2][0], 0.75f * xr[1][2] + 0.25f * xr[2][2]);
  P.b.o = f2(0.75f * xr[1][1] + 0.25f * xr[2][1], 0.75f * xr[1][3] + 0.25f * xr[2][3]);
  return P;
}

// Row stride of a shared plane, in float4: the smallest RS >= RT with
// 2 RS = RT (mod 8).  Thread t = tp RT + tr reads float4 2 tp RS + tr (+ a
// constant), which is then t plus a multiple of 8 -- eight consecutive
// threads hit eight different 16-byte bank groups (no bank conflicts).
constexpr int row_stride(int rt) {
  int r = rt;
  while ((2 * r - rt) % 8 != 0) ++r;
  return r;
}

// Row stride of a pair plane, in float2: the smallest RS2 >= RT with
// 2 RS2 = RT (mod 16), so that the 16 threads of a half-warp, reading float2
// 2 tp RS2 + tr (+ a constant), hit 16 different 8-byte bank pairs.
constexpr int pair_stride(int rt) {
  int r = rt;
  while ((2 * r - rt) % 16 != 0) ++r;
  return r;
}

// HYO > 0 overrides the rows of halo (so that every mode can share one block
// size in the batched solver); PAD = false keeps rows unpadded (RS = RT), for
// the batched solver, whose other phases want the shared memory as L1.
template <int MODE, int TX, int TY, int HYO = 0, bool PAD = true>
struct Shape {
  static constexpr int HZ = (MODE == kDown) ? 3 : 2;  // planes of halo in z
  static constexpr int HY = HYO > 0 ? HYO : ((MODE == kDown) ? 4 : 2);  // rows of halo in y (even)
  static constexpr int RT = (TX + 8) / 4;              // float4 columns per row
  static constexpr int RS = PAD ? row_stride(RT) : RT;  // float4 between rows in shared memory
  static constexpr int RR = TY + 2 * HY;               // rows
  static constexpr int RP = RR / 2;                    // row pairs
  static constexpr int NT = RT * RP;                   // threads
  static constexpr int PL = RS * RR;                   // float4 per shared plane
  static constexpr int RS2 = pair_stride(RT);          // float2 between rows of a pair plane
  static constexpr int PL2 = RS2 * RR;                 // float2 per pair plane
  static constexpr int NU = 4, NF = 4, NRED = 2, NFIN = (MODE == kDown) ? 2 : 0;
  static constexpr int CX = TX / 2 + 8;  // coarse tile columns (up leg)
  static constexpr int CY = RP + 2;      // coarse tile rows
  static constexpr int NC = (MODE == kUp) ? 2 * CX * CY : 0;  // floats of the two coarse slots
  static constexpr int NUB = 2;  // pair planes of the u planes' black cells
  static constexpr size_t SMEM =
      (size_t)(NU + NF) * PL * 16 + (size_t)(NRED + NUB + NFIN) * PL2 * 8 + (size_t)NC * 4;
  // with tensor copies every ring slot starts on a 128-byte boundary: slots
  // PLS float4 apart, and SMEM_TMA bytes in all
  static constexpr int PLS = (PL + 7) / 8 * 8;
  static constexpr size_t SMEM_TMA = SMEM + (size_t)(NU + NF) * (PLS - PL) * 16;
};

// The program of one CTA on one tile (bx, by) and z-chunk bz; `smem` holds
// Shape::SMEM bytes.  NTB: the CTA's size when it is larger than Shape::NT
// (0: exactly NT); threads tid >= Shape::NT of a larger CTA take part in the
// barriers only.  Element offsets are 32-bit: levels have fewer than 2^32
// cells (fused_ok).
// TMA: tiles whose window lies inside the level (and, along a periodic axis,
// needs no wrap) take their planes of u and f by one tensor copy each, issued
// by one thread, from the tensor maps tmu and tmf (boxes of 4 RS columns by
// RR rows by one plane: a ring slot); the others by cp.async.  A copy that
// does not land in time raises *err, and the CTA stops its z-march.
template <int MODE, bool ZERO, int PM, int TX, int TY, int HYO = 0, bool PAD = true,
          int NTB = 0, bool TMA = false, int PF = 0>
__device__ __forceinline__ void fused_tile(const float* u_in, float* u_out, const float* f,
                                           const float* ec, float* fc,
                                           const FusedParams& p, int bx, int by, int bz,
                                           float4* smem, const void* tmu = nullptr,
                                           const void* tmf = nullptr, int* err = nullptr) {
  using S_ = Shape<MODE, TX, TY, HYO, PAD>;
  constexpr int HZ = S_::HZ, HY = S_::HY, RT = S_::RT, RS = S_::RS, RP = S_::RP, PL = S_::PL;
  constexpr int PLS = TMA ? S_::PLS : PL;  // float4 between ring slots
  float4* s_u = smem;                     // [4][PLS] planes of u (async copies)
  float4* s_f = s_u + S_::NU * PLS;       // [4][PLS] planes of f (async copies)
  // [2][PL2] pair planes of the red cells after the red half-step
  float2* s_red = reinterpret_cast<float2*>(s_f + S_::NF * PLS);
  // [2][PL2] pair planes of the black cells of u (with the correction, on the
  // up leg) as loaded: the red half-step's neighbours
  float2* s_ub = s_red + S_::NRED * S_::PL2;
  // [2][PL2] pair planes of the final black cells (down leg): the red cells'
  // defect neighbours
  float2* s_finp = s_ub + S_::NUB * S_::PL2;
  float* s_c = reinterpret_cast<float*>(s_finp + S_::NFIN * S_::PL2);  // [2][CY][CX] coarse (up)

  constexpr bool SPARE = NTB > S_::NT;  // the CTA has threads without a patch
  const int tid = (!SPARE || threadIdx.x < S_::NT) ? threadIdx.x : 0;  // spare: mirror thread 0
  const bool act = !SPARE || threadIdx.x < S_::NT;
  const int tr = tid % RT, tp = tid / RT;
  const int x0 = bx * TX, y0 = by * TY;
  const int z0 = bz * p.cz;
  const int z1 = min(z0 + p.cz, p.nz);
  const int gx4 = x0 - 4 + 4 * tr;   // x of the patch's first cell (may be outside)
  const int gyA = y0 - HY + 2 * tp;  // even row of the patch (may be outside)
  constexpr bool PX = Per<PM>::X, PY = Per<PM>::Y, PZ = Per<PM>::Z;
  const int gx4w = PX ? wrap(gx4, p.nx) : gx4;
  const int gyAw = PY ? wrap(gyA, p.ny) : gyA;
  // the patch holds real cells
  const bool col_ok = (PX || (gx4 >= 0 && gx4 < p.nx)) && (PY || (gyA >= 0 && gyA < p.ny));
  Flags fl;
  fl.xlo = !PX && gx4 == 0;
  fl.xhi = !PX && gx4 + 3 == p.nx - 1;
  fl.ylo = !PY && gyA == 0;
  fl.yhi = !PY && gyA + 1 == p.ny - 1;
  const bool out = tr >= 1 && tr <= TX / 4 && tp >= HY / 2 && tp < HY / 2 + TY / 2;
  const unsigned plane = (unsigned)p.nx * (unsigned)p.ny;
  const unsigned offA = col_ok ? (unsigned)gyAw * p.nx + gx4w : 0u;  // row a; row b is nx further
  const int ia = (2 * tp) * RS + tr, ib = ia + RS;  // shared indices of rows a, b
  constexpr int RS2 = S_::RS2, PL2 = S_::PL2;
  const int pa = (2 * tp) * RS2 + tr, pb = pa + RS2;  // their pair-plane indices
  const int offU2 = tp > 0 ? -RS2 : 0, offD2 = tp < RP - 1 ? RS2 : 0;
  const int offL = tr > 0 ? -1 : 0, offR = tr < RT - 1 ? 1 : 0;
  const int q_first = z0 - HZ, q_last = z1 - 1 + HZ;

  // TMA tiles: their window [x0 - 4, x0 + TX + 4) x [y0 - HY, y0 + TY + HY)
  // inside the level (the box's extra padding columns may leave it: they are
  // zero-filled and never read); mbarrier b counts the copies of plane b mod 4
  __shared__ unsigned long long tma_bar[TMA ? 4 : 1];
  bool stop = false;  // a tensor copy did not land in time (the same in every thread)
  int q_stop = 0;     // the plane whose copies were late
  const bool tma_tile = TMA && x0 - 4 >= 0 && x0 + TX + 4 <= p.nx && y0 - HY >= 0 &&
                        y0 + TY + HY <= p.ny;
  if (TMA && tma_tile) {
    if (threadIdx.x == 0) {
      for (int b = 0; b < 4; ++b) mbar_init(&tma_bar[b], 1);
      fence_proxy_async();
    }
    __syncthreads();
  }
  // Copies of plane qu of u into ring slot SU and plane qu - 1 of f into
  // slot SF (the slots are compile-time: qu mod 4 is fixed by the step).
  auto issue = [&](auto SUc, auto SFc, int qu) {
    constexpr int SU = decltype(SUc)::value, SF = decltype(SFc)::value;
    if (TMA && PF > 0 && threadIdx.x == 0 && qu + PF <= q_last) {
      const int qp = qu + PF;
      const int zp = PZ ? wrap(qp, p.nz) : qp, zpf = PZ ? wrap(qp - 1, p.nz) : qp - 1;
      const int px = max(x0 - 4, 0), py = max(y0 - HY, 0);
      if (!ZERO) tma_prefetch_3d(tmu, px, py, zp);
      tma_prefetch_3d(tmf, px, py, zpf);
    }
    if (TMA && tma_tile) {
      if (threadIdx.x == 0 && qu <= q_last) {
        unsigned long long* bar = &tma_bar[SU];
        const int qf = qu - 1;
        const int zu = PZ ? wrap(qu, p.nz) : qu, zf = PZ ? wrap(qf, p.nz) : qf;
        fence_proxy_async();  // earlier reads of the slots come before the copies
        mbar_expect_tx(bar, (ZERO ? 1u : 2u) * (unsigned)(PL * 16));
        if (!ZERO) tma_load_3d(&s_u[SU * PLS], tmu, x0 - 4, y0 - HY, zu, bar);
        tma_load_3d(&s_f[SF * PLS], tmf, x0 - 4, y0 - HY, zf, bar);
      }
      return;
    }
    if (act && qu <= q_last) {
      if (!ZERO) {
        const bool in = col_ok && (PZ || (qu >= 0 && qu < p.nz));
        const unsigned o = (unsigned)(PZ ? wrap(qu, p.nz) : (in ? qu : 0)) * plane + offA;
        float4* d = &s_u[SU * PLS];
        cp_async16(&d[ia], u_in + o, in ? 16 : 0);
        cp_async16(&d[ib], u_in + (o + p.nx), in ? 16 : 0);
      }
      const int qf = qu - 1;
      const bool inf = col_ok && (PZ || (qf >= 0 && qf < p.nz));
      const unsigned o = (unsigned)(PZ ? wrap(qf, p.nz) : (inf ? qf : 0)) * plane + offA;
      float4* d = &s_f[SF * PLS];
      cp_async16(&d[ia], f + o, inf ? 16 : 0);
      cp_async16(&d[ib], f + (o + p.nx), inf ? 16 : 0);
    }
  };

  // Up leg: copy coarse plane Kc (any index from -2 to cnz + 1) into slot SL.
  const int cx0 = (x0 >> 1) - 4, cy0 = (y0 >> 1) - HY / 2 - 1;
  auto copy_coarse = [&](auto SLc, int Kc) {
    constexpr int SL = decltype(SLc)::value, CW = S_::CX / 4;  // float4 per tile row
    const int cnx = p.nx >> 1, cny = p.ny >> 1, cnz = p.nz >> 1;
    const int t = threadIdx.x;
    if (t < CW * S_::CY) {
      const int i = t / CW, j = t - i * CW;
      int X = cx0 + 4 * j, Y = cy0 + i, K = Kc;
      bool in = true;
      if (PX) X = wrap(X, cnx);
      else in = X >= 0 && X < cnx;
      if (PY) Y = wrap(Y, cny);
      else in = in && Y >= 0 && Y < cny;
      if (PZ) K = wrap(K, cnz);
      else K = K < 0 ? 0 : (K >= cnz ? cnz - 1 : K);
      if (!in) { X = 0; Y = 0; }
      cp_async16(s_c + SL * S_::CX * S_::CY + i * S_::CX + 4 * j,
                 ec + (((unsigned)K * cny + Y) * cnx + X), in ? 16 : 0);
    }
  };
  auto plane_sign = [&](int Kc) {
    return PZ ? 1.f : (Kc < 0 ? p.sz0 : (Kc >= (p.nz >> 1) ? p.sz1 : 1.f));
  };

  Patch r1 = zero_patch(), r2 = r1, r3 = r1, r4 = r1, f2p = r1, f3p = r1;
  // down leg: black defects come from the black half-step (sor_pairs DEF), red
  // ones from the defect pass; accz holds the coarse planes' sums by parity
  constexpr bool SPLIT = MODE == kDown;
  float2 accz[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  // Up leg: the (x, y)-interpolated coarse planes K-1, K, K+1 around fine
  // planes 2K, 2K+1 live in W[0] (even K) and W[1] (odd K); fine plane 2K
  // takes 3/4 of plane K and 1/4 of plane K-1, fine plane 2K+1 3/4 of K and
  // 1/4 of K+1.  Coarse plane K+1 is combined at fine plane 2K+1 from shared
  // slot (K+1) mod 2, whose copy was issued two steps earlier; plane K+2 is
  // then copied into slot K mod 2.
  Patch W[2];
  CoarseIdx ci;
  if (MODE == kUp) {
    if (!(PX && PY)) ci = coarse_idx<PM>(p, gx4, gyA, cx0, cy0);
    // q_first = z0 - 2 with z0 a multiple of 4: K0 = q_first / 2 is odd
    const int K0 = q_first >> 1;
    copy_coarse(std::integral_constant<int, 0>{}, K0 - 1);
    copy_coarse(std::integral_constant<int, 1>{}, K0);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    W[0] = xy_combine(xy_read<PM, S_::CX>(s_c, ci, tr, tp, plane_sign(K0 - 1)));
    W[1] = xy_combine(xy_read<PM, S_::CX>(s_c + S_::CX * S_::CY, ci, tr, tp, plane_sign(K0)));
    __syncthreads();
    copy_coarse(std::integral_constant<int, 0>{}, K0 + 1);  // committed with plane q_first
  }

  // One plane step.  J = (q - q_first) mod 4 fixes the ring slots and the
  // colours at compile time: q_first = z0 - HZ with z0 a multiple of 4.
  auto step = [&](auto Jc, int q) {
    constexpr int J = decltype(Jc)::value;
    constexpr int QP = ((J - HZ) % 4 + 4) % 4;  // q mod 4
    constexpr int SL_U = QP, SL_FM1 = (QP + 3) % 4;
    constexpr int ZP_RED = (QP + 3) % 2;  // parity of plane q-1
    constexpr int ZP_BLK = (QP + 2) % 2;  // parity of plane q-2
    constexpr int ZP_DEF = (QP + 1) % 2;  // parity of plane q-3
    if (TMA && tma_tile) {
      // plane q's copies; a wait that ran out stops the whole CTA (uniformly)
      const bool late = !mbar_wait(&tma_bar[QP], (unsigned)(((q - q_first) >> 2) & 1), err);
      if (MODE == kUp) cp_async_wait<1>();  // and this thread's copies of the coarse plane
      if (__syncthreads_or(late)) {
        stop = true;
        q_stop = q;
        return;
      }
    } else {
      cp_async_wait<1>();  // this thread's copies of plane q have landed
      __syncthreads();     // ... and everyone's; the previous step is finished
    }
    issue(std::integral_constant<int, (QP + 2) % 4>{}, std::integral_constant<int, (QP + 1) % 4>{},
          q + 2);
    if (MODE == kUp && (QP & 1) && q + 2 <= q_last)  // q = 2K+1: plane K+2 into slot K mod 2
      copy_coarse(std::integral_constant<int, (QP >> 1) & 1>{}, (q >> 1) + 2);
    cp_async_commit();
    // [A] plane q of u (old values), plus the prolonged correction (up leg)
    Patch r0 = zero_patch();
    if (!ZERO) {
      r0.a = unpack(s_u[SL_U * PLS + ia]);
      r0.b = unpack(s_u[SL_U * PLS + ib]);
    }
    if (MODE == kUp) {
      constexpr int KP = (QP >> 1) & 1;  // parity of K = floor(q / 2)
      const int K = q >> 1;
      if (QP & 1)
        W[1 - KP] = xy_combine(xy_read<PM, S_::CX>(s_c + (1 - KP) * S_::CX * S_::CY, ci, tr, tp,
                                                    plane_sign(K + 1)));
      if (col_ok && (PZ || (q >= 0 && q < p.nz))) {
        const float2 w0 = make_float2(0.75f, 0.75f), w1 = make_float2(0.25f, 0.25f);
        const Patch& PK = W[KP];
        const Patch& PN = W[1 - KP];
        r0.a.e = __ffma2_rn(w1, PN.a.e, __ffma2_rn(w0, PK.a.e, r0.a.e));
        r0.a.o = __ffma2_rn(w1, PN.a.o, __ffma2_rn(w0, PK.a.o, r0.a.o));
        r0.b.e = __ffma2_rn(w1, PN.b.e, __ffma2_rn(w0, PK.b.e, r0.b.e));
        r0.b.o = __ffma2_rn(w1, PN.b.o, __ffma2_rn(w0, PK.b.o, r0.b.o));
      }
    }
    if (!ZERO && act) {  // black cells of plane q: row a's o cells on an even plane, row b's e
      s_ub[(QP & 1) * PL2 + pa] = part<(QP & 1) != 0>(r0.a);
      s_ub[(QP & 1) * PL2 + pb] = part<(QP & 1) == 0>(r0.b);
    }
    Patch f1;
    f1.a = unpack(s_f[SL_FM1 * PLS + ia]);
    f1.b = unpack(s_f[SL_FM1 * PLS + ib]);
    // [B] red half-step on plane q-1: the red cells of the even row are its
    // e cells when the plane is even
    {
      const int pz = q - 1;
      const bool zlo = !PZ && pz == 0, zhi = !PZ && pz == p.nz - 1;
      if (q > q_first) {
        if (ZERO) {
          // every neighbour of a red cell is still 0
          const float2 cf2 = make_float2(p.cf, p.cf);
          if (ZP_RED == 0) {
            r1.a.e = __fmul2_rn(cf2, f1.a.e);
            r1.b.o = __fmul2_rn(cf2, f1.b.o);
          } else {
            r1.a.o = __fmul2_rn(cf2, f1.a.o);
            r1.b.e = __fmul2_rn(cf2, f1.b.e);
          }
        } else {
          sor_pairs<PM, ZP_RED == 0>(r1, &s_ub[ZP_RED * PL2], pa, pb, offL, offR, offU2, offD2,
                                      r2, r0, f1, p, fl, zlo, zhi);
        }
      }
      if (act) {  // the red cells: row a's e cells on an even plane, row b's o cells
        s_red[ZP_RED * PL2 + pa] = part<ZP_RED == 0>(r1.a);
        s_red[ZP_RED * PL2 + pb] = part<ZP_RED != 0>(r1.b);
      }
    }
    // [C] black half-step on plane q-2 (red values of planes q-3 .. q-1)
    {
      const int pz = q - 2;
      const bool zlo = !PZ && pz == 0, zhi = !PZ && pz == p.nz - 1;
      float2 dblk = make_float2(0.f, 0.f);
      if (q > q_first + 1)
        sor_pairs<PM, ZP_BLK != 0, SPLIT>(r2, &s_red[ZP_BLK * PL2], pa, pb, offL, offR, offU2,
                                           offD2, r3, r1, f2p, p, fl, zlo, zhi, &dblk);
      if (SPLIT && act && out && pz >= z0 && pz < z1) {
        // black defects of plane q-2 open (even plane) or join its coarse plane's sum
        constexpr int ZA = ((QP + 2) % 4) >> 1;  // parity of the coarse plane (q-2)/2
        if ((QP + 2) % 2 == 0) accz[ZA] = dblk;
        else accz[ZA] = add2(accz[ZA], dblk);
      }
      if (MODE == kDown && act) {  // black cells: row a's o cells on an even plane, row b's e
        s_finp[ZP_BLK * PL2 + pa] = part<ZP_BLK != 0>(r2.a);
        s_finp[ZP_BLK * PL2 + pb] = part<ZP_BLK == 0>(r2.b);
      }
      if (act && out && pz >= z0 && pz < z1) {
        const unsigned o = (unsigned)pz * plane + offA;
        *reinterpret_cast<float4*>(u_out + o) = pack(r2.a);
        *reinterpret_cast<float4*>(u_out + (o + p.nx)) = pack(r2.b);
      }
    }
    // [D] defect of plane q-3's red cells (its black cells' came from [C]) and
    // the 2x2x2 restriction
    if (MODE == kDown) {
      const int pz = q - 3;
      if (act && pz >= z0 && pz < z1 && out) {
        const bool zlo = !PZ && pz == 0, zhi = !PZ && pz == p.nz - 1;
        constexpr int ZA = ((QP + 1) % 4) >> 1;  // parity of the coarse plane (q-3)/2
        accz[ZA] = add2(accz[ZA], defect_red<PM, ZP_DEF == 0>(r3, &s_finp[ZP_DEF * PL2], pa, pb,
                                                               RS2, r4, r2, f3p, p, fl, zlo, zhi));
        if (ZP_DEF != 0) {
          const unsigned cnx = (unsigned)p.nx >> 1, cny = (unsigned)p.ny >> 1;
          const unsigned X = gx4 >> 1, Yc = gyA >> 1, Zc = pz >> 1;
          *reinterpret_cast<float2*>(fc + ((Zc * cny + Yc) * cnx + X)) =
              __fmul2_rn(make_float2(0.125f, 0.125f), accz[ZA]);
        }
      }
    }
    r4 = r3; r3 = r2; r2 = r1; r1 = r0;
    f3p = f2p; f2p = f1;
  };

  constexpr int Q0 = ((-HZ) % 4 + 4) % 4;  // q_first mod 4
  issue(std::integral_constant<int, Q0>{}, std::integral_constant<int, (Q0 + 3) % 4>{}, q_first);
  cp_async_commit();
  issue(std::integral_constant<int, (Q0 + 1) % 4>{}, std::integral_constant<int, Q0>{},
        q_first + 1);
  cp_async_commit();
  for (int q = q_first; q <= q_last; q += 4) {
    step(std::integral_constant<int, 0>{}, q);
    if (stop || q + 1 > q_last) break;
    step(std::integral_constant<int, 1>{}, q + 1);
    if (stop || q + 2 > q_last) break;
    step(std::integral_constant<int, 2>{}, q + 2);
    if (stop || q + 3 > q_last) break;
    step(std::integral_constant<int, 3>{}, q + 3);
    if (stop) break;
  }
  if (TMA && stop && threadIdx.x == 0) {
    // give the copies still in flight (planes q_stop and q_stop + 1) a
    // bounded time to land before the CTA's shared memory is released
    for (int q = q_stop; q <= q_stop + 1 && q <= q_last; ++q)
      mbar_wait(&tma_bar[q & 3], (unsigned)(((q - q_first) >> 2) & 1), nullptr);
  }
  cp_async_wait<0>();
}

// Register caps.  The register file is split among the four schedulers, so
// two 7-warp CTAs (down leg, 16-row tiles) fit on an SM at <= 128 registers
// and three 6-warp CTAs (up leg) at <= 96; the 32-row tiles take one CTA per
// SM (their shared memory alone decides).  The up leg with a non-periodic face
// needs more than 96 registers: it takes 128 and two CTAs per SM, which
// measured 28-33 % faster than spilling at three (mask 0, 1, 4 on a
// 256 x 256 x 512 box) and no slower for mask 3.
template <int MODE, int TY, int PM = 7>
constexpr int fused_max_regs() {
  return TY == 16 ? (MODE == kUp ? (PM == 7 ? 96 : 128) : 128) : 168;
}

template <int MODE, bool ZERO, int PM, int TX, int TY>
__global__ void __maxnreg__((fused_max_regs<MODE, TY, PM>()))
    k_fused(const float* __restrict__ u_in, float* __restrict__ u_out, const float* __restrict__ f,
            const float* __restrict__ ec, float* __restrict__ fc, FusedParams p) {
  extern __shared__ float4 smem[];
  fused_tile<MODE, ZERO, PM, TX, TY>(u_in, u_out, f, ec, fc, p, blockIdx.x, blockIdx.y, blockIdx.z,
                                     smem);
}

}  // namespace fused
}  // namespace mg
