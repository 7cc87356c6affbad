// mg_fused_ud.cuh -- the up leg of one V-cycle and the down leg of the next on
// the same FP32 level, fused into one z-marching pass: temporal blocking of
// the smoother, two SMOOTH steps per pass over HBM.
//
// Between two V(1,1) cycles on a level (Algorithm 1: steps 5-7 of cycle k,
// then steps 1-3 of cycle k+1) u goes through
//   u + I_{l-1}^l e_{l-1} -> SMOOTH -> SMOOTH -> d = f - L u -> f_{l-1} = I_l^{l-1} d
// without leaving the chip: the pass reads u, f and the coarse correction and
// writes u and the restricted defect, 13 bytes per cell in FP32 where the two
// legs apart move 25.
//
// The tile program is the one of mg_fused.cuh stretched by two half-steps.
// Per plane step q:
//   [A] plane q of u plus the prolonged correction,
//   [B] red half-step of the first SMOOTH on plane q-1,
//   [C] its black half-step on plane q-2,
//   [D] red half-step of the second SMOOTH on plane q-3,
//   [E] its black half-step on plane q-4, with the black cells' defects; plane
//       q-4 is written,
//   [F] the red cells' defects of plane q-5 and, every second plane, the
//       2x2x2 restriction.
// Each half-step reads the other colour of its own plane from a colour-pair
// plane written one step earlier, as in the single legs.  The halo a tile
// recomputes grows with the two extra half-steps: 5 planes in z, 6 rows in y
// and 8 cells in x (two float4 columns, to keep 16-byte alignment).
#pragma once

#include "mg_fused.cuh"

namespace mg {
namespace fused {

template <int TX, int TY>
struct ShapeUD {
  static constexpr int HZ = 5;   // planes of halo in z
  static constexpr int HY = 6;   // rows of halo in y (three row pairs)
  static constexpr int HX4 = 2;  // float4 columns of halo on each side in x
  static constexpr int RT = TX / 4 + 2 * HX4;   // float4 columns per row
  static constexpr int RS = row_stride(RT);     // float4 between rows in shared memory
  static constexpr int RR = TY + 2 * HY;        // rows
  static constexpr int RP = RR / 2;             // row pairs
  static constexpr int NT = RT * RP;            // threads
  static constexpr int PL = RS * RR;            // float4 per shared plane
  static constexpr int RS2 = pair_stride(RT);   // float2 between rows of a pair plane
  static constexpr int PL2 = RS2 * RR;          // float2 per pair plane
  static constexpr int CXO = 8;                 // coarse columns left of x0 / 2
  static constexpr int CX = TX / 2 + 2 * CXO;   // coarse tile columns
  static constexpr int CY = RP + 2;             // coarse tile rows
  static constexpr int C0 = CXO - 2 * HX4 - 1;  // tile column of thread 0's first coarse cell
  static constexpr int NPAIR = 10;              // five pair planes, each double-buffered
  static constexpr size_t SMEM =
      (size_t)8 * PL * 16 + (size_t)NPAIR * PL2 * 8 + (size_t)2 * CX * CY * 4;
};

// The program of one CTA on tile (bx, by), z-chunk bz.  `smem` holds
// ShapeUD::SMEM bytes.  32-bit element offsets (levels below 2^32 cells).
template <int PM, int TX, int TY>
__device__ __forceinline__ void updown_tile(const float* u_in, float* u_out, const float* f,
                                            const float* ec, float* fc, const FusedParams& p,
                                            int bx, int by, int bz, float4* smem) {
  using S_ = ShapeUD<TX, TY>;
  constexpr int HZ = S_::HZ, HY = S_::HY, RT = S_::RT, RS = S_::RS, RP = S_::RP, PL = S_::PL;
  constexpr int RS2 = S_::RS2, PL2 = S_::PL2, CX = S_::CX, CY = S_::CY;
  float4* s_u = smem;           // [4][PL] planes of u (async copies)
  float4* s_f = s_u + 4 * PL;   // [4][PL] planes of f (async copies)
  // [2][PL2] each: the colour-pair planes, by the half-step that reads them
  float2* s_ub = reinterpret_cast<float2*>(s_f + 4 * PL);  // black of u + correction -> [B]
  float2* s_r1 = s_ub + 2 * PL2;                           // red after [B] -> [C]
  float2* s_b1 = s_r1 + 2 * PL2;                           // black after [C] -> [D]
  float2* s_r2 = s_b1 + 2 * PL2;                           // red after [D] -> [E]
  float2* s_fin = s_r2 + 2 * PL2;                          // final black after [E] -> [F]
  float* s_c = reinterpret_cast<float*>(s_fin + 2 * PL2);  // [2][CY][CX] coarse planes

  const int tid = threadIdx.x;
  const int tr = tid % RT, tp = tid / RT;
  const int x0 = bx * TX, y0 = by * TY;
  const int z0 = bz * p.cz;
  const int z1 = min(z0 + p.cz, p.nz);
  const int gx4 = x0 - 4 * S_::HX4 + 4 * tr;  // x of the patch's first cell (may be outside)
  const int gyA = y0 - HY + 2 * tp;           // even row of the patch (may be outside)
  constexpr bool PX = Per<PM>::X, PY = Per<PM>::Y, PZ = Per<PM>::Z;
  const int gx4w = PX ? wrap(gx4, p.nx) : gx4;
  const int gyAw = PY ? wrap(gyA, p.ny) : gyA;
  const bool col_ok = (PX || (gx4 >= 0 && gx4 < p.nx)) && (PY || (gyA >= 0 && gyA < p.ny));
  Flags fl;
  fl.xlo = !PX && gx4 == 0;
  fl.xhi = !PX && gx4 + 3 == p.nx - 1;
  fl.ylo = !PY && gyA == 0;
  fl.yhi = !PY && gyA + 1 == p.ny - 1;
  const bool out = tr >= S_::HX4 && tr < S_::HX4 + TX / 4 && tp >= HY / 2 && tp < HY / 2 + TY / 2;
  const unsigned plane = (unsigned)p.nx * (unsigned)p.ny;
  const unsigned offA = col_ok ? (unsigned)gyAw * p.nx + gx4w : 0u;
  const int ia = (2 * tp) * RS + tr, ib = ia + RS;
  const int pa = (2 * tp) * RS2 + tr, pb = pa + RS2;
  const int offU2 = tp > 0 ? -RS2 : 0, offD2 = tp < RP - 1 ? RS2 : 0;
  const int offL = tr > 0 ? -1 : 0, offR = tr < RT - 1 ? 1 : 0;
  const int q_first = z0 - HZ, q_last = z1 - 1 + HZ;

  // plane qu of u into ring slot SU, plane qu - 1 of f into slot SF
  auto issue = [&](auto SUc, auto SFc, int qu) {
    constexpr int SU = decltype(SUc)::value, SF = decltype(SFc)::value;
    if (qu <= q_last) {
      const bool in = col_ok && (PZ || (qu >= 0 && qu < p.nz));
      const unsigned o = (unsigned)(PZ ? wrap(qu, p.nz) : (in ? qu : 0)) * plane + offA;
      cp_async16(&s_u[SU * PL + ia], u_in + o, in ? 16 : 0);
      cp_async16(&s_u[SU * PL + ib], u_in + (o + p.nx), in ? 16 : 0);
      const int qf = qu - 1;
      const bool inf = col_ok && (PZ || (qf >= 0 && qf < p.nz));
      const unsigned of = (unsigned)(PZ ? wrap(qf, p.nz) : (inf ? qf : 0)) * plane + offA;
      cp_async16(&s_f[SF * PL + ia], f + of, inf ? 16 : 0);
      cp_async16(&s_f[SF * PL + ib], f + (of + p.nx), inf ? 16 : 0);
    }
  };

  // coarse plane Kc (any index from -4 to cnz + 1) into slot SL: CX columns
  // from x0/2 - CXO, CY rows from y0/2 - HY/2 - 1
  const int cx0 = (x0 >> 1) - S_::CXO, cy0 = (y0 >> 1) - HY / 2 - 1;
  auto copy_coarse = [&](auto SLc, int Kc) {
    constexpr int SL = decltype(SLc)::value, CW = CX / 4;
    const int cnx = p.nx >> 1, cny = p.ny >> 1, cnz = p.nz >> 1;
    if (tid < CW * CY) {
      const int i = tid / CW, j = tid - i * CW;
      int X = cx0 + 4 * j, Y = cy0 + i, K = Kc;
      bool in = true;
      if (PX) X = wrap(X, cnx);
      else in = X >= 0 && X < cnx;
      if (PY) Y = wrap(Y, cny);
      else in = in && Y >= 0 && Y < cny;
      if (PZ) K = wrap(K, cnz);
      else K = K < 0 ? 0 : (K >= cnz ? cnz - 1 : K);
      if (!in) { X = 0; Y = 0; }
      cp_async16(s_c + SL * CX * CY + i * CX + 4 * j, ec + (((unsigned)K * cny + Y) * cnx + X),
                 in ? 16 : 0);
    }
  };
  auto plane_sign = [&](int Kc) {
    return PZ ? 1.f : (Kc < 0 ? p.sz0 : (Kc >= (p.nz >> 1) ? p.sz1 : 1.f));
  };

  Patch r1 = zero_patch(), r2 = r1, r3 = r1, r4 = r1, r5 = r1, r6 = r1;
  // f of planes q-3 .. q-5 (planes q-1 and q-2 are read from the ring, which
  // keeps a plane of f until the step after its black half-step)
  Patch f3p = r1, f4p = r1, f5p = r1;
  float2 accz[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  // the (x, y)-interpolated coarse planes, by the parity of their index (as
  // in the up leg of mg_fused.cuh)
  Patch W[2];
  CoarseIdx ci;
  if (!(PX && PY)) ci = coarse_idx<PM>(p, gx4, gyA, cx0, cy0);
  {
    // q_first = z0 - 5 with z0 a multiple of 8: K0 = floor(q_first / 2) is odd
    const int K0 = q_first >> 1;
    copy_coarse(std::integral_constant<int, 0>{}, K0 - 1);
    copy_coarse(std::integral_constant<int, 1>{}, K0);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    W[0] = xy_combine(xy_read<PM, CX, S_::C0>(s_c, ci, tr, tp, plane_sign(K0 - 1)));
    W[1] = xy_combine(xy_read<PM, CX, S_::C0>(s_c + CX * CY, ci, tr, tp, plane_sign(K0)));
    __syncthreads();
    copy_coarse(std::integral_constant<int, 0>{}, K0 + 1);  // committed with plane q_first
  }

  auto zflags = [&](int pz, bool& zlo, bool& zhi) {
    zlo = !PZ && pz == 0;
    zhi = !PZ && pz == p.nz - 1;
  };

  auto step = [&](auto Jc, int q) {
    constexpr int J = decltype(Jc)::value;
    constexpr int QP = ((J - HZ) % 4 + 4) % 4;  // q mod 4
    constexpr int SL_U = QP, SL_FM1 = (QP + 3) % 4, SL_FM2 = (QP + 2) % 4;
    // parities of planes q-1 .. q-5
    constexpr int ZB = (QP + 1) % 2, ZC = QP % 2, ZD = (QP + 1) % 2, ZE = QP % 2,
                  ZF = (QP + 1) % 2;
    cp_async_wait<1>();  // this thread's copies of plane q have landed
    __syncthreads();     // ... and everyone's; the previous step is finished
    issue(std::integral_constant<int, (QP + 2) % 4>{}, std::integral_constant<int, (QP + 1) % 4>{},
          q + 2);
    if ((QP & 1) && q + 2 <= q_last)  // q = 2K+1: coarse plane K+2 into slot K mod 2
      copy_coarse(std::integral_constant<int, (QP >> 1) & 1>{}, (q >> 1) + 2);
    cp_async_commit();
    // [A] plane q of u plus the trilinear correction
    Patch r0;
    r0.a = unpack(s_u[SL_U * PL + ia]);
    r0.b = unpack(s_u[SL_U * PL + ib]);
    {
      constexpr int KP = (QP >> 1) & 1;  // parity of K = floor(q / 2)
      const int K = q >> 1;
      if (QP & 1)
        W[1 - KP] = xy_combine(xy_read<PM, CX, S_::C0>(s_c + (1 - KP) * CX * CY, ci, tr, tp,
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
    // black cells of plane q: row a's o cells on an even plane, row b's e
    s_ub[(QP & 1) * PL2 + pa] = part<(QP & 1) != 0>(r0.a);
    s_ub[(QP & 1) * PL2 + pb] = part<(QP & 1) == 0>(r0.b);
    // f of plane q-1 (its red cells serve [B]) and of plane q-2 ([C], then
    // kept for [D] - [F]): slot (q-2) mod 4 is refilled only after the next
    // step's barrier
    Patch f1, f2p;
    f1.a = unpack(s_f[SL_FM1 * PL + ia]);
    f1.b = unpack(s_f[SL_FM1 * PL + ib]);
    f2p.a = unpack(s_f[SL_FM2 * PL + ia]);
    f2p.b = unpack(s_f[SL_FM2 * PL + ib]);
    bool zlo, zhi;
    // [B] first SMOOTH, red half-step on plane q-1
    zflags(q - 1, zlo, zhi);
    if (q > q_first)
      sor_pairs<PM, ZB == 0>(r1, &s_ub[ZB * PL2], pa, pb, offL, offR, offU2, offD2, r2, r0, f1, p,
                             fl, zlo, zhi);
    s_r1[ZB * PL2 + pa] = part<ZB == 0>(r1.a);
    s_r1[ZB * PL2 + pb] = part<ZB != 0>(r1.b);
    // [C] first SMOOTH, black half-step on plane q-2
    zflags(q - 2, zlo, zhi);
    if (q > q_first + 1)
      sor_pairs<PM, ZC != 0>(r2, &s_r1[ZC * PL2], pa, pb, offL, offR, offU2, offD2, r3, r1, f2p,
                             p, fl, zlo, zhi);
    s_b1[ZC * PL2 + pa] = part<ZC != 0>(r2.a);
    s_b1[ZC * PL2 + pb] = part<ZC == 0>(r2.b);
    // [D] second SMOOTH, red half-step on plane q-3
    zflags(q - 3, zlo, zhi);
    if (q > q_first + 2)
      sor_pairs<PM, ZD == 0>(r3, &s_b1[ZD * PL2], pa, pb, offL, offR, offU2, offD2, r4, r2, f3p,
                             p, fl, zlo, zhi);
    s_r2[ZD * PL2 + pa] = part<ZD == 0>(r3.a);
    s_r2[ZD * PL2 + pb] = part<ZD != 0>(r3.b);
    // [E] second SMOOTH, black half-step on plane q-4 (with the black cells'
    // defects); plane q-4 is final
    {
      const int pz = q - 4;
      zflags(pz, zlo, zhi);
      float2 dblk = make_float2(0.f, 0.f);
      if (q > q_first + 3)
        sor_pairs<PM, ZE != 0, true>(r4, &s_r2[ZE * PL2], pa, pb, offL, offR, offU2, offD2, r5,
                                     r3, f4p, p, fl, zlo, zhi, &dblk);
      if (out && pz >= z0 && pz < z1) {
        constexpr int ZA = QP >> 1;  // parity of the coarse plane (q-4)/2
        if (ZE == 0) accz[ZA] = dblk;
        else accz[ZA] = add2(accz[ZA], dblk);
        const unsigned o = (unsigned)pz * plane + offA;
        *reinterpret_cast<float4*>(u_out + o) = pack(r4.a);
        *reinterpret_cast<float4*>(u_out + (o + p.nx)) = pack(r4.b);
      }
      s_fin[ZE * PL2 + pa] = part<ZE != 0>(r4.a);
      s_fin[ZE * PL2 + pb] = part<ZE == 0>(r4.b);
    }
    // [F] the red cells' defects of plane q-5, and the restriction
    {
      const int pz = q - 5;
      if (out && pz >= z0 && pz < z1) {
        zflags(pz, zlo, zhi);
        constexpr int ZA = ((QP + 3) % 4) >> 1;  // parity of the coarse plane (q-5)/2
        accz[ZA] = add2(accz[ZA], defect_red<PM, ZF == 0>(r5, &s_fin[ZF * PL2], pa, pb, RS2, r6,
                                                           r4, f5p, p, fl, zlo, zhi));
        if (ZF != 0) {
          const unsigned cnx = (unsigned)p.nx >> 1, cny = (unsigned)p.ny >> 1;
          const unsigned X = gx4 >> 1, Yc = gyA >> 1, Zc = pz >> 1;
          *reinterpret_cast<float2*>(fc + ((Zc * cny + Yc) * cnx + X)) =
              __fmul2_rn(make_float2(0.125f, 0.125f), accz[ZA]);
        }
      }
    }
    r6 = r5; r5 = r4; r4 = r3; r3 = r2; r2 = r1; r1 = r0;
    f5p = f4p; f4p = f3p; f3p = f2p;
  };

  constexpr int Q0 = ((-HZ) % 4 + 4) % 4;  // q_first mod 4
  issue(std::integral_constant<int, Q0>{}, std::integral_constant<int, (Q0 + 3) % 4>{}, q_first);
  cp_async_commit();
  issue(std::integral_constant<int, (Q0 + 1) % 4>{}, std::integral_constant<int, Q0>{},
        q_first + 1);
  cp_async_commit();
  for (int q = q_first; q <= q_last; q += 4) {
    step(std::integral_constant<int, 0>{}, q);
    if (q + 1 > q_last) break;
    step(std::integral_constant<int, 1>{}, q + 1);
    if (q + 2 > q_last) break;
    step(std::integral_constant<int, 2>{}, q + 2);
    if (q + 3 > q_last) break;
    step(std::integral_constant<int, 3>{}, q + 3);
  }
  cp_async_wait<0>();
}

// Register caps: one CTA per SM (shared memory decides), and the register file
// is split among the four schedulers, whose warps each hold their share: 14
// warps of 32-row tiles (four on some scheduler) at 128, 9 warps of 16-row
// tiles (three on some scheduler) at 168.
template <int TY>
constexpr int updown_max_regs() {
  return TY == 32 ? 128 : 168;
}

template <int PM, int TX, int TY>
__global__ void __maxnreg__((updown_max_regs<TY>()))
    k_updown(const float* __restrict__ u_in, float* __restrict__ u_out,
             const float* __restrict__ f, const float* __restrict__ ec, float* __restrict__ fc,
             FusedParams p) {
  extern __shared__ float4 smem[];
  updown_tile<PM, TX, TY>(u_in, u_out, f, ec, fc, p, blockIdx.x, blockIdx.y, blockIdx.z, smem);
}

}  // namespace fused
}  // namespace mg
