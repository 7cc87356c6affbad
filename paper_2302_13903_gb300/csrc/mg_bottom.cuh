// mg_bottom.cuh -- block-level programs for the coarse end of a V-cycle
// (device code shared by the single-CTA bottom kernel and the batched solver).
// Each step is a block-strided loop over one level followed by __syncthreads;
// global memory written by the CTA is visible to the whole CTA after the
// barrier.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

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
  // SOR and defect coefficients in T per level (set by set_coefficients)
  T cu, cs;
  T cf[kBottomLevels], ih2[kBottomLevels];
};

// u <- cu u + cs sum_nb + cf f with cf = -omega h^2 / 6; 1 / h^2 for defects.
template <typename T>
__host__ __device__ inline void set_coefficients(BottomArgs<T>& a) {
  a.cu = (T)(1.0 - a.omega);
  a.cs = (T)(a.omega / 6.0);
  for (int l = 0; l < kBottomLevels; ++l) {
    const double h = a.h[l];
    a.cf[l] = (T)(-a.omega * h * h / 6.0);
    a.ih2[l] = h > 0.0 ? (T)(1.0 / (h * h)) : T(0);
  }
}

// ---------------------------------------------------------------------------
// Fast V-cycle for the homogeneous rules (every cycle below the top of a
// correction solve): levels are cubes of 2^lg cells, indices are split with
// shifts, and a neighbour outside the level is the periodic wrap, the cell
// itself (zero gradient) or minus the cell (zero fixed) -- the ghost of
// Sec. 2.3.6 for a zero boundary value, with no branch to a general routine.
// KIND is one rule for every face, or BC_MIXED: each face's kind from the
// mask fk of the homogeneous rule (bits 2q..2q+1 for face q).

template <int KIND>
__device__ __forceinline__ int hkind(int fk, int face) {
  return KIND == BC_MIXED ? (fk >> (2 * face)) & 3 : KIND;
}

template <typename T, int KIND>
__device__ __forceinline__ T hnb(const T* u, int c, bool inside, int off_in, int off_wrap,
                                 T self, int fk, int face) {
  if (inside) return u[c + off_in];
  const int kind = hkind<KIND>(fk, face);
  if (kind == BC_PERIODIC) return u[c + off_wrap];
  return kind == BC_ZEROGRAD ? self : -self;
}

// Sum of the six neighbours of cell c = (i, j, k), in the order x-, x+, y-,
// y+, z-, z+.
template <typename T, int KIND>
__device__ __forceinline__ T hsum(const T* u, int c, int i, int j, int k, int n, T self,
                                  int fk) {
  const int sy = n, sz = n * n, w = n - 1;
  T s = hnb<T, KIND>(u, c, i > 0, -1, w, self, fk, 0);
  s += hnb<T, KIND>(u, c, i < w, 1, -w, self, fk, 1);
  s += hnb<T, KIND>(u, c, j > 0, -sy, w * sy, self, fk, 2);
  s += hnb<T, KIND>(u, c, j < w, sy, -w * sy, self, fk, 3);
  s += hnb<T, KIND>(u, c, k > 0, -sz, w * sz, self, fk, 4);
  s += hnb<T, KIND>(u, c, k < w, sz, -w * sz, self, fk, 5);
  return s;
}

template <typename T, int KIND>
__device__ void h_smooth(const BottomArgs<T>& a, int l, int steps, bool zero_guess) {
  const int n = a.n[l], lg = __ffs(n) - 1, N = n * n * n;
  T* u = a.u[l];
  const T* f = a.f[l];
  const T cu = a.cu, cs = a.cs, cf = a.cf[l];
  if (zero_guess && steps == 0) {
    for (int t = threadIdx.x; t < N; t += blockDim.x) u[t] = T(0);
    __syncthreads();
    return;
  }
  for (int q = 0; q < steps; ++q) {
    if (q == 0 && zero_guess) {
      for (int t = threadIdx.x; t < N; t += blockDim.x) {
        const int i = t & (n - 1), j = (t >> lg) & (n - 1), k = t >> (2 * lg);
        u[t] = ((i + j + k) & 1) ? T(0) : cf * f[t];
      }
    } else {
      for (int t = threadIdx.x; t < N / 2; t += blockDim.x) {  // red
        const int r = t >> (lg - 1), j = r & (n - 1), k = r >> lg;
        const int i = 2 * (t & ((n >> 1) - 1)) + ((j + k) & 1);
        const int c = (r << lg) + i;
        const T self = u[c];
        u[c] = cu * self + cs * hsum<T, KIND>(u, c, i, j, k, n, self, a.hom.fk) + cf * f[c];
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < N / 2; t += blockDim.x) {  // black
      const int r = t >> (lg - 1), j = r & (n - 1), k = r >> lg;
      const int i = 2 * (t & ((n >> 1) - 1)) + ((j + k + 1) & 1);
      const int c = (r << lg) + i;
      const T self = u[c];
      u[c] = cu * self + cs * hsum<T, KIND>(u, c, i, j, k, n, self, a.hom.fk) + cf * f[c];
    }
    __syncthreads();
  }
}

// fc = average over the 8 children of f - L u (Algorithm 1, steps 2-3).
template <typename T, int KIND>
__device__ void h_defect_restrict(const BottomArgs<T>& a, int l) {
  const int n = a.n[l], nc = n >> 1, lgc = __ffs(nc) - 1, Nc = nc * nc * nc;
  const T* u = a.u[l];
  const T* f = a.f[l];
  T* fc = a.f[l - 1];
  const T ih2 = a.ih2[l];
  for (int t = threadIdx.x; t < Nc; t += blockDim.x) {
    const int I = t & (nc - 1), J = (t >> lgc) & (nc - 1), K = t >> (2 * lgc);
    T acc = 0;
    for (int cz = 0; cz < 2; ++cz)
      for (int by = 0; by < 2; ++by)
        for (int ax = 0; ax < 2; ++ax) {
          const int i = 2 * I + ax, j = 2 * J + by, k = 2 * K + cz;
          const int c = (k * n + j) * n + i;
          const T self = u[c];
          acc += f[c] - (hsum<T, KIND>(u, c, i, j, k, n, self, a.hom.fk) - T(6) * self) * ih2;
        }
    fc[t] = acc * T(0.125);
  }
}

// Coarse value at (I, J, K) with up to one cell outside on each axis: wrap,
// or the nearest cell times +1 (zero gradient) / -1 per axis left (zero fixed),
// by the rule of the face that was crossed.
template <typename T, int KIND>
__device__ __forceinline__ T hcoarse(const T* uc, int I, int J, int K, int nc, int fk) {
  T sg = T(1);
  auto fix = [&](int& q, int axis) {
    if (q >= 0 && q < nc) return;
    const int kind = hkind<KIND>(fk, 2 * axis + (q < 0 ? 0 : 1));
    if (kind == BC_PERIODIC) q = q < 0 ? q + nc : q - nc;
    else {
      q = q < 0 ? 0 : nc - 1;
      if (kind != BC_ZEROGRAD) sg = -sg;
    }
  };
  fix(I, 0);
  fix(J, 1);
  fix(K, 2);
  return sg * uc[(K * nc + J) * nc + I];
}

// u_l += trilinear(u_{l-1}) (Algorithm 1, steps 5-6), one thread per coarse cell.
template <typename T, int KIND>
__device__ void h_prolong_add(const BottomArgs<T>& a, int l) {
  const int n = a.n[l], nc = n >> 1, lgc = __ffs(nc) - 1, Nc = nc * nc * nc;
  const T* uc = a.u[l - 1];
  T* uf = a.u[l];
  for (int t = threadIdx.x; t < Nc; t += blockDim.x) {
    const int I = t & (nc - 1), J = (t >> lgc) & (nc - 1), K = t >> (2 * lgc);
    T c[3][3][3];
#pragma unroll
    for (int cz = 0; cz < 3; ++cz)
#pragma unroll
      for (int cy = 0; cy < 3; ++cy)
#pragma unroll
        for (int cx = 0; cx < 3; ++cx)
          c[cz][cy][cx] = hcoarse<T, KIND>(uc, I + cx - 1, J + cy - 1, K + cz - 1, nc, a.hom.fk);
    T vx[3][3][2];
#pragma unroll
    for (int cz = 0; cz < 3; ++cz)
#pragma unroll
      for (int cy = 0; cy < 3; ++cy)
        dev::interp1<T, false>(c[cz][cy][0], c[cz][cy][1], c[cz][cy][2], vx[cz][cy][0],
                               vx[cz][cy][1]);
    T vy[3][2][2];
#pragma unroll
    for (int cz = 0; cz < 3; ++cz)
#pragma unroll
      for (int px = 0; px < 2; ++px)
        dev::interp1<T, false>(vx[cz][0][px], vx[cz][1][px], vx[cz][2][px], vy[cz][0][px],
                               vy[cz][1][px]);
#pragma unroll
    for (int py = 0; py < 2; ++py)
#pragma unroll
      for (int px = 0; px < 2; ++px) {
        T lo, hi;
        dev::interp1<T, false>(vy[0][py][px], vy[1][py][px], vy[2][py][px], lo, hi);
        const int q0 = ((2 * K) * n + 2 * J + py) * n + 2 * I + px;
        uf[q0] += lo;
        uf[q0 + n * n] += hi;
      }
  }
}

template <typename T, int KIND>
__device__ void h_vcycle(const BottomArgs<T>& a, int top, bool zero_guess) {
  for (int l = top; l >= 1; --l) {
    h_smooth<T, KIND>(a, l, a.pre, l < top || zero_guess);
    h_defect_restrict<T, KIND>(a, l);
    __syncthreads();
  }
  if (threadIdx.x == 0) dev::coarsest_one(a.f[0], a.u[0], a.h[0], a.hom);
  __syncthreads();
  for (int l = 1; l <= top; ++l) {
    h_prolong_add<T, KIND>(a, l);
    __syncthreads();
    h_smooth<T, KIND>(a, l, a.post, false);
  }
}

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

// One V-cycle on levels top .. 0 with rule bc_top on level `top`.  PER_FACE:
// whether a rule per face (homogeneous, the same on every level) takes the
// fast cycle too (the batched solver has one rule per grid).
template <typename T, bool PER_FACE = true>
__device__ void vcycle(const BottomArgs<T>& a, int top, const Bc& bc_top, bool zero_guess) {
  if (bc_top.kind == a.hom.kind && bc_top.value == 0.0 && bc_top.kind != BC_OPEN &&
      bc_top.kind != BC_MIXED) {
    if (a.hom.kind == BC_PERIODIC) h_vcycle<T, BC_PERIODIC>(a, top, zero_guess);
    else if (a.hom.kind == BC_ZEROGRAD) h_vcycle<T, BC_ZEROGRAD>(a, top, zero_guess);
    else h_vcycle<T, BC_FIXED>(a, top, zero_guess);
    return;
  }
  if (PER_FACE && bc_top.kind == BC_MIXED && a.hom.kind == BC_MIXED && !bc_top.faces &&
      !a.hom.faces && bc_top.fk == a.hom.fk) {
    h_vcycle<T, BC_MIXED>(a, top, zero_guess);
    return;
  }
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
// The copy of the arguments with the shared-memory pointers lives in shared
// memory too: its per-level arrays are indexed by a run-time level, which in
// a thread's own copy would put them in local memory.
template <typename T, typename Body>
__device__ void in_shared(const BottomArgs<T>& a, T* smem, bool load_u, Body body) {
  __shared__ BottomArgs<T> b;
  if (threadIdx.x == 0) {
    b = a;
    const int total = cells_upto(a);
    int off = 0;
    for (int l = 0; l <= a.top; ++l) {
      b.u[l] = smem + off;
      b.f[l] = smem + total + off;
      off += a.n[l] * a.n[l] * a.n[l];
    }
  }
  __syncthreads();
  const int top = a.top, ct = a.n[top] * a.n[top] * a.n[top];
  // 16-byte global accesses where the arrays allow, a thread's loads all
  // issued before its shared stores (the copies are a chain of L2 round
  // trips otherwise); the shared copies are 4- or 8-byte aligned only
  using Vec = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  constexpr int V = 16 / sizeof(T);
  const bool vec = ct % V == 0 &&
                   ((reinterpret_cast<unsigned long long>(a.f[top]) |
                     reinterpret_cast<unsigned long long>(a.u[top])) & 15) == 0;
  auto copy_in = [&](const T* src, T* dst) {
    if (!vec) {
      for (int t = threadIdx.x; t < ct; t += blockDim.x) dst[t] = src[t];
      return;
    }
    constexpr int K = 4;
    const Vec* s4 = reinterpret_cast<const Vec*>(src);
    for (int t0 = threadIdx.x; t0 < ct / V; t0 += K * blockDim.x) {
      Vec r[K];
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (t0 + k * (int)blockDim.x < ct / V) r[k] = s4[t0 + k * blockDim.x];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int t = t0 + k * blockDim.x;
        if (t < ct / V) {
          const T* rv = reinterpret_cast<const T*>(&r[k]);
#pragma unroll
          for (int j = 0; j < V; ++j) dst[V * t + j] = rv[j];
        }
      }
    }
  };
  copy_in(a.f[top], b.f[top]);
  if (load_u) copy_in(a.u[top], b.u[top]);
  __syncthreads();
  body(b);
  __syncthreads();
  if (vec) {
    Vec* d4 = reinterpret_cast<Vec*>(a.u[top]);
    for (int t = threadIdx.x; t < ct / V; t += blockDim.x) {
      Vec r;
      T* rv = reinterpret_cast<T*>(&r);
#pragma unroll
      for (int j = 0; j < V; ++j) rv[j] = b.u[top][V * t + j];
      d4[t] = r;
    }
  } else {
    for (int t = threadIdx.x; t < ct; t += blockDim.x) a.u[top][t] = b.u[top][t];
  }
  __syncthreads();
}

}  // namespace bottom
}  // namespace mg
