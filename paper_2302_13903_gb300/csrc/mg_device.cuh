// mg_device.cuh -- device helpers shared by the per-level kernels, the
// single-CTA bottom solver and the batched solver.
//
// Layout: every level is an nx*ny*nz array of active cells, z-major, x
// fastest; there are no ghost cells in memory.  A neighbour outside the level
// is synthesised from the boundary rule at load time (Sec. 2.3.6): periodic
// wraps, zero gradient copies the adjacent cell, fixed / open give
// 2 b - (adjacent cell) with b the value on the face.  Where a stencil leaves
// the level along more than one axis (edges and corners of the 27-point
// prolongations) the face rule is applied along x, then y, then z.
//
// Each operation is written once as a "range" body: work items t0, t0 + dt,
// ... of one level, so that a grid-wide kernel (t0 = global thread, dt = all
// threads) and one CTA (t0 = threadIdx.x, dt = blockDim.x) share the code.
// Pointers are not __restrict__: a CTA reads values it wrote itself after a
// barrier.
#pragma once

#include <cuda_runtime.h>

#include "mg_internal.h"

namespace mg {
namespace dev {

__host__ __device__ inline size_t at(const Grid& g, int i, int j, int k) {
  return ((size_t)k * (size_t)g.ny + (size_t)j) * (size_t)g.nx + (size_t)i;
}

// Value on a face point; `a`, `b` are padded tangential indices (0..n+1).
__device__ inline double face_value(const Bc& bc, const Grid& g, int face, int a, int b) {
  if (bc.kind == BC_FIXED) return bc.value;
  if (bc.kind == BC_MIXED && !bc.faces) return 0.0;
  size_t off;
  size_t fx = (size_t)(g.ny + 2) * (g.nz + 2), fy = (size_t)(g.nx + 2) * (g.nz + 2),
         fz = (size_t)(g.nx + 2) * (g.ny + 2);
  if (face < 2) off = face * fx + (size_t)b * (g.ny + 2) + a;
  else if (face < 4) off = 2 * fx + (face - 2) * fy + (size_t)b * (g.nx + 2) + a;
  else off = 2 * fx + 2 * fy + (face - 4) * fz + (size_t)b * (g.nx + 2) + a;
  return bc.faces[off];
}

// Value at (i, j, k) where at least one index is -1 or n: the rule along z is
// the outermost, then y, then x (so the x rule acts on the stored value).
template <typename T>
__device__ __noinline__ T ghost(const T* u, int i, int j, int k, const Grid g,
                                const Bc bc) {
  int i2 = i, j2 = j, k2 = k;
  T az = 1, cz = 0, ay = 1, cy = 0, ax = 1, cx = 0;
  if ((unsigned)k >= (unsigned)g.nz) {
    const int hi = k >= g.nz, kind = face_kind(bc, 4 + hi);
    k2 = kind == BC_PERIODIC ? (hi ? 0 : g.nz - 1) : (hi ? g.nz - 1 : 0);
    if (kind == BC_FIXED || kind == BC_OPEN) {
      az = -1;
      cz = (T)(2.0 * face_value(bc, g, 4 + hi, i + 1, j + 1));
    }
  }
  if ((unsigned)j >= (unsigned)g.ny) {
    const int hi = j >= g.ny, kind = face_kind(bc, 2 + hi);
    j2 = kind == BC_PERIODIC ? (hi ? 0 : g.ny - 1) : (hi ? g.ny - 1 : 0);
    if (kind == BC_FIXED || kind == BC_OPEN) {
      ay = -1;
      cy = (T)(2.0 * face_value(bc, g, 2 + hi, i + 1, k2 + 1));
    }
  }
  if ((unsigned)i >= (unsigned)g.nx) {
    const int hi = i >= g.nx, kind = face_kind(bc, hi);
    i2 = kind == BC_PERIODIC ? (hi ? 0 : g.nx - 1) : (hi ? g.nx - 1 : 0);
    if (kind == BC_FIXED || kind == BC_OPEN) {
      ax = -1;
      cx = (T)(2.0 * face_value(bc, g, 0 + hi, j2 + 1, k2 + 1));
    }
  }
  T v = u[at(g, i2, j2, k2)];
  v = ax * v + cx;
  v = ay * v + cy;
  v = az * v + cz;
  return v;
}

// (i, j, k) of flat index t in an nx * ny * (any) array: shifts when nx and ny
// are powers of two (every level of a solve), divisions otherwise.
struct Split {
  int nx, ny, lx, lxy;
  bool pow2;
  __device__ __forceinline__ Split(int nx_, int ny_) : nx(nx_), ny(ny_) {
    pow2 = (nx & (nx - 1)) == 0 && (ny & (ny - 1)) == 0;
    lx = __ffs(nx) - 1;
    lxy = lx + __ffs(ny) - 1;
  }
  __device__ __forceinline__ void operator()(long long t, int& i, int& j, int& k) const {
    if (pow2) {
      i = (int)(t & (nx - 1));
      j = (int)((t >> lx) & (ny - 1));
      k = (int)(t >> lxy);
    } else {
      i = (int)(t % nx);
      const long long r = t / nx;
      j = (int)(r % ny);
      k = (int)(r / ny);
    }
  }
};

template <typename T>
__device__ __forceinline__ T fetch(const T* u, int i, int j, int k, const Grid& g,
                                   const Bc& bc) {
  if ((unsigned)i < (unsigned)g.nx && (unsigned)j < (unsigned)g.ny && (unsigned)k < (unsigned)g.nz)
    return u[at(g, i, j, k)];
  return ghost(u, i, j, k, g, bc);
}

// Sum of the six face neighbours of (i, j, k), in the order x-, x+, y-, y+, z-, z+.
template <typename T>
__device__ __forceinline__ T neighbour_sum(const T* u, int i, int j, int k,
                                           const Grid& g, const Bc& bc) {
  if (i > 0 && i < g.nx - 1 && j > 0 && j < g.ny - 1 && k > 0 && k < g.nz - 1) {
    const size_t c = at(g, i, j, k), sy = (size_t)g.nx, sz = (size_t)g.nx * g.ny;
    return u[c - 1] + u[c + 1] + u[c - sy] + u[c + sy] + u[c - sz] + u[c + sz];
  }
  return fetch(u, i - 1, j, k, g, bc) + fetch(u, i + 1, j, k, g, bc) + fetch(u, i, j - 1, k, g, bc) +
         fetch(u, i, j + 1, k, g, bc) + fetch(u, i, j, k - 1, g, bc) + fetch(u, i, j, k + 1, g, bc);
}

// SMOOTH: one colour of red-black SOR (Eqs. rbsor1-rbsor2),
// u <- (1 - omega) u + (omega / 6) sum_nb + (-omega h^2 / 6) f.

template <typename T>
__device__ __forceinline__ void sor_range(T* u, const T* f, Grid g, Bc bc, T cu, T cs, T cf,
                                          int colour, long long t0, long long dt) {
  const int hx = g.nx >> 1;
  const long long total = (long long)hx * g.ny * g.nz;
  const Split sp(hx, g.ny);
  for (long long t = t0; t < total; t += dt) {
    int m, j, k;
    sp(t, m, j, k);
    const int i = 2 * m + ((j + k + colour) & 1);
    const size_t c = at(g, i, j, k);
    const T s = neighbour_sum(u, i, j, k, g, bc);
    u[c] = cu * u[c] + cs * s + cf * f[c];
  }
}

// Red half-sweep from u = 0: every neighbour is 0 (and so is every ghost of
// the homogeneous rule), so red cells become cf * f; black cells are zeroed.
template <typename T>
__device__ __forceinline__ void sor_red_zero_range(T* u, const T* f, Grid g, T cf, long long t0,
                                                   long long dt) {
  const long long total = g.cells();
  const Split sp(g.nx, g.ny);
  for (long long t = t0; t < total; t += dt) {
    int i, j, k;
    sp(t, i, j, k);
    u[t] = ((i + j + k) & 1) ? T(0) : cf * f[t];
  }
}

// Defect of the eight children of each coarse cell, averaged (Algorithm 1,
// steps 2-3 with Eq. restriction).
template <typename T>
__device__ __forceinline__ void defect_restrict_range(const T* u, const T* f, T* fc, Grid g, Bc bc,
                                                      T inv_h2, long long t0, long long dt) {
  const Grid gc{g.nx / 2, g.ny / 2, g.nz / 2};
  const long long total = gc.cells();
  const Split sp(gc.nx, gc.ny);
  for (long long t = t0; t < total; t += dt) {
    int I, J, K;
    sp(t, I, J, K);
    T acc = 0;
    for (int c = 0; c < 2; ++c)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
          const int i = 2 * I + a, j = 2 * J + b, k = 2 * K + c;
          const size_t q = at(g, i, j, k);
          const T s = neighbour_sum(u, i, j, k, g, bc);
          acc += f[q] - (s - T(6) * u[q]) * inv_h2;
        }
    fc[t] = acc * T(0.125);
  }
}

template <typename T>
__device__ __forceinline__ void restrict_range(const T* uf, T* uc, Grid gf, long long t0,
                                               long long dt) {
  const Grid gc{gf.nx / 2, gf.ny / 2, gf.nz / 2};
  const long long total = gc.cells();
  const Split sp(gc.nx, gc.ny);
  for (long long t = t0; t < total; t += dt) {
    int I, J, K;
    sp(t, I, J, K);
    T acc = 0;
    for (int c = 0; c < 2; ++c)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) acc += uf[at(gf, 2 * I + a, 2 * J + b, 2 * K + c)];
    uc[t] = acc * T(0.125);
  }
}

// Prolongation, one thread per coarse cell writing its 2x2x2 children.  The
// 27 coarse values around the parent (ghosts from the coarse rule) are
// interpolated along x, then y, then z with the 1-D weights of the fine
// parity: trilinear (Eq. trilinear) takes 1/4, 3/4 of the parents I-1, I for
// an even (lower) child and 3/4, 1/4 of I, I+1 for an odd one; the FMG
// operator I' takes 5/32, 30/32, -3/32 of I-1, I, I+1 (even) and the mirror
// (odd).
template <typename T, bool HIGH>
__device__ __forceinline__ void interp1(const T a, const T b, const T c, T& even, T& odd) {
  if (!HIGH) {
    even = T(0.25) * a + T(0.75) * b;
    odd = T(0.75) * b + T(0.25) * c;
  } else {
    even = T(5.0 / 32.0) * a + T(30.0 / 32.0) * b + T(-3.0 / 32.0) * c;
    odd = T(-3.0 / 32.0) * a + T(30.0 / 32.0) * b + T(5.0 / 32.0) * c;
  }
}

template <typename T, bool HIGH>
__device__ __forceinline__ void prolong_range(const T* uc, T* uf, Grid gf, Bc bc, int add,
                                              long long t0, long long dt) {
  const Grid gc{gf.nx / 2, gf.ny / 2, gf.nz / 2};
  const long long total = gc.cells();
  const Split sp(gc.nx, gc.ny);
  for (long long t = t0; t < total; t += dt) {
    int I, J, K;
    sp(t, I, J, K);
    T c[3][3][3];
    if (I > 0 && I < gc.nx - 1 && J > 0 && J < gc.ny - 1 && K > 0 && K < gc.nz - 1) {
      const size_t sy = (size_t)gc.nx, sz = (size_t)gc.nx * gc.ny, o = at(gc, I, J, K);
#pragma unroll
      for (int cz = 0; cz < 3; ++cz)
#pragma unroll
        for (int cy = 0; cy < 3; ++cy)
#pragma unroll
          for (int cx = 0; cx < 3; ++cx)
            c[cz][cy][cx] = uc[o + (cz - 1) * sz + (cy - 1) * sy + (cx - 1)];
    } else {
#pragma unroll
      for (int cz = 0; cz < 3; ++cz)
#pragma unroll
        for (int cy = 0; cy < 3; ++cy)
#pragma unroll
          for (int cx = 0; cx < 3; ++cx)
            c[cz][cy][cx] = fetch(uc, I + cx - 1, J + cy - 1, K + cz - 1, gc, bc);
    }
    T vx[3][3][2];  // [cz][cy][x parity]
#pragma unroll
    for (int cz = 0; cz < 3; ++cz)
#pragma unroll
      for (int cy = 0; cy < 3; ++cy)
        interp1<T, HIGH>(c[cz][cy][0], c[cz][cy][1], c[cz][cy][2], vx[cz][cy][0], vx[cz][cy][1]);
    T vy[3][2][2];  // [cz][y parity][x parity]
#pragma unroll
    for (int cz = 0; cz < 3; ++cz)
#pragma unroll
      for (int px = 0; px < 2; ++px)
        interp1<T, HIGH>(vx[cz][0][px], vx[cz][1][px], vx[cz][2][px], vy[cz][0][px], vy[cz][1][px]);
#pragma unroll
    for (int py = 0; py < 2; ++py)
#pragma unroll
      for (int px = 0; px < 2; ++px) {
        T lo, hi;
        interp1<T, HIGH>(vy[0][py][px], vy[1][py][px], vy[2][py][px], lo, hi);
        const size_t q0 = at(gf, 2 * I + px, 2 * J + py, 2 * K);
        const size_t q1 = q0 + (size_t)gf.nx * gf.ny;
        uf[q0] = add ? uf[q0] + lo : lo;
        uf[q1] = add ? uf[q1] + hi : hi;
      }
  }
}

// The same prolongation over z-chunks of coarse columns: thread work item t
// is coarse column (I, J) = t mod (nx_c ny_c) and chunk t / (nx_c ny_c) of cz
// coarse planes.  The (x, y) interpolation of each coarse plane is formed
// once and kept in registers for the three pairs of fine planes that use it;
// every fine value takes the same operations in the same order as in
// prolong_range (x, then y, then z), so the results are the same bits.
template <typename T, bool HIGH>
__device__ __forceinline__ void xy_interp(const T* uc, const Grid& gc, const Bc& bc, int I, int J,
                                          int K, T out[2][2]) {
  T c[3][3];
  if (I > 0 && I < gc.nx - 1 && J > 0 && J < gc.ny - 1 && K >= 0 && K < gc.nz) {
    const size_t sy = (size_t)gc.nx, o = at(gc, I, J, K);
#pragma unroll
    for (int cy = 0; cy < 3; ++cy)
#pragma unroll
      for (int cx = 0; cx < 3; ++cx) c[cy][cx] = uc[o + (cy - 1) * sy + (cx - 1)];
  } else {
#pragma unroll
    for (int cy = 0; cy < 3; ++cy)
#pragma unroll
      for (int cx = 0; cx < 3; ++cx) c[cy][cx] = fetch(uc, I + cx - 1, J + cy - 1, K, gc, bc);
  }
  T vx[3][2];
#pragma unroll
  for (int cy = 0; cy < 3; ++cy)
    interp1<T, HIGH>(c[cy][0], c[cy][1], c[cy][2], vx[cy][0], vx[cy][1]);
#pragma unroll
  for (int px = 0; px < 2; ++px)
    interp1<T, HIGH>(vx[0][px], vx[1][px], vx[2][px], out[0][px], out[1][px]);
}

template <typename T, bool HIGH>
__device__ __forceinline__ void prolong_zchunk(const T* uc, T* uf, const Grid& gf, const Bc& bc,
                                               int add, long long t, int cz) {
  const Grid gc{gf.nx / 2, gf.ny / 2, gf.nz / 2};
  const long long cols = (long long)gc.nx * gc.ny;
  const int ch = (int)(t / cols);
  const int col = (int)(t - (long long)ch * cols);
  const int J = col / gc.nx, I = col - J * gc.nx;
  const int K0 = ch * cz, K1 = min(K0 + cz, gc.nz);
  T pm[2][2], p0[2][2], pp[2][2];
  xy_interp<T, HIGH>(uc, gc, bc, I, J, K0 - 1, pm);
  xy_interp<T, HIGH>(uc, gc, bc, I, J, K0, p0);
  const size_t plane = (size_t)gf.nx * gf.ny;
  for (int K = K0; K < K1; ++K) {
    xy_interp<T, HIGH>(uc, gc, bc, I, J, K + 1, pp);
#pragma unroll
    for (int py = 0; py < 2; ++py)
#pragma unroll
      for (int px = 0; px < 2; ++px) {
        T lo, hi;
        interp1<T, HIGH>(pm[py][px], p0[py][px], pp[py][px], lo, hi);
        const size_t q0 = at(gf, 2 * I + px, 2 * J + py, 2 * K), q1 = q0 + plane;
        uf[q0] = add ? uf[q0] + lo : lo;
        uf[q1] = add ? uf[q1] + hi : hi;
      }
#pragma unroll
    for (int py = 0; py < 2; ++py)
#pragma unroll
      for (int px = 0; px < 2; ++px) {
        pm[py][px] = p0[py][px];
        p0[py][px] = pp[py][px];
      }
  }
}

// COARSEST on a single cell: a ghost is 2 b_face - u on a fixed / open face
// and u itself on a periodic / zero-gradient one, so with a such faces
// sum(ghosts) - 6u = 2 sum(b) - 2 a u = h^2 f; with none it is singular.
template <typename T>
__device__ __forceinline__ void coarsest_one(const T* f, T* u, double h, Bc bc,
                                             bool keep = false) {
  const Grid g{1, 1, 1};
  int a = 0;
  double sb = 0.0;
  for (int face = 0; face < 6; ++face) {
    const int kind = face_kind(bc, face);
    if (kind == BC_FIXED || kind == BC_OPEN) {
      ++a;
      sb += face_value(bc, g, face, 1, 1);
    }
  }
  if (a == 0) {
    if (!keep) u[0] = T(0);  // singular: any value solves it; keep the start (FAS) or 0
    return;
  }
  u[0] = (T)((2.0 * sb - h * h * (double)f[0]) / (2.0 * a));
}

}  // namespace dev
}  // namespace mg
