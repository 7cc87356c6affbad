// mg_multipole.cu -- open boundary values from a multipole expansion (App. A).
//
// The moments Q_lm = sum rho dV sqrt(4 pi/(2l+1)) r'^l Y_lm(r') only need the
// solid harmonics r^l Y_lm, which are homogeneous polynomials of degree l in
// (x, y, z).  So one pass over rho accumulates the 35 raw monomial moments
// M_abc = sum rho x^a y^b z^c (a+b+c <= 4) about the grid centre; the centre of
// mass, the shift of the moments to it (binomial expansion) and the 25 Q_lm
// follow on the device from those 35 numbers.  Along a row only x varies, so
// the pass costs five FP64 accumulations per cell (sum rho x^a, a = 0..4)
// and the y, z powers are applied once per row.
//
// The boundary potential -G sum Q_lm sqrt(4 pi/(2l+1)) Y_lm(r)/r^(l+1) equals
// -G sum Q_lm sqrt(4 pi/(2l+1)) R_lm(r) / r^(2l+1) with the same polynomials.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "mg_device.cuh"
#include "mg_internal.h"

namespace mg {
namespace {

constexpr int kMono = 35;  // monomials x^a y^b z^c with a+b+c <= 4
constexpr int kTerms = 25; // (l, m) pairs with l <= 4

// Monomial exponents, ordered by degree, then a descending, then b descending.
__constant__ unsigned char c_mono[kMono][3];

// r^l Y_lm written out as polynomials from the Cartesian table of App. A:
// each term is (lm index, monomial index, coefficient).  Coefficients are
// filled on the host: sqrt(c / pi) times the polynomial's integer factor.
constexpr int kMaxTerms = 96;
__constant__ int c_nterm;
__constant__ int c_term_lm[kMaxTerms];
__constant__ int c_term_mono[kMaxTerms];
__constant__ double c_term_coef[kMaxTerms];

struct HostTables {
  unsigned char mono[kMono][3];
  int nterm = 0;
  int lm[kMaxTerms], mi[kMaxTerms];
  double coef[kMaxTerms];

  int mono_index(int a, int b, int c) const {
    for (int q = 0; q < kMono; ++q)
      if (mono[q][0] == a && mono[q][1] == b && mono[q][2] == c) return q;
    return -1;
  }
  void add(int l, int m, double norm_c_over_pi, double factor, int a, int b, int c) {
    const double pi = 3.14159265358979323846;
    lm[nterm] = l * l + m + l;
    mi[nterm] = mono_index(a, b, c);
    coef[nterm] = std::sqrt(norm_c_over_pi / pi) * factor;
    ++nterm;
  }
  HostTables() {
    int q = 0;
    for (int d = 0; d <= 4; ++d)
      for (int a = d; a >= 0; --a)
        for (int b = d - a; b >= 0; --b) {
          mono[q][0] = (unsigned char)a;
          mono[q][1] = (unsigned char)b;
          mono[q][2] = (unsigned char)(d - a - b);
          ++q;
        }
    // l = 0
    add(0, 0, 1.0 / 4, 1, 0, 0, 0);
    // l = 1: y, z, x
    add(1, -1, 3.0 / 4, 1, 0, 1, 0);
    add(1, 0, 3.0 / 4, 1, 0, 0, 1);
    add(1, 1, 3.0 / 4, 1, 1, 0, 0);
    // l = 2
    add(2, -2, 15.0 / 4, 1, 1, 1, 0);
    add(2, -1, 15.0 / 4, 1, 0, 1, 1);
    add(2, 0, 5.0 / 16, -1, 2, 0, 0);  // 3z^2 - r^2 = 2z^2 - x^2 - y^2
    add(2, 0, 5.0 / 16, -1, 0, 2, 0);
    add(2, 0, 5.0 / 16, 2, 0, 0, 2);
    add(2, 1, 15.0 / 4, 1, 1, 0, 1);
    add(2, 2, 15.0 / 4, 0.5, 2, 0, 0);  // (x^2 - y^2)/2
    add(2, 2, 15.0 / 4, -0.5, 0, 2, 0);
    // l = 3
    add(3, -3, 35.0 / 32, 3, 2, 1, 0);  // y(3x^2 - y^2)
    add(3, -3, 35.0 / 32, -1, 0, 3, 0);
    add(3, -2, 105.0 / 4, 1, 1, 1, 1);  // xyz
    add(3, -1, 21.0 / 32, 4, 0, 1, 2);  // y(5z^2 - r^2) = 4yz^2 - x^2 y - y^3
    add(3, -1, 21.0 / 32, -1, 2, 1, 0);
    add(3, -1, 21.0 / 32, -1, 0, 3, 0);
    add(3, 0, 7.0 / 16, 2, 0, 0, 3);    // z(5z^2 - 3r^2) = 2z^3 - 3x^2 z - 3y^2 z
    add(3, 0, 7.0 / 16, -3, 2, 0, 1);
    add(3, 0, 7.0 / 16, -3, 0, 2, 1);
    add(3, 1, 21.0 / 32, 4, 1, 0, 2);   // x(5z^2 - r^2) = 4xz^2 - x^3 - xy^2
    add(3, 1, 21.0 / 32, -1, 3, 0, 0);
    add(3, 1, 21.0 / 32, -1, 1, 2, 0);
    add(3, 2, 105.0 / 4, 0.5, 2, 0, 1); // z(x^2 - y^2)/2
    add(3, 2, 105.0 / 4, -0.5, 0, 2, 1);
    add(3, 3, 35.0 / 32, 1, 3, 0, 0);   // x(x^2 - 3y^2)
    add(3, 3, 35.0 / 32, -3, 1, 2, 0);
    // l = 4
    add(4, -4, 315.0 / 4, 0.5, 3, 1, 0);   // xy(x^2 - y^2)/2
    add(4, -4, 315.0 / 4, -0.5, 1, 3, 0);
    add(4, -3, 315.0 / 32, 3, 2, 1, 1);    // yz(3x^2 - y^2)
    add(4, -3, 315.0 / 32, -1, 0, 3, 1);
    add(4, -2, 45.0 / 16, 6, 1, 1, 2);     // xy(7z^2 - r^2) = 6xyz^2 - x^3 y - x y^3
    add(4, -2, 45.0 / 16, -1, 3, 1, 0);
    add(4, -2, 45.0 / 16, -1, 1, 3, 0);
    add(4, -1, 45.0 / 32, 4, 0, 1, 3);     // yz(7z^2 - 3r^2) = 4yz^3 - 3x^2 yz - 3y^3 z
    add(4, -1, 45.0 / 32, -3, 2, 1, 1);
    add(4, -1, 45.0 / 32, -3, 0, 3, 1);
    add(4, 0, 9.0 / 256, 3, 4, 0, 0);      // 35z^4 - 30z^2 r^2 + 3r^4
    add(4, 0, 9.0 / 256, 3, 0, 4, 0);      //  = 3x^4 + 3y^4 + 8z^4 + 6x^2y^2
    add(4, 0, 9.0 / 256, 8, 0, 0, 4);      //    - 24x^2z^2 - 24y^2z^2
    add(4, 0, 9.0 / 256, 6, 2, 2, 0);
    add(4, 0, 9.0 / 256, -24, 2, 0, 2);
    add(4, 0, 9.0 / 256, -24, 0, 2, 2);
    add(4, 1, 45.0 / 32, 4, 1, 0, 3);      // xz(7z^2 - 3r^2) = 4xz^3 - 3x^3 z - 3xy^2 z
    add(4, 1, 45.0 / 32, -3, 3, 0, 1);
    add(4, 1, 45.0 / 32, -3, 1, 2, 1);
    add(4, 2, 45.0 / 16, 3, 2, 0, 2);      // (x^2 - y^2)(7z^2 - r^2)/2
    add(4, 2, 45.0 / 16, -3, 0, 2, 2);     //  = (6x^2z^2 - 6y^2z^2 - x^4 + y^4)/2
    add(4, 2, 45.0 / 16, -0.5, 4, 0, 0);
    add(4, 2, 45.0 / 16, 0.5, 0, 4, 0);
    add(4, 3, 315.0 / 32, 1, 3, 0, 1);     // xz(x^2 - 3y^2)
    add(4, 3, 315.0 / 32, -3, 1, 2, 1);
    add(4, 4, 315.0 / 4, 0.125, 4, 0, 0);  // (x^4 - 6x^2y^2 + y^4)/8
    add(4, 4, 315.0 / 4, -0.75, 2, 2, 0);
    add(4, 4, 315.0 / 4, 0.125, 0, 4, 0);
  }
};

// The tables live in __constant__ memory, which exists once per device: each
// device gets them on first use.
cudaError_t upload_tables() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return cudaSuccess;
  HostTables t;
  if ((e = cudaMemcpyToSymbol(c_mono, t.mono, sizeof t.mono)) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_nterm, &t.nterm, sizeof(int))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_term_lm, t.lm, sizeof(int) * t.nterm)) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_term_mono, t.mi, sizeof(int) * t.nterm)) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_term_coef, t.coef, sizeof(double) * t.nterm)) != cudaSuccess)
    return e;
  done[dev] = true;
  return cudaSuccess;
}

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// One warp per row (j, k): lanes stride over x and accumulate sum rho x^a,
// a = 0..4; a butterfly sum gives every lane the row totals; lane q owns
// monomials q and q + 32 and adds S_a y^b z^c for its (a, b, c).  Warps of a
// block are combined in warp order; blocks write [block][35] partials.
__global__ void k_raw_moments(const double* __restrict__ rho, Grid g, double h,
                              double* __restrict__ partials) {
  __shared__ double sm[kWarps][kMono];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long rows = (long long)g.ny * g.nz;
  const long long gw = (long long)blockIdx.x * kWarps + w, nw = (long long)gridDim.x * kWarps;
  double acc0 = 0.0, acc1 = 0.0;
  const int m0 = lane, m1 = lane + 32;
  int a0 = c_mono[m0][0], b0 = c_mono[m0][1], e0 = c_mono[m0][2];
  int a1 = 0, b1 = 0, e1 = 0;
  if (m1 < kMono) { a1 = c_mono[m1][0]; b1 = c_mono[m1][1]; e1 = c_mono[m1][2]; }
  // rows of at most 256 cells: the powers of x of this lane's (at most 8)
  // columns are the same in every row and are formed once, so a cell costs one
  // add and four independent multiply-adds
  const bool narrow = g.nx <= 256;
  double xs[8][4];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const double x = ((double)(lane + 32 * c) + 0.5 - 0.5 * g.nx) * h;
    xs[c][0] = x;
    xs[c][1] = x * x;
    xs[c][2] = xs[c][1] * x;
    xs[c][3] = xs[c][2] * x;
  }
  for (long long row = gw; row < rows; row += nw) {
    const int j = (int)(row % g.ny), k = (int)(row / g.ny);
    const double* r = rho + (size_t)row * g.nx;
    double s[5] = {0, 0, 0, 0, 0};
    if (narrow) {
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int i = lane + 32 * c;
        if (i < g.nx) {
          const double t = r[i];
          s[0] += t;
          s[1] = fma(t, xs[c][0], s[1]);
          s[2] = fma(t, xs[c][1], s[2]);
          s[3] = fma(t, xs[c][2], s[3]);
          s[4] = fma(t, xs[c][3], s[4]);
        }
      }
    } else {
      for (int i = lane; i < g.nx; i += 32) {
        const double x = ((double)i + 0.5 - 0.5 * g.nx) * h;
        double t = r[i];
        s[0] += t; t *= x;
        s[1] += t; t *= x;
        s[2] += t; t *= x;
        s[3] += t; t *= x;
        s[4] += t;
      }
    }
    for (int p = 0; p < 5; ++p)
      for (int o = 16; o > 0; o >>= 1) s[p] += __shfl_xor_sync(0xffffffffu, s[p], o);
    const double y = ((double)j + 0.5 - 0.5 * g.ny) * h, z = ((double)k + 0.5 - 0.5 * g.nz) * h;
    double yp[5], zp[5];
    yp[0] = zp[0] = 1.0;
    for (int p = 1; p < 5; ++p) { yp[p] = yp[p - 1] * y; zp[p] = zp[p - 1] * z; }
    acc0 += s[a0] * yp[b0] * zp[e0];
    if (m1 < kMono) acc1 += s[a1] * yp[b1] * zp[e1];
  }
  sm[w][m0] = acc0;
  if (m1 < kMono) sm[w][m1] = acc1;
  __syncthreads();
  for (int m = threadIdx.x; m < kMono; m += blockDim.x) {
    double t = 0.0;
    for (int q = 0; q < kWarps; ++q) t += sm[q][m];
    partials[(size_t)blockIdx.x * kMono + m] = t;
  }
}

__device__ double binom(int n, int k) {
  double r = 1.0;
  for (int q = 1; q <= k; ++q) r = r * (n - k + q) / q;
  return r;
}

// One block: reduce partials per monomial in block order, then the centre of
// mass (thread 0), the moments about it (one monomial per thread) and Q_lm
// (thread 0).
__global__ void k_moments_finish(const double* __restrict__ partials, int nb, double h, int lmax,
                                 int use_com, double ox, double oy, double oz,
                                 double* __restrict__ out) {
  __shared__ double M[kMono];
  __shared__ double Cs[kMono];
  __shared__ double P[3][5];  // (-o)^p per axis, p = 0..4
  for (int m = threadIdx.x; m < kMono; m += blockDim.x) {
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += partials[(size_t)b * kMono + m];
    M[m] = t;
  }
  __syncthreads();
  // M[0] = sum rho, M[1..3] = sum rho x, y, z (indices of (1,0,0), (0,1,0), (0,0,1))
  if (threadIdx.x == 0) {
    double o[3] = {ox, oy, oz};
    if (use_com && M[0] != 0.0) {
      o[0] = M[1] / M[0];
      o[1] = M[2] / M[0];
      o[2] = M[3] / M[0];
    }
    for (int d = 0; d < 3; ++d) {
      P[d][0] = 1.0;
      for (int p = 1; p < 5; ++p) P[d][p] = P[d][p - 1] * -o[d];
      out[25 + d] = o[d];
    }
  }
  __syncthreads();
  // moments about o: C_q = sum over r <= q of the binomial shifts (one
  // monomial per thread)
  for (int q = threadIdx.x; q < kMono; q += blockDim.x) {
    const int a = c_mono[q][0], b = c_mono[q][1], c = c_mono[q][2];
    double acc = 0.0;
    for (int r = 0; r < kMono; ++r) {
      const int a2 = c_mono[r][0], b2 = c_mono[r][1], c2 = c_mono[r][2];
      if (a2 > a || b2 > b || c2 > c) continue;
      const double w = binom(a, a2) * binom(b, b2) * binom(c, c2) * P[0][a - a2] *
                       P[1][b - b2] * P[2][c - c2];
      acc += w * M[r];
    }
    Cs[q] = acc;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double dv = h * h * h;
  const double* C = Cs;
  const double pi = 3.14159265358979323846;
  double Q[kTerms];
  for (int q = 0; q < kTerms; ++q) Q[q] = 0.0;
  for (int t = 0; t < c_nterm; ++t) Q[c_term_lm[t]] += c_term_coef[t] * C[c_term_mono[t]];
  for (int l = 0; l <= 4; ++l)
    for (int m = -l; m <= l; ++m) {
      const int q = l * l + m + l;
      Q[q] = (l <= lmax) ? Q[q] * dv * sqrt(4.0 * pi / (2.0 * l + 1.0)) : 0.0;
    }
  for (int q = 0; q < kTerms; ++q) out[q] = Q[q];
  out[28] = M[0] * dv;
}

// Potential of the expansion at every face point of a level.  The block first
// folds the moments into the coefficient of each monomial of the potential's
// degree-l parts (P_l = sqrt(4 pi / (2l + 1)) sum_m Q_lm r^l Y_lm, homogeneous
// of degree l), so that a point costs the 35 monomials at compile-time
// indices and one reciprocal square root: phi = -G sum_l P_l / r^(2l+1).
__global__ void k_open_faces(Grid g, double h, const double* __restrict__ qo, int lmax, double G,
                             double* __restrict__ faces) {
  __shared__ double A[kMono];
  const double pi = 3.14159265358979323846;
  for (int q = threadIdx.x; q < kMono; q += blockDim.x) {
    const int l = c_mono[q][0] + c_mono[q][1] + c_mono[q][2];
    double a = 0.0;
    for (int t = 0; t < c_nterm; ++t)
      if (c_term_mono[t] == q) a += qo[c_term_lm[t]] * c_term_coef[t];
    A[q] = l <= lmax ? a * sqrt(4.0 * pi / (2.0 * l + 1.0)) : 0.0;
  }
  __syncthreads();
  const long long fx = (long long)(g.ny + 2) * (g.nz + 2), fy = (long long)(g.nx + 2) * (g.nz + 2),
                  fz = (long long)(g.nx + 2) * (g.ny + 2);
  const long long total = 2 * (fx + fy + fz);
  const double ox = qo[25], oy = qo[26], oz = qo[27];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long q = t;
    int face, na;
    if (q < 2 * fx) { face = (int)(q / fx); q %= fx; na = g.ny + 2; }
    else if (q < 2 * fx + 2 * fy) { q -= 2 * fx; face = 2 + (int)(q / fy); q %= fy; na = g.nx + 2; }
    else { q -= 2 * fx + 2 * fy; face = 4 + (int)(q / fz); q %= fz; na = g.nx + 2; }
    const int a = (int)(q % na), b = (int)(q / na);
    const double side = (face & 1) ? 0.5 : -0.5;
    double x, y, z;
    if (face < 2) {
      x = side * g.nx * h; y = ((double)a - 0.5 - 0.5 * g.ny) * h; z = ((double)b - 0.5 - 0.5 * g.nz) * h;
    } else if (face < 4) {
      x = ((double)a - 0.5 - 0.5 * g.nx) * h; y = side * g.ny * h; z = ((double)b - 0.5 - 0.5 * g.nz) * h;
    } else {
      x = ((double)a - 0.5 - 0.5 * g.nx) * h; y = ((double)b - 0.5 - 0.5 * g.ny) * h; z = side * g.nz * h;
    }
    x -= ox; y -= oy; z -= oz;
    const double r2 = x * x + y * y + z * z;
    double xp[5], yp[5], zp[5];
    xp[0] = yp[0] = zp[0] = 1.0;
#pragma unroll
    for (int p = 1; p < 5; ++p) { xp[p] = xp[p - 1] * x; yp[p] = yp[p - 1] * y; zp[p] = zp[p - 1] * z; }
    // the monomials in the order of c_mono: degree, then a, then b descending
    double P[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    int m = 0;
#pragma unroll
    for (int d = 0; d <= 4; ++d)
#pragma unroll
      for (int ea = d; ea >= 0; --ea)
#pragma unroll
        for (int eb = d - ea; eb >= 0; --eb) {
          P[d] += A[m] * (xp[ea] * yp[eb] * zp[d - ea - eb]);
          ++m;
        }
    const double ir = 1.0 / sqrt(r2), ir2 = ir * ir;
    double phi = 0.0, w = ir;  // 1 / r^(2l+1)
#pragma unroll
    for (int l = 0; l <= 4; ++l) {
      phi += P[l] * w;
      w *= ir2;
    }
    faces[t] = -G * phi;
  }
}

// A start value for phi under the open rule: the expansion's monopole and
// dipole, -G (P_0 / r + P_1 / r^3), at every cell, with r at least rmin (the
// expansion is singular at its origin).  It matches the face potentials up to
// the quadrupole and higher terms, so the first residual has no boundary
// layer; its accuracy inside does not matter (the outer loop corrects it
// exactly), and FP32 arithmetic suffices.
__global__ void k_open_guess(double* __restrict__ phi, Grid g, double h,
                             const double* __restrict__ qo, double G, float rmin) {
  __shared__ float A[4];  // coefficients of 1, x, y, z (the first four monomials)
  const double pi = 3.14159265358979323846;
  if (threadIdx.x < 4) {
    const int q = threadIdx.x, l = q == 0 ? 0 : 1;
    double a = 0.0;
    for (int t = 0; t < c_nterm; ++t)
      if (c_term_mono[t] == q) a += qo[c_term_lm[t]] * c_term_coef[t];
    A[q] = (float)(-G * a * sqrt(4.0 * pi / (2.0 * l + 1.0)));
  }
  __syncthreads();
  const float ox = (float)qo[25], oy = (float)qo[26], oz = (float)qo[27], hf = (float)h;
  const float cx = 0.5f * g.nx, cy = 0.5f * g.ny, cz = 0.5f * g.nz;
  const long long total = g.cells();
  const dev::Split sp(g.nx, g.ny);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    sp(t, i, j, k);
    const float x = ((float)i + 0.5f - cx) * hf - ox, y = ((float)j + 0.5f - cy) * hf - oy,
                z = ((float)k + 0.5f - cz) * hf - oz;
    const float r = fmaxf(sqrtf(x * x + y * y + z * z), rmin), ir = 1.0f / r;
    phi[t] = (double)((A[0] + (A[1] * x + A[2] * y + A[3] * z) * ir * ir) * ir);
  }
}

}  // namespace

cudaError_t prepare_multipole() { return upload_tables(); }

cudaError_t launch_open_guess(double* phi, Grid g, double h, const double* qo, double G,
                              cudaStream_t s) {
  cudaError_t e = upload_tables();
  if (e != cudaSuccess) return e;
  ++g_launches;
  long long nb = (g.cells() + kThreads - 1) / kThreads;
  if (nb > sm_count() * 16LL) nb = sm_count() * 16LL;
  // r at least 1/8 of the shortest side: inside that the start value is flat
  // (a larger value there would only coarsen the fixed-point scale chosen from
  // max |phi|)
  const int nmin = g.nx < g.ny ? (g.nx < g.nz ? g.nx : g.nz) : (g.ny < g.nz ? g.ny : g.nz);
  k_open_guess<<<(int)nb, kThreads, 0, s>>>(phi, g, h, qo, G, (float)(0.125 * nmin * h));
  return cudaGetLastError();
}

cudaError_t launch_raw_moments(const double* rho, Grid g, double h, double* partials, int* nb_out,
                               cudaStream_t s) {
  cudaError_t e = upload_tables();
  if (e != cudaSuccess) return e;
  const long long rows = (long long)g.ny * g.nz;
  long long nb = (rows + kWarps - 1) / kWarps;
  if (nb > kMaxReduceBlocks / 4) nb = kMaxReduceBlocks / 4;  // partials: nb * 35 doubles
  *nb_out = (int)nb;
  ++g_launches;
  k_raw_moments<<<(int)nb, kThreads, 0, s>>>(rho, g, h, partials);
  return cudaGetLastError();
}

cudaError_t launch_raw_moments_blocks(const double* rho, Grid g, double h, double* partials,
                                     int nb, cudaStream_t s) {
  cudaError_t e = upload_tables();
  if (e != cudaSuccess) return e;
  ++g_launches;
  k_raw_moments<<<nb, kThreads, 0, s>>>(rho, g, h, partials);
  return cudaGetLastError();
}

cudaError_t launch_moments_finish(const double* partials, int nb, double h, int lmax, int use_com,
                                  const double* origin_in, double* out, cudaStream_t s) {
  cudaError_t e = upload_tables();
  if (e != cudaSuccess) return e;
  ++g_launches;
  k_moments_finish<<<1, 64, 0, s>>>(partials, nb, h, lmax, use_com, origin_in[0], origin_in[1],
                                    origin_in[2], out);
  return cudaGetLastError();
}

cudaError_t launch_open_faces(Grid g, double h, const double* qo, int lmax, double G,
                              double* faces, cudaStream_t s) {
  cudaError_t e = upload_tables();
  if (e != cudaSuccess) return e;
  const long long total = (long long)faces_count(g);
  long long nb = (total + kThreads - 1) / kThreads;
  if (nb > sm_count() * 16LL) nb = sm_count() * 16LL;
  ++g_launches;
  k_open_faces<<<(int)nb, kThreads, 0, s>>>(g, h, qo, lmax, G, faces);
  return cudaGetLastError();
}

}  // namespace mg
