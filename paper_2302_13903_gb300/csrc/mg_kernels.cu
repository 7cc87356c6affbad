// mg_kernels.cu -- per-level multigrid kernels for sm_103a (FP64 and FP32).
//
// Layout: every level is an nx*ny*nz array of active cells, z-major, x
// fastest; there are no ghost cells in memory.  A neighbour outside the level
// is synthesised from the boundary rule at load time (Sec. 2.3.6): periodic
// wraps, zero gradient copies the adjacent cell, fixed / open give
// 2 b - (adjacent cell) with b the value on the face.  Where a stencil leaves
// the level along more than one axis (edges and corners of the 27-point
// prolongations) the face rule is applied along x, then y, then z.
//
// These are the straightforward kernels: one thread per output cell (or per
// coarse cell for the fused defect + restriction), grid-stride loops over the
// bodies in mg_device.cuh, and deterministic two-stage reductions.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "mg_device.cuh"
#include "mg_internal.h"

namespace mg {

thread_local long long g_launches = 0;

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum (blockDim.x == kThreads); result valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[kThreads / 32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) ws[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = lane < kThreads / 32 ? ws[lane] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;
}

int grid_for(long long work) {
  long long b = (work + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  if (b > sm_count() * 64LL) b = sm_count() * 64LL;
  return (int)b;
}

// ---------------------------------------------------------------------------
// d = f - (sum_nb - 6u) / h^2; optional store and partial sums of d^2.
template <typename T>
__global__ void k_defect(const T* __restrict__ u, const T* __restrict__ f, T* __restrict__ d,
                         Grid g, Bc bc, T inv_h2, double* __restrict__ partials) {
  const long long total = g.cells();
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.nx);
    const long long r = t / g.nx;
    const int j = (int)(r % g.ny), k = (int)(r / g.ny);
    const T s = dev::neighbour_sum(u, i, j, k, g, bc);
    const T dv = f[t] - (s - T(6) * u[t]) * inv_h2;
    if (d) d[t] = dv;
    acc += (double)dv * (double)dv;
  }
  if (partials) {
    const double b = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = b;
  }
}

template <typename T>
__global__ void k_sor(T* u, const T* f, Grid g, Bc bc, T cu, T cs, T cf, int colour) {
  dev::sor_range(u, f, g, bc, cu, cs, cf, colour, blockIdx.x * (long long)blockDim.x + threadIdx.x,
                 (long long)gridDim.x * blockDim.x);
}

template <typename T>
__global__ void k_sor_red_zero(T* u, const T* f, Grid g, T cf) {
  dev::sor_red_zero_range(u, f, g, cf, blockIdx.x * (long long)blockDim.x + threadIdx.x,
                          (long long)gridDim.x * blockDim.x);
}

template <typename T>
__global__ void k_defect_restrict(const T* u, const T* f, T* fc, Grid g, Bc bc, T inv_h2) {
  dev::defect_restrict_range(u, f, fc, g, bc, inv_h2,
                             blockIdx.x * (long long)blockDim.x + threadIdx.x,
                             (long long)gridDim.x * blockDim.x);
}

template <typename T>
__global__ void k_restrict(const T* uf, T* uc, Grid gf) {
  dev::restrict_range(uf, uc, gf, blockIdx.x * (long long)blockDim.x + threadIdx.x,
                      (long long)gridDim.x * blockDim.x);
}

template <typename T, bool HIGH>
__global__ void k_prolong(const T* uc, T* uf, Grid gf, Bc bc, int add, int cz, long long items) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < items;
       t += (long long)gridDim.x * blockDim.x)
    dev::prolong_zchunk<T, HIGH>(uc, uf, gf, bc, add, t, cz);
}

template <typename T>
__global__ void k_coarsest(const T* f, T* u, double h, Bc bc, bool keep) {
  if (threadIdx.x == 0 && blockIdx.x == 0) dev::coarsest_one(f, u, h, bc, keep);
}

template <typename T>
__global__ void k_fill(T* __restrict__ u, long long n, T v) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    u[t] = v;
}

__global__ void k_add_const(double* __restrict__ u, long long n, double v) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    u[t] += v;
}

__global__ void k_source(const double* __restrict__ rho, double* __restrict__ f, long long n,
                         double four_pi_G, double* __restrict__ partials) {
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const double v = four_pi_G * rho[t];
    f[t] = v;
    acc += v;
  }
  const double b = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = b;
}

template <typename T>
__global__ void k_sum(const T* __restrict__ a, long long n, int squares,
                      double* __restrict__ partials) {
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const double v = (double)a[t];
    acc += squares ? v * v : v;
  }
  const double b = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = b;
}

__global__ void k_finish_sum(const double* __restrict__ partials, int nb, double* __restrict__ out) {
  double acc = 0.0;
  for (int t = threadIdx.x; t < nb; t += blockDim.x) acc += partials[t];
  const double b = block_sum(acc);
  if (threadIdx.x == 0) out[0] = b;
}

// a -= total[0] / n (the total was formed on the device in a fixed order).
__global__ void k_subtract_mean(double* __restrict__ a, long long n, const double* __restrict__ total) {
  const double mean = total[0] / (double)n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    a[t] -= mean;
}

__global__ void k_outer_residual(const double* __restrict__ u, const double* __restrict__ f,
                                 float* __restrict__ r32, Grid g, Bc bc, double inv_h2,
                                 double scale, double* __restrict__ partials) {
  const long long total = g.cells();
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.nx);
    const long long r = t / g.nx;
    const int j = (int)(r % g.ny), k = (int)(r / g.ny);
    const double s = dev::neighbour_sum(u, i, j, k, g, bc);
    const double d = f[t] - (s - 6.0 * u[t]) * inv_h2;
    r32[t] = (float)(d * scale);
    acc += d * d;
  }
  const double b = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = b;
}

__global__ void k_scale_to_f32(const double* __restrict__ a, float* __restrict__ b, long long n,
                               double scale) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    b[t] = (float)(scale * a[t]);
}

__global__ void k_correct(double* __restrict__ u, const float* __restrict__ e, long long n,
                          double inv_scale) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    u[t] += inv_scale * (double)e[t];
}

// Algorithm 3 step 5 on a coarse level: f += L ur (the restricted potential's
// Laplacian with the level's own rule) and the start value u = ur.
__global__ void k_fas_rhs(const double* __restrict__ ur, double* __restrict__ f,
                          double* __restrict__ u, Grid g, Bc bc, double inv_h2) {
  const long long total = g.cells();
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.nx);
    const long long r = t / g.nx;
    const int j = (int)(r % g.ny), k = (int)(r / g.ny);
    const double s = dev::neighbour_sum(ur, i, j, k, g, bc);
    f[t] += (s - 6.0 * ur[t]) * inv_h2;
    u[t] = ur[t];
  }
}

// Algorithm 3 step 7: u -= ur (the coarse-grid correction).
__global__ void k_sub(double* __restrict__ u, const double* __restrict__ ur, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    u[t] -= ur[t];
}

// g = -grad phi at cell centres (Sec. 3.2.3): per axis the average of the two
// face accelerations -(phi_{i+1} - phi_i) / h and -(phi_i - phi_{i-1}) / h,
// neighbours outside the level from the rule; g = [g_x | g_y | g_z].
__global__ void k_gravity(const double* __restrict__ u, double* __restrict__ g, Grid gr, Bc bc,
                          double h) {
  const long long total = gr.cells();
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % gr.nx);
    const long long r = t / gr.nx;
    const int j = (int)(r % gr.ny), k = (int)(r / gr.ny);
    const double c = u[t];
    const double xl = -(c - dev::fetch(u, i - 1, j, k, gr, bc)) / h;
    const double xr = -(dev::fetch(u, i + 1, j, k, gr, bc) - c) / h;
    const double yl = -(c - dev::fetch(u, i, j - 1, k, gr, bc)) / h;
    const double yr = -(dev::fetch(u, i, j + 1, k, gr, bc) - c) / h;
    const double zl = -(c - dev::fetch(u, i, j, k - 1, gr, bc)) / h;
    const double zr = -(dev::fetch(u, i, j, k + 1, gr, bc) - c) / h;
    g[t] = 0.5 * (xl + xr);
    g[total + t] = 0.5 * (yl + yr);
    g[2 * total + t] = 0.5 * (zl + zr);
  }
}

}  // namespace

int sm_count() {
  static std::atomic<int> cached[64];  // zero-initialised (static storage)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 152;
  }
  int n = cached[dev].load();
  if (n == 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
      cudaGetLastError();
      n = 152;
    }
    cached[dev].store(n);
  }
  return n;
}

int reduce_blocks(long long n) {
  long long b = (n + kThreads * 4 - 1) / (kThreads * 4);
  if (b < 1) b = 1;
  if (b > kMaxReduceBlocks) b = kMaxReduceBlocks;
  return (int)b;
}

template <typename T>
cudaError_t launch_sor(T* u, const T* f, Grid g, double h, Bc bc, double omega, int colour,
                       cudaStream_t s) {
  const long long work = (long long)(g.nx / 2) * g.ny * g.nz;
  ++g_launches;
  k_sor<T><<<grid_for(work), kThreads, 0, s>>>(u, f, g, bc, (T)(1.0 - omega), (T)(omega / 6.0),
                                               (T)(-omega * h * h / 6.0), colour);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sor_red_zero(T* u, const T* f, Grid g, double h, double omega,
                                cudaStream_t s) {
  ++g_launches;
  k_sor_red_zero<T><<<grid_for(g.cells()), kThreads, 0, s>>>(u, f, g, (T)(-omega * h * h / 6.0));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_defect(const T* u, const T* f, T* d, Grid g, double h, Bc bc, double* partials,
                          cudaStream_t s) {
  ++g_launches;
  const int nb = partials ? reduce_blocks(g.cells()) : grid_for(g.cells());
  k_defect<T><<<nb, kThreads, 0, s>>>(u, f, d, g, bc, (T)(1.0 / (h * h)), partials);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_defect_restrict(const T* u, const T* f, T* fc, Grid g, double h, Bc bc,
                                   cudaStream_t s) {
  ++g_launches;
  k_defect_restrict<T><<<grid_for(g.cells() / 8), kThreads, 0, s>>>(u, f, fc, g, bc,
                                                                    (T)(1.0 / (h * h)));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict(const T* uf, T* uc, Grid gf, cudaStream_t s) {
  ++g_launches;
  k_restrict<T><<<grid_for(gf.cells() / 8), kThreads, 0, s>>>(uf, uc, gf);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong(const T* uc, T* uf, Grid gf, Bc bc_coarse, int high_order, int add,
                           cudaStream_t s) {
  ++g_launches;
  // z-chunks of coarse columns: 8 planes each while that leaves about 2^18
  // work items (enough threads for the device), fewer on small levels
  const long long cols = (long long)(gf.nx / 2) * (gf.ny / 2);
  const int cnz = gf.nz / 2;
  int cz = 8;
  while (cz > 1 && cols * ((cnz + cz - 1) / cz) < (1LL << 18)) cz /= 2;
  const long long items = cols * ((cnz + cz - 1) / cz);
  if (high_order)
    k_prolong<T, true><<<grid_for(items), kThreads, 0, s>>>(uc, uf, gf, bc_coarse, add, cz, items);
  else
    k_prolong<T, false><<<grid_for(items), kThreads, 0, s>>>(uc, uf, gf, bc_coarse, add, cz, items);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarsest(const T* f, T* u, double h, Bc bc, cudaStream_t s, bool keep) {
  ++g_launches;
  k_coarsest<T><<<1, 32, 0, s>>>(f, u, h, bc, keep);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fill(T* u, long long n, T v, cudaStream_t s) {
  ++g_launches;
  k_fill<T><<<grid_for(n), kThreads, 0, s>>>(u, n, v);
  return cudaGetLastError();
}

cudaError_t launch_source(const double* rho, double* f, long long n, double four_pi_G,
                          double* partials, cudaStream_t s) {
  ++g_launches;
  k_source<<<reduce_blocks(n), kThreads, 0, s>>>(rho, f, n, four_pi_G, partials);
  return cudaGetLastError();
}

cudaError_t launch_subtract_mean(double* a, long long n, const double* partials, int nb,
                                 double* total_slot, cudaStream_t s) {
  ++g_launches;
  k_finish_sum<<<1, kThreads, 0, s>>>(partials, nb, total_slot);
  ++g_launches;
  k_subtract_mean<<<grid_for(n), kThreads, 0, s>>>(a, n, total_slot);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sum(const T* a, long long n, int squares, double* partials, cudaStream_t s) {
  ++g_launches;
  k_sum<T><<<reduce_blocks(n), kThreads, 0, s>>>(a, n, squares, partials);
  return cudaGetLastError();
}

cudaError_t launch_fas_rhs(const double* ur, double* f, double* u, Grid g, double h, Bc bc,
                           cudaStream_t s) {
  ++g_launches;
  k_fas_rhs<<<grid_for(g.cells()), kThreads, 0, s>>>(ur, f, u, g, bc, 1.0 / (h * h));
  return cudaGetLastError();
}

cudaError_t launch_sub(double* u, const double* ur, long long n, cudaStream_t s) {
  ++g_launches;
  k_sub<<<grid_for(n), kThreads, 0, s>>>(u, ur, n);
  return cudaGetLastError();
}

cudaError_t launch_gravity(const double* u, double* g, Grid gr, double h, Bc bc, cudaStream_t s) {
  ++g_launches;
  k_gravity<<<grid_for(gr.cells()), kThreads, 0, s>>>(u, g, gr, bc, h);
  return cudaGetLastError();
}

cudaError_t launch_finish_sum(const double* partials, int nb, double* out, cudaStream_t s) {
  ++g_launches;
  k_finish_sum<<<1, kThreads, 0, s>>>(partials, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_outer_residual(const double* u, const double* f, float* r32, Grid g, double h,
                                  Bc bc, double scale, double* partials, cudaStream_t s) {
  ++g_launches;
  k_outer_residual<<<reduce_blocks(g.cells()), kThreads, 0, s>>>(u, f, r32, g, bc, 1.0 / (h * h),
                                                                 scale, partials);
  return cudaGetLastError();
}

cudaError_t launch_add_const(double* u, long long n, double v, cudaStream_t s) {
  ++g_launches;
  k_add_const<<<grid_for(n), kThreads, 0, s>>>(u, n, v);
  return cudaGetLastError();
}

cudaError_t launch_scale_to_f32(const double* a, float* b, long long n, double scale,
                               cudaStream_t s) {
  ++g_launches;
  k_scale_to_f32<<<grid_for(n), kThreads, 0, s>>>(a, b, n, scale);
  return cudaGetLastError();
}

cudaError_t launch_correct(double* u, const float* e32, long long n, double inv_scale,
                           cudaStream_t s) {
  ++g_launches;
  k_correct<<<grid_for(n), kThreads, 0, s>>>(u, e32, n, inv_scale);
  return cudaGetLastError();
}

#define MG_INSTANTIATE(T)                                                                        \
  template cudaError_t launch_sor<T>(T*, const T*, Grid, double, Bc, double, int, cudaStream_t); \
  template cudaError_t launch_sor_red_zero<T>(T*, const T*, Grid, double, double, cudaStream_t); \
  template cudaError_t launch_defect<T>(const T*, const T*, T*, Grid, double, Bc, double*,       \
                                        cudaStream_t);                                           \
  template cudaError_t launch_defect_restrict<T>(const T*, const T*, T*, Grid, double, Bc,       \
                                                 cudaStream_t);                                  \
  template cudaError_t launch_restrict<T>(const T*, T*, Grid, cudaStream_t);                     \
  template cudaError_t launch_prolong<T>(const T*, T*, Grid, Bc, int, int, cudaStream_t);        \
  template cudaError_t launch_coarsest<T>(const T*, T*, double, Bc, cudaStream_t, bool);         \
  template cudaError_t launch_fill<T>(T*, long long, T, cudaStream_t);                           \
  template cudaError_t launch_sum<T>(const T*, long long, int, double*, cudaStream_t);

MG_INSTANTIATE(float)
MG_INSTANTIATE(double)

}  // namespace mg
