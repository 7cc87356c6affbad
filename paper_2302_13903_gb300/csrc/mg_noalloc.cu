// mg_noalloc.cu -- multipole moments without any device allocation.
//
// Some callers cannot call cudaMalloc: a host application whose device memory
// is entirely reserved by its own pool allocator and that forbids allocations
// from plugins, code that must not risk an out-of-memory failure or the
// latency of the allocator in the middle of a time step, or a process running
// under a hard device-memory budget that is already spent.  For them this
// file provides mg_op_multipole_moments_noalloc: the same moments as
// mg_op_multipole_moments, with its scratch (per-block partial sums and the
// 29-value result) held in one fixed, file-scope device array instead of
// memory allocated per call.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/mg.h"
#include "mg_internal.h"

namespace {

constexpr int kMono = 35;             // partial sums per block
constexpr int kRowsPerBlock = 32;     // 8 warps, 4 rows each
constexpr int kStaticBlocks = 8192;   // -> at most 262144 rows (ny * nz)
constexpr size_t kResultOffset = (size_t)kStaticBlocks * kMono;
constexpr size_t kStaticDoubles = kResultOffset + 32;  // 2.24 MiB in all

// Held by every device that loads the library, until the process exits.  In
// host code this name is only a stand-in; the device address comes from
// cudaGetSymbolAddress below.
__device__ __align__(256) double g_moment_scratch[kStaticDoubles];

std::mutex g_mu;
double* g_addr[64] = {};

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached.
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_moment_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

// Failures are reported through mg_last_error(NULL), like the other entry
// points without a context, and on stderr.
mg_status fail(mg_status st, const std::string& msg) {
  mg::set_last_error(msg);
  std::fprintf(stderr, "%s\n", msg.c_str());
  return st;
}

mg_status fail_cuda(cudaError_t e, const char* what) {
  return fail(MG_ERR_CUDA, std::string("mg_op_multipole_moments_noalloc: ") + what + ": " +
                               cudaGetErrorString(e));
}

}  // namespace

extern "C" mg_status mg_op_multipole_moments_noalloc(int nx, int ny, int nz, double h,
                                                     const double* rho_dev, int lmax, int use_com,
                                                     double* origin_host, double* Q_host,
                                                     void* stream) {
  if (nx < 1 || ny < 1 || nz < 1 || !(h > 0.0) || !rho_dev || !origin_host || !Q_host ||
      lmax < 0 || lmax > 4)
    return fail(MG_ERR_ARG, "mg_op_multipole_moments_noalloc: invalid argument");
  const long long rows = (long long)ny * nz;
  const long long nb = (rows + kRowsPerBlock - 1) / kRowsPerBlock;
  if (nb > kStaticBlocks)
    return fail(MG_ERR_ARG, "mg_op_multipole_moments_noalloc: grid has " +
                                std::to_string(rows) + " rows (ny*nz); the fixed scratch holds at "
                                "most " + std::to_string(kStaticBlocks * kRowsPerBlock) +
                                " rows -- use mg_op_multipole_moments instead");
  cudaStream_t s = (cudaStream_t)stream;
  double* scratch = nullptr;
  cudaError_t e = mg::prepare_multipole();  // constant tables, once per device
  if (e != cudaSuccess) return fail_cuda(e, "constant tables");
  e = scratch_address(&scratch);
  if (e != cudaSuccess) return fail_cuda(e, "cudaGetSymbolAddress");
  // Every block writes all 35 of its partial sums, and the finishing kernel
  // reads only what this call wrote, so nothing needs clearing first.
  const mg::Grid g{nx, ny, nz};
  e = mg::launch_raw_moments_blocks(rho_dev, g, h, scratch, (int)nb, s);
  if (e != cudaSuccess) return fail_cuda(e, "moments kernel");
  e = mg::launch_moments_finish(scratch, (int)nb, h, lmax, use_com, origin_host,
                                scratch + kResultOffset, s);
  if (e != cudaSuccess) return fail_cuda(e, "finish kernel");
  double result[29];
  e = cudaMemcpyAsync(result, scratch + kResultOffset, sizeof result, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_cuda(e, "copy result");
  std::memcpy(Q_host, result, 25 * sizeof(double));
  std::memcpy(origin_host, result + 25, 3 * sizeof(double));
  return MG_OK;
}
