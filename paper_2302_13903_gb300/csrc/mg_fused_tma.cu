// mg_fused_tma.cu -- the fused FP32 legs of a periodic level with their
// planes of u and f brought into shared memory by tensor copies
// (cp.async.bulk.tensor) in place of per-thread 16-byte cp.async: one thread
// of the CTA issues one copy per array and plane, and an mbarrier per ring
// slot counts the bytes that land.  Tiles whose window wraps around the level
// keep the per-thread copies.  The down leg (steps 1-3 of Algorithm 1) runs on
// 64 x 32 tiles; from a zero start (only f is read) its issuing thread also
// asks L2 for the planes two steps beyond the ring
// (cp.async.bulk.prefetch.tensor).  The up leg (steps 5-7) runs on 64 x 16
// tiles; its coarse planes keep per-thread copies.  Same arithmetic as the
// legs with per-thread copies, so the same bits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>

#include "mg_fused.cuh"
#include "mg_internal.h"

namespace mg {
namespace {

using fused::FusedParams;
using S32 = fused::Shape<fused::kDown, 64, 32>;
using SUp = fused::Shape<fused::kUp, 64, 16>;
static_assert(S32::PLS * 16 % 128 == 0 && SUp::PLS * 16 % 128 == 0, "ring slots on 128 bytes");
static_assert(4 * S32::RS <= 256 && S32::RR <= 256 && 4 * SUp::RS <= 256 && SUp::RR <= 256,
              "a tensor-copy box side is at most 256");

// The down leg's L2 prefetch distance beyond the ring, in planes: 2 from a
// zero start (where it measured faster), none otherwise (measured slower).
template <bool ZERO>
constexpr int kPrefetch = ZERO ? 2 : 0;

template <bool ZERO>
__global__ void __maxnreg__((fused::fused_max_regs<fused::kDown, 32>()))
    k_fused_down_tma(const float* __restrict__ u_in, float* __restrict__ u_out,
                     const float* __restrict__ f, float* __restrict__ fc, FusedParams p,
                     const __grid_constant__ CUtensorMap tmu,
                     const __grid_constant__ CUtensorMap tmf, int* err) {
  extern __shared__ float4 smem_tma[];
  // tensor copies land on 128-byte boundaries: round the base up (the launch
  // gives 128 bytes more than the shape needs)
  const unsigned off = (unsigned)__cvta_generic_to_shared(smem_tma);
  float4* base = smem_tma + ((128u - (off & 127u)) & 127u) / 16u;
  fused::fused_tile<fused::kDown, ZERO, 7, 64, 32, 0, true, 0, true, kPrefetch<ZERO>>(
      u_in, u_out, f, nullptr, fc, p, blockIdx.x, blockIdx.y, blockIdx.z, base, &tmu, &tmf, err);
}

// the up leg's L2 prefetch distance: none (2 and 4 planes measured slower)
constexpr int kPrefetchUp = 0;

__global__ void __maxnreg__((fused::fused_max_regs<fused::kUp, 16>()))
    k_fused_up_tma(const float* __restrict__ u_in, float* __restrict__ u_out,
                   const float* __restrict__ f, const float* __restrict__ ec, FusedParams p,
                   const __grid_constant__ CUtensorMap tmu,
                   const __grid_constant__ CUtensorMap tmf, int* err) {
  extern __shared__ float4 smem_tma[];
  const unsigned off = (unsigned)__cvta_generic_to_shared(smem_tma);
  float4* base = smem_tma + ((128u - (off & 127u)) & 127u) / 16u;
  fused::fused_tile<fused::kUp, false, 7, 64, 16, 0, true, 0, true, kPrefetchUp>(
      u_in, u_out, f, ec, nullptr, p, blockIdx.x, blockIdx.y, blockIdx.z, base, &tmu, &tmf, err);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    cudaGetLastError();
  });
  return fn;
}

// A map of an nx * ny * nz FP32 level whose box is one ring slot of shape SH:
// 4 RS columns by RR rows by one plane; elements outside the level read as
// zero.  The driver checks the base (16-byte aligned) and the strides.
template <typename SH>
cudaError_t plane_map(CUtensorMap* m, const float* a, Grid g) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
  const cuuint64_t strides[2] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.nx * g.ny * 4};
  const cuuint32_t box[3] = {(cuuint32_t)(4 * SH::RS), (cuuint32_t)SH::RR, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(a), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

int* down_tma_op_flag() {
  static std::once_flag once;
  static int* flag = nullptr;
  std::call_once(once, [] {
    void* ptr = nullptr;
    if (cudaHostAlloc(&ptr, sizeof(int), cudaHostAllocMapped | cudaHostAllocPortable) ==
        cudaSuccess) {
      *static_cast<volatile int*>(ptr) = 0;
      flag = static_cast<int*>(ptr);
    }
    cudaGetLastError();
  });
  return flag;
}

bool down_tma_ok(Grid g, const Bc& bc) {
  return fused_ok(g, bc) && bc.kind == BC_PERIODIC && g.nx % 64 == 0 && g.ny % 32 == 0 &&
         encode_fn() != nullptr;
}

cudaError_t launch_fused_down_tma(const float* u_in, float* u_out, const float* f, float* fc,
                                  Grid g, double h, double omega, bool zero_guess, int cz,
                                  int* err, cudaStream_t s) {
  if (!down_tma_ok(g, Bc{BC_PERIODIC, 0.0, nullptr, 0}) || !err || !f || !u_out || !fc ||
      (!zero_guess && !u_in))
    return cudaErrorInvalidValue;
  FusedParams p = fused::params(g, h, Bc{BC_PERIODIC, 0.0, nullptr, 0}, omega);
  p.cz = fused::chunk_planes(p, 64, 32, cz);
  if (!fused_cfg_ok(g, TileCfg{64, cz, 32})) return cudaErrorInvalidValue;
  CUtensorMap mu{}, mf{};
  cudaError_t e = plane_map<S32>(&mf, f, g);
  if (e == cudaSuccess && !zero_guess) e = plane_map<S32>(&mu, u_in, g);
  if (e != cudaSuccess) return e;
  const int bytes = (int)S32::SMEM_TMA + 128;
  static std::once_flag attr_once[64];
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) return e != cudaSuccess ? e : cudaErrorInvalidValue;
  cudaError_t attr = cudaSuccess;
  std::call_once(attr_once[dev], [&] {
    attr = cudaFuncSetAttribute(k_fused_down_tma<false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(k_fused_down_tma<true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  });
  if (attr != cudaSuccess) return attr;
  const dim3 grid(g.nx / 64, g.ny / 32, (g.nz + p.cz - 1) / p.cz);
  ++g_launches;
  if (zero_guess)
    k_fused_down_tma<true><<<grid, S32::NT, bytes, s>>>(u_in, u_out, f, fc, p, mu, mf, err);
  else
    k_fused_down_tma<false><<<grid, S32::NT, bytes, s>>>(u_in, u_out, f, fc, p, mu, mf, err);
  return cudaGetLastError();
}

}  // namespace mg

namespace mg {

bool up_tma_ok(Grid g, const Bc& bc) {
  return fused_ok(g, bc) && bc.kind == BC_PERIODIC && g.nx % 64 == 0 && g.ny % 16 == 0 &&
         encode_fn() != nullptr;
}

cudaError_t launch_fused_up_tma(const float* u_in, float* u_out, const float* f, const float* ec,
                                Grid g, double h, double omega, int cz, int* err,
                                cudaStream_t s) {
  if (!up_tma_ok(g, Bc{BC_PERIODIC, 0.0, nullptr, 0}) || !err || !f || !u_out || !u_in || !ec)
    return cudaErrorInvalidValue;
  if (!fused_cfg_ok(g, TileCfg{64, cz, 16})) return cudaErrorInvalidValue;
  FusedParams p = fused::params(g, h, Bc{BC_PERIODIC, 0.0, nullptr, 0}, omega);
  p.cz = fused::chunk_planes(p, 64, 16, cz);
  CUtensorMap mu{}, mf{};
  cudaError_t e = plane_map<SUp>(&mf, f, g);
  if (e == cudaSuccess) e = plane_map<SUp>(&mu, u_in, g);
  if (e != cudaSuccess) return e;
  const int bytes = (int)SUp::SMEM_TMA + 128;
  static std::once_flag attr_once[64];
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) return e != cudaSuccess ? e : cudaErrorInvalidValue;
  cudaError_t attr = cudaSuccess;
  std::call_once(attr_once[dev], [&] {
    attr = cudaFuncSetAttribute(k_fused_up_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                bytes);
  });
  if (attr != cudaSuccess) return attr;
  const dim3 grid(g.nx / 64, g.ny / 16, (g.nz + p.cz - 1) / p.cz);
  ++g_launches;
  k_fused_up_tma<<<grid, SUp::NT, bytes, s>>>(u_in, u_out, f, ec, p, mu, mf, err);
  return cudaGetLastError();
}

}  // namespace mg
