// Tensor-memory-accelerator (TMA) staging helpers: mbarrier transaction
// barriers, tiled bulk tensor loads into shared memory, and the host-side
// encoding of the tensor maps.  Every wait is bounded: a wait that gives up
// reports false and the caller records a timeout status.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdint>

namespace lbm {

// Tensor maps of one pipelined step: populations [L][Q][ny][nx] as a 4-D
// tensor, porosity and fixed temperature [ny][nx] as 2-D tensors.
struct TmaMaps {
  CUtensorMap pop, phi, T;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
// orders earlier generic-proxy accesses of shared memory before later async-proxy (TMA) writes
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase of the given parity; false after `limit` unsuccessful probes.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit = 1 << 22) {
  for (int k = 0; k < limit; ++k)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

// ---- host side --------------------------------------------------------------

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); null when the driver does not provide it.
inline PFN_cuTensorMapEncodeTiled_v12000 tma_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// Row boxes of W elements: populations as {nx, ny, Q, L} with a box of
// {W, 1, 1, L} (one direction, every lattice), static fields as {nx, ny} with
// a box of {W, 1}.  Requires nx * sizeof(R) to be a multiple of 16 bytes and
// 16-byte aligned bases; returns false otherwise or when encoding fails.
template <class R>
bool encode_row_maps(TmaMaps& m, const R* pops, const R* phi, const R* T, int nx, int ny, int Q, int L, int W) {
  auto enc = tma_encoder();
  if (!enc || (nx * sizeof(R)) % 16 != 0) return false;
  const CUtensorMapDataType dt = sizeof(R) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const cuuint64_t s = sizeof(R), N = (cuuint64_t)nx * ny;
  auto aligned = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
  {
    cuuint64_t dim[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)Q, (cuuint64_t)L};
    cuuint64_t str[3] = {nx * s, N * s, Q * N * s};
    cuuint32_t box[4] = {(cuuint32_t)W, 1, 1, (cuuint32_t)L};
    cuuint32_t es[4] = {1, 1, 1, 1};
    if (!aligned(pops) ||
        enc(&m.pop, dt, 4, const_cast<R*>(pops), dim, str, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
            CUDA_SUCCESS)
      return false;
  }
  cuuint64_t dim2[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
  cuuint64_t str2[1] = {nx * s};
  cuuint32_t box2[2] = {(cuuint32_t)W, 1};
  cuuint32_t es2[2] = {1, 1};
  for (int k = 0; k < 2; ++k) {
    const R* src = k == 0 ? phi : T;
    CUtensorMap* dst = k == 0 ? &m.phi : &m.T;
    if (!src) {
      *dst = m.pop;                      // unused by the kernel (energy lattices carry T)
      continue;
    }
    if (!aligned(src) ||
        enc(dst, dt, 2, const_cast<R*>(src), dim2, str2, box2, es2, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
            CUDA_SUCCESS)
      return false;
  }
  return true;
}

}  // namespace lbm
