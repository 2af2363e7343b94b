// tma.cuh -- inline-PTX helpers for mbarrier-tracked TMA tile loads
// (cp.async.bulk.tensor) on sm_103a, and the host-side tensor-map encoder
// obtained from the driver at run time.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mithra {

__device__ inline uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

// makes the initialised barriers visible to the async (TMA) proxy
__device__ inline void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ inline void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ inline void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ inline bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Waits for phase `parity` of bar with an iteration limit; on timeout sets bit
// 1 of *err and returns false (the caller carries on; the result is flagged).
__device__ inline bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* err) {
  for (long long it = 0; it < (1LL << 24); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  atomicOr(err, 2);
  return false;
}

// orders earlier generic-proxy accesses of shared memory before later
// async-proxy (TMA) writes to it
// Per-thread asynchronous copy of 4 or 8 bytes from global to shared memory
// (cp.async, cached in L1); cp_async_commit closes a group of them,
// cp_async_wait_all waits for all of this thread's groups.
template <int kBytes>
__device__ inline void cp_async(void* dst, const void* src) {
  static_assert(kBytes == 4 || kBytes == 8, "cp.async.ca copies 4, 8 or 16 bytes");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_addr(dst)), "l"(src),
               "n"(kBytes)
               : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ inline void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 3-D tiled TMA load of one box of a field map (encode_field_map) into shared
// memory, completion counted in bytes on bar.  (i, j, k) is the box's first
// vertex; the four components of a vertex are folded into the innermost
// dimension (element 4 i), so the inner coordinate is 16 or 32 bytes times
// i: a multiple of 16 bytes for every i, negative ones included.
__device__ inline void tma_load_field(void* dst, const CUtensorMap* tm, int i, int j, int k,
                                      uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(4 * i), "r"(j), "r"(k), "r"(smem_addr(bar))
      : "memory");
}

// ---------------------------------------------------------------------------
// host side

typedef CUresult (*TensorMapEncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                         const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                         const cuuint32_t*, CUtensorMapInterleave,
                                         CUtensorMapSwizzle, CUtensorMapL2promotion,
                                         CUtensorMapFloatOOBfill);

inline TensorMapEncodeTiled tensor_map_encoder() {
  static TensorMapEncodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<TensorMapEncodeTiled>(p);
  }
  return fn;
}

// Tensor map of a 4-component field array (nx*ny*nz vertices of 4 values of
// elem_bytes each, x fastest) with a box of bx x by x bz vertices.  The map
// is 3-D with the components folded into x (4 nx values per row, boxes of
// 4 bx): the TMA unit then moves rows of 4 bx values instead of one vertex
// (16 or 32 bytes) at a time.
inline bool encode_field_map(CUtensorMap* tm, void* base, int elem_bytes, int nx, int ny, int nz,
                             int bx, int by, int bz = 1) {
  TensorMapEncodeTiled enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t row = 4ull * elem_bytes * nx;
  const cuuint64_t dims[3] = {4ull * nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {row, row * ny};
  const cuuint32_t box[3] = {4u * bx, (cuuint32_t)by, (cuuint32_t)bz};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(tm, elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                       : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                   3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace mithra
