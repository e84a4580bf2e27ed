// Tensor-memory-accelerator (TMA) staging for the streaming kernels: tiled bulk-tensor loads into
// shared memory, completion tracked by an mbarrier, and bounded waits.
#pragma once

#include <cuda.h>  // CUtensorMap and its enums (the encoder is reached through the runtime)
#include <cuda_runtime.h>
#include <stdint.h>

namespace csx {

// ---------------------------------------------------------------------------------- device -----
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

// make the initialised barriers visible to the TMA unit before the first copy names them
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// one arrival that also announces `bytes` of transactions still to land in this phase
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Wait for the phase with the given parity to complete, giving up after about `max_cycles` SM
// clock cycles. Returns false on time-out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity,
                                                  long long max_cycles) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > max_cycles) return false;
  return true;
}

// Tiled loads (box set by the tensor map) into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_addr(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(smem_addr(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tma_prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];\n" ::"l"(map) : "memory");
}

// Shared-memory position of 16-byte chunk `c` of row `r` in a box written with 128-byte swizzling
// (rows of 128 bytes, buffer 1024-byte aligned): the chunk index is XORed with r mod 8, so the
// eight rows that one quarter-warp reads with 16-byte loads fall into eight distinct bank groups.
__device__ __forceinline__ int swz128(int r, int c) { return r * 8 + (c ^ (r & 7)); }
// The same for 64-byte rows written with 64-byte swizzling (buffer 512-byte aligned).
__device__ __forceinline__ int swz64(int r, int c) { return r * 4 + (c ^ ((r >> 1) & 3)); }

// ------------------------------------------------------------------------------------ host -----
// cuTensorMapEncodeTiled through the runtime's driver entry point (no link-time libcuda
// dependency). Returns 0 on success.
// dims[rank] in elements, strides_bytes[rank - 1] for dimensions 1.., box[rank] in elements.
int encode_tiled(CUtensorMap* map, CUtensorMapDataType type, unsigned rank, const void* base,
                 const cuuint64_t* dims, const cuuint64_t* strides_bytes, const cuuint32_t* box,
                 CUtensorMapSwizzle swizzle);

}  // namespace csx
