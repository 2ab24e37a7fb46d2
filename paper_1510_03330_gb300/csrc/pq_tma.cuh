// Tensor Memory Accelerator (TMA) building blocks in inline PTX for sm_103a:
// tiled tensor loads into shared memory with mbarrier transaction counting,
// and the host-side encoding of the tensor maps (driver entry point
// cuTensorMapEncodeTiled).
//
// Every load in this library starts at an innermost coordinate that is a
// multiple of 8 BF16 elements (16 bytes) and targets a 1024-byte aligned
// shared-memory address, as the hardware requires.
#pragma once

#include <cuda.h>
#include <cstdint>

#include "pq_tc.cuh"

namespace pq {
namespace tma {

__device__ __forceinline__ void mbar_expect_tx(void *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(bar)), "r"(bytes)
               : "memory");
}

// 4-D tiled load of one box into shared memory; completion is counted on bar.
__device__ __forceinline__ void load4(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                      void *bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(tc::smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void load3(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, void *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(tc::smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void prefetch_map(const CUtensorMap *map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

}  // namespace tma
}  // namespace pq
