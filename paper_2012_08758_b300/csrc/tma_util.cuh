// TMA and mbarrier primitives (inline PTX, PTX ISA for sm_90+ / sm_100 family)
// shared by the TMA-staged kernels.
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "mhd_internal.h"

namespace mhd {
namespace tma {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      "  .reg .pred p;\n"
      "  mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "  selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: gives up after TRIES polls.  Each poll may suspend the
// thread for a hardware-defined time, measured by the self-test at about
// 8 us on B300, so the kernels' 2^17 polls give up after about a second.
constexpr uint32_t MAX_TRIES = 1u << 17;

template <uint32_t TRIES = MAX_TRIES>
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  for (uint32_t i = 0; i < TRIES; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0,
                                            int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
      : "memory");
}

}  // namespace tma

// Shared-memory stage of one z-plane of all seven fields of a TX x TY tile
// with its 3-point x/y halo, as one TMA box: rows of SX = TX + 8 values (the
// box starts 4 points left of the tile so that rows are 16-byte aligned).
template <typename T, int TY, int TXW = 32>
struct TmaShape {
  static constexpr int TX = TXW;     // tile width in points (32, or 64 for the paired kernel)
  static constexpr int SX = TX + 8;  // box width: x0-4 .. x0+TX+3 (16-byte multiple)
  static constexpr int SY = TY + 2 * RAD;
  static constexpr int FIELD = SX * SY;
  static constexpr int STAGE_BYTES_RAW = NF * FIELD * (int)sizeof(T);
  static constexpr int STAGE_BYTES = (STAGE_BYTES_RAW + 127) / 128 * 128;
};

}  // namespace mhd
