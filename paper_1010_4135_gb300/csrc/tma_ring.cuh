// Plane-ring staging shared by the tiled step kernels (sm_103a).
//
// A CTA owns a TX x TY column of cells.  Each z plane of all 15 fields, with
// a halo of TMA_LEFT = 4 cells in x (two are read) and two in y, arrives in
// shared memory through one 4D TMA copy (box BX x BY x 1 x 15) into a ring of
// NSLOT slots, each completing on its own mbarrier.  All waits are bounded
// (WAIT_LIMIT polls).
#pragma once

#include <cuda.h>

#include "lbm_internal.cuh"

namespace lbm {
namespace ring {

constexpr int TX = 32, TY = 8;
constexpr int BX = TX + 2 * TMA_LEFT, BY = TY + 4;  // tile with its halo
constexpr int PL = BX * BY;                          // floats per field in one plane tile
constexpr int SLOT_BYTES_TX = NV * PL * 4;           // bytes one TMA copy delivers (28,800)
constexpr int SLOT_STRIDE = (SLOT_BYTES_TX + 127) / 128 * 128;
constexpr int NSLOT = 4;
constexpr int SMEM_BYTES = NSLOT * SLOT_STRIDE + NSLOT * 8;
constexpr unsigned WAIT_LIMIT = 1u << 22;   // try_wait polls before giving up (seconds)

static_assert(SLOT_STRIDE % 128 == 0 && SLOT_STRIDE >= SLOT_BYTES_TX, "slot pitch");

// L2 promotion of the plane copies (tensor maps of the tiled kernels).  On
// 256^3, 128-byte promotion against 256-byte: DRAM reads -1.5 %, 0.4630
// against 0.4643 ms per step (none: the same as 128-byte; 64-byte: 0.4638).
constexpr CUtensorMapL2promotion kPlaneL2Promotion = CU_TENSOR_MAP_L2_PROMOTION_L2_128B;
static_assert(BX * 4 % 16 == 0, "TMA box inner extent must be a 16-byte multiple");

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}

// Bounded wait (at most `limit` polls); returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned limit = WAIT_LIMIT) {
  for (unsigned it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_plane(float* dst, const CUtensorMap* map, int x, int y, int z,
                                               uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(0), "r"(smem_u32(bar))
      : "memory");
}

// Ask the TMA unit to bring a plane tile into L2 ahead of its shared-memory
// copy (no shared memory, no completion to wait for).
__device__ __forceinline__ void tma_prefetch_plane(const CUtensorMap* map, int x, int y, int z) {
  asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(z), "r"(0)
               : "memory");
}

}  // namespace ring
}  // namespace lbm
