// Tensor-memory-accelerator (TMA) row loads and mbarriers, inline PTX for sm_103a.
//
// The fused step kernel stages each row of the nine population planes into
// shared memory with one 3-D tiled bulk copy per warp: a box of 32 columns x
// 1 row x 9 planes of this GPU's own memory (no multicast), described by a
// tensor map per cavity and ping-pong buffer built on the host
// (cuTensorMapEncodeTiled). Columns outside the cavity read as zeros. A copy
// signals an mbarrier with its byte count; the warp waits on the barrier's
// phase with a bounded number of tries, and a wait that gives up reports it
// in the step's status word instead of hanging.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ifd {

// Bits of the step status word (Bufs::status)
constexpr unsigned STATUS_NONFINITE = 1u;  // a non-finite velocity was formed
constexpr unsigned STATUS_TMA_TIMEOUT = 2u;  // a TMA row load did not complete in time

// Tries of a bounded mbarrier wait, each suspending for at most ~1 us: a wait
// gives up after roughly a second.
constexpr int MBAR_TRIES = 1 << 20;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

// Makes barrier initialisation visible to the async proxy (the TMA unit).
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) accesses of the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// Acquires a tensor map that the host wrote to global memory before the
// launch, for the TMA unit's reads of it (tensormap proxy).
__device__ __forceinline__ void tmap_acquire(const void *tmap) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(
                   reinterpret_cast<uint64_t>(tmap))
               : "memory");
}

// One thread: arms the barrier for `bytes` and issues the copy of the box at
// (x, y, 0) of the tensor map into dst (128-byte aligned shared memory).
// x must be a multiple of 16 bytes' worth of elements.
__device__ __forceinline__ void tma_load_box3(void *dst, const void *tmap, int x, int y,
                                              uint64_t *bar, uint32_t bytes) {
  const uint32_t b = smem_addr(bar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(b), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(0), "r"(b)
      : "memory");
}

// Waits until the barrier's phase with parity `parity` has completed; gives up
// after MBAR_TRIES tries and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const uint32_t b = smem_addr(bar);
  for (int i = 0; i < MBAR_TRIES; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(b), "r"(parity), "r"(1000u)
        : "memory");
    if (done) return true;
  }
  return false;
}

}  // namespace ifd
