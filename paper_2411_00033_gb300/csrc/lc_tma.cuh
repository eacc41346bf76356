// lc_tma.cuh -- bulk asynchronous copies (TMA without a tensor map) from
// global to shared memory, completing on an mbarrier, with a bounded wait.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// Both addresses 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void lc_bulk_g2s(void* dst, const void* src, uint32_t bytes, uint32_t mbar) {
  const uint32_t d = uint32_t(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
               :: "r"(d), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}
__device__ __forceinline__ void lc_mbar_init(uint32_t mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(mbar) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void lc_mbar_expect(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" :: "r"(mbar), "r"(bytes) : "memory");
}
// Order earlier generic-proxy accesses to shared memory before a bulk copy.
__device__ __forceinline__ void lc_fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ bool lc_mbar_try(uint32_t mbar, uint32_t phase) {
  uint32_t done;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(done) : "r"(mbar), "r"(phase) : "memory");
  return done != 0;
}
// Wait for the phase with a deadline of about one second; false on timeout.
__device__ __forceinline__ bool lc_mbar_wait_bounded(uint32_t mbar, uint32_t phase) {
  const long long t0 = clock64();
  while (!lc_mbar_try(mbar, phase)) {
    if (clock64() - t0 > (1ll << 31)) return false;
  }
  return true;
}
