// alb_bulk.cuh -- bulk asynchronous copies (TMA engine, untiled form) between
// global and shared memory, with mbarrier completion, for the streaming
// kernels that move contiguous byte ranges.
//
// Rules the callers keep: global and shared addresses 16-byte aligned, sizes
// a multiple of 16; a shared buffer written by threads is fenced to the async
// proxy (fence_proxy_async) and barrier-synchronised before a bulk store reads
// it; a buffer is refilled only after the bulk store reading it has finished
// its reads (bulk_wait_read).  Every wait on an mbarrier is bounded.
#pragma once

#include "alb_common.cuh"

namespace alb {

constexpr uint32_t kMbarSpinLimit = 1u << 22;   // x >= 64 ns sleeps: a few tenths of a second at least

ALB_D uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

ALB_D void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// make initialised barriers visible to the async proxy
ALB_D void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

// the single arrival of a phase, announcing `bytes` of async-copy transactions
ALB_D void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

ALB_D bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok = 0;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity (at most `limit` tries,
// each followed by a short sleep); false when it gave up.
ALB_D bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit = kMbarSpinLimit) {
  for (uint32_t i = 0; i < limit; i++) {
    if (mbar_try_wait(bar, parity)) return true;
    __nanosleep(64);
  }
  return false;
}

ALB_D void bulk_load(void* smem_dst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_addr(smem_dst)),
      "l"(gsrc), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

ALB_D void bulk_store(void* gdst, const void* smem_src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(gdst), "r"(smem_addr(smem_src)),
               "r"(bytes)
               : "memory");
}

ALB_D void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }

// all but the newest N bulk-store groups have finished reading shared memory
template <int N>
ALB_D void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;\n" ::"n"(N) : "memory");
}

// all bulk-store groups are complete (writes performed)
ALB_D void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

// order this thread's shared-memory writes before later async-proxy reads
ALB_D void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

}  // namespace alb
