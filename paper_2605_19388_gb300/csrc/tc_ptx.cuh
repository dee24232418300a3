// tc_ptx.cuh -- inline-PTX building blocks of the tensor-core kernels (mbarrier waits with a
// bounded budget, TMA tensor copies, shared-memory matrix descriptors, tcgen05 MMA issue).
#pragma once
#include <cuda.h>

#include "common.cuh"

namespace dfm {

constexpr unsigned TC_WAIT_CYCLES = 2000000000u;  // ~1 s at 2 GHz

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// Wait for the phase with the given parity to complete; false on timeout.
// The phase is tested without blocking; between tests the warp sleeps for
// about `sleep_ns`, chosen per role: a waiting warp takes issue slots from
// the converter warps of its scheduler on every poll, so warps that wait
// most of the time (the epilogue, the producer) poll rarely and the MMA
// issuer, whose wake-up delays the pipeline, polls often.
__device__ __forceinline__ bool mbar_test(unsigned addr, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(addr), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, unsigned sleep_ns = 32,
                                          unsigned budget = TC_WAIT_CYCLES) {
  const unsigned addr = smem_u32(bar);
  if (mbar_test(addr, parity)) return true;
  const unsigned start = (unsigned)clock();
  while (true) {
    if ((unsigned)clock() - start > budget) return false;  // wrap-safe: the budget is below 2^32
    __nanosleep(sleep_ns);
    if (mbar_test(addr, parity)) return true;
  }
}
// The same wait by every lane of a warp, with one warp-uniform result.
__device__ __forceinline__ bool mbar_wait_warp(unsigned long long* bar, unsigned parity, unsigned sleep_ns = 32,
                                               unsigned budget = TC_WAIT_CYCLES) {
  return __all_sync(DFM_FULL_MASK, mbar_wait(bar, parity, sleep_ns, budget)) != 0;
}

// One lane of the (fully active) warp, the same on every call.
__device__ __forceinline__ bool elect_one() {
  unsigned pred;
  asm volatile("{\n .reg .pred p;\n elect.sync _|p, 0xffffffff;\n selp.u32 %0, 1, 0, p;\n}" : "=r"(pred));
  return pred != 0;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, int c0, int c1, int c2, const void* src) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                   reinterpret_cast<unsigned long long>(map)),
               "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(src))
               : "memory");
}

// Shared-memory matrix descriptor: K-major operand tile with 128-byte
// swizzle, 8-row groups 1024 bytes apart (stride byte offset), descriptor
// version 1, base offset 0.
__device__ __forceinline__ unsigned long long smem_desc_sw128(unsigned addr) {
  unsigned long long d = 0;
  d |= (unsigned long long)((addr >> 4) & 0x3FFF);
  d |= (unsigned long long)(1) << 16;              // leading byte offset (unused by swizzled K-major)
  d |= (unsigned long long)((1024 >> 4) & 0x3FFF) << 32;
  d |= 1ull << 46;                                 // version
  d |= 2ull << 61;                                 // 128-byte swizzle
  return d;
}


// One tcgen05.mma of kind::f16 or kind::tf32 with the instruction descriptor `idesc`; acc = 0
// overwrites the accumulator, otherwise adds to it.
__device__ __forceinline__ void umma_f16_id(unsigned tmem_d, unsigned long long a, unsigned long long b, unsigned idesc,
                                            unsigned acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_tf32_id(unsigned tmem_d, unsigned long long a, unsigned long long b,
                                             unsigned idesc, unsigned acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// Arrive on `bar` once every tcgen05 operation this thread issued before has completed.
__device__ __forceinline__ void umma_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

}  // namespace dfm
