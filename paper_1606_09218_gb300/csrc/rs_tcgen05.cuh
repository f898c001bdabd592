// PTX helpers shared by the tcgen05 kernels: mbarriers with bounded waits, bulk copies,
// shared-memory matrix descriptors (canonical K-major layout, no swizzle), kind::f16 MMAs and
// their commits, tensor-memory loads, FP16 hi / lo splitting.  Internal linkage: every
// translation unit that includes this header gets its own copy.
#pragma once

#include <cuda_fp16.h>
#include <cstdint>

#include "rs_internal.cuh"

namespace rs {
namespace {

constexpr long long WAIT_LIMIT = 4000000;  // polls of a bounded mbarrier wait (about 1 s)

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity.  Returns false when another role has
// aborted or when the limit ran out (then this thread raises the abort and FLAG_TIMEOUT).
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                         DevScalars* sc) {
  for (long long i = 0; i < WAIT_LIMIT; ++i) {
    if (mbar_test(bar, parity)) return true;
    if ((i & 255) == 255 && *abort_flag) return false;
  }
  *abort_flag = 1;
  atomicOr(&sc->flags, (unsigned)FLAG_TIMEOUT);
  return false;
}

// the same for a whole warp: lane 0 waits, the result is broadcast (warp-uniform control flow)
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          DevScalars* sc) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) ok = wait_bar(bar, parity, abort_flag, sc) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// Bounded wait that ignores the abort flag (draining work in flight before exit).
__device__ __forceinline__ void drain_bar(uint64_t* bar, uint32_t parity, DevScalars* sc) {
  for (long long i = 0; i < WAIT_LIMIT; ++i)
    if (mbar_test(bar, parity)) return;
  atomicOr(&sc->flags, (unsigned)FLAG_TIMEOUT);
}

// contiguous global -> shared copy completed on an mbarrier (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"((uint64_t)src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// shared -> global bulk copy (16-byte aligned, size % 16 == 0), tracked by bulk groups

// split a pair of FP32 values into FP16 hi / lo pairs (first value in the low half)
__device__ __forceinline__ void split_h2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(x0, x1);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// eight FP32 values -> 16 bytes of FP16 hi and 16 bytes of FP16 lo
__device__ __forceinline__ void split8_f16(const float* x, uint4& hi, uint4& lo) {
  split_h2(x[0], x[1], hi.x, lo.x);
  split_h2(x[2], x[3], hi.y, lo.y);
  split_h2(x[4], x[5], hi.z, lo.z);
  split_h2(x[6], x[7], hi.w, lo.w);
}

// canonical K-major layout without swizzle: 8-row x 16-byte core matrices, the K chunks of a
// row group contiguous (LBO = 128 B), row groups (chunks per row) * 128 B apart.
__device__ __forceinline__ uint32_t kmajor_offset(int row, int chunk, int chunks_per_row) {
  return ((uint32_t)(row >> 3) * (uint32_t)chunks_per_row + (uint32_t)chunk) * 128u + (uint32_t)(row & 7) * 16u;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);          // start address
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;      // leading dimension (K) byte offset
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;      // stride dimension (M/N) byte offset
  d |= (uint64_t)1 << 46;                            // fixed 0b001
  return d;                                           // base offset 0, no swizzle
}

// instruction descriptor (kind::f16): D FP32, A and B FP16, both K-major, M = mm, N = nn
__device__ __forceinline__ uint32_t idesc_f16(int nn, int mm = 128) {
  return (1u << 4) | ((uint32_t)(nn >> 3) << 17) | ((uint32_t)(mm >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"((uint64_t)dst),
               "r"(smem_addr(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 8 consecutive accumulator columns of this warp's 32 lanes (one row per lane)
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Power-of-two exponent e with x < 2^e (0 for x <= 0 or non-finite).
__device__ __forceinline__ int exp2_above(double x) {
  if (!(x > 0.0) || !isfinite(x)) return 0;
  int e = 0;
  frexp(x, &e);
  return e;
}

}  // namespace
}  // namespace rs
