// Blackwell tensor-core building blocks shared by the kernels that issue
// tcgen05.mma (k_gemm_tc.cu, k_unet.cu): shared-memory mbarriers with bounded
// waits, the K-major 128-byte-swizzle shared-memory descriptor, the kind::f16
// instruction descriptor (BF16 inputs, FP32 accumulation), the MMA issue and
// commit, and the 32-lane tensor-memory load of the epilogue.
#pragma once

#include <cuda_runtime.h>

#include "vie_internal.cuh"

namespace vie {
namespace tc {

constexpr long long kWaitLimit = 2000000000LL;  // clock cycles (about 1 s): the default bound

__device__ __forceinline__ unsigned su32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on phase `parity` of an mbarrier; false on timeout or abort.
// limit: clock cycles to wait; a zero limit gives up at once (no budget).
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, volatile int *abort_flag,
                                          long long limit = kWaitLimit) {
  if (limit <= 0) return false;
  const long long t0 = clock64();
  while (!mbar_test(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > limit) return false;
  }
  return true;
}


// K-major operand, 128-byte swizzle, rows of 128 bytes, 8-row groups 1024 B apart.
__device__ __forceinline__ unsigned long long smem_desc_sw128(unsigned addr) {
  unsigned long long d = 0;
  d |= (unsigned long long)((addr >> 4) & 0x3FFF);        // start address
  d |= (unsigned long long)(16 >> 4) << 16;               // leading byte offset (unused)
  d |= (unsigned long long)(1024 >> 4) << 32;             // stride byte offset
  d |= 1ull << 46;                                        // descriptor version
  d |= 2ull << 61;                                        // 128-byte swizzle
  return d;
}

// K-major operand, 64-byte swizzle: rows of 64 bytes (32 BF16 along K),
// 8-row groups 512 B apart (the layout a TMA box with a 64-byte inner extent
// and 64-byte swizzle writes).
__device__ __forceinline__ unsigned long long smem_desc_sw64(unsigned addr) {
  unsigned long long d = 0;
  d |= (unsigned long long)((addr >> 4) & 0x3FFF);        // start address
  d |= (unsigned long long)(16 >> 4) << 16;               // leading byte offset (unused)
  d |= (unsigned long long)(512 >> 4) << 32;              // stride byte offset
  d |= 1ull << 46;                                        // descriptor version
  d |= 4ull << 61;                                        // 64-byte swizzle
  return d;
}

// Tiled TMA loads into shared memory, completing on an mbarrier (coordinates
// innermost first; the innermost times the element size a multiple of 16 B).
__device__ __forceinline__ void tma_load_2d(unsigned dst, const void *map, unsigned bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
      "[%2];" ::"r"(dst),
      "l"(map), "r"(bar), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tma_load_4d(unsigned dst, const void *map, unsigned bar, int c, int x, int y,
                                            int b) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], "
      "[%2];" ::"r"(dst),
      "l"(map), "r"(bar), "r"(c), "r"(x), "r"(y), "r"(b)
      : "memory");
}

// kind::f16 instruction descriptor: D F32, A and B BF16, both K-major.
__host__ __device__ constexpr unsigned idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(unsigned tmem_d, unsigned long long a, unsigned long long b,
                                         unsigned idesc, unsigned accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(unsigned taddr, float *v) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc
}  // namespace vie
