// March of one work unit of the displacement-major pair kernels (2D and 3D):
// the chunked per-displacement stencils, kR targets stacked along the run
// axis in one thread.  Shared by k_pairs_disp.cu and k_pairs_disp3.cu.
#pragma once

#include <cuda_runtime.h>

namespace vie {
namespace dmarch {

constexpr int kR = 8;          // targets per thread, stacked along the run axis
constexpr int kChunkLengths[] = {2, 3, 4, 6, 8};
constexpr int kMaxChunk = 8;   // longest chunk

// lattice value M elements of stride ST (ST = 0: runtime stride st) after addr
template <int ST, int M>
__device__ __forceinline__ float lds_at(unsigned addr, int st) {
  float v;
  if constexpr (ST > 0) {
    asm("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(addr), "n"(4 * ST * M));
  } else {
    asm("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr + 4u * (unsigned)(st * M)));
  }
  return v;
}

// v[M .. CNT) = the lattice values M .. CNT - 1 strides after addr
template <int ST, int M, int CNT>
struct LoadRun {
  static __device__ __forceinline__ void go(unsigned addr, int st, float *v) {
    v[M] = lds_at<ST, M>(addr, st);
    LoadRun<ST, M + 1, CNT>::go(addr, st, v);
  }
};
template <int ST, int CNT>
struct LoadRun<ST, CNT, CNT> {
  static __device__ __forceinline__ void go(unsigned, int, float *) {}
};

// acc[q] += sum over the chunks of W_D of w(c) sigma[target q + c].
// A chunk record is RS float4s: the offset of its first cell from the target
// in lattice elements (int bits), then its LC weights, zero-padded.
template <int LC, int ST>
__device__ __forceinline__ void march_chunks(const float4 *__restrict__ rec, int chunks, unsigned base,
                                             int st, float (&acc)[kR]) {
  constexpr int RS = (LC + 4) / 4;
#pragma unroll 1
  for (int c = 0; c < chunks; ++c, rec += RS) {
    float w[4 * RS];
#pragma unroll
    for (int i = 0; i < RS; ++i) {
      const float4 f = __ldg(rec + i);
      w[4 * i] = f.x;
      w[4 * i + 1] = f.y;
      w[4 * i + 2] = f.z;
      w[4 * i + 3] = f.w;
    }
    const unsigned addr = base + 4u * (unsigned)__float_as_int(w[0]);
    float v[LC + kR - 1];
    LoadRun<ST, 0, LC + kR - 1>::go(addr, st, v);
#pragma unroll
    for (int t = 0; t < LC; ++t)
#pragma unroll
      for (int q = 0; q < kR; ++q) acc[q] = fmaf(w[1 + t], v[t + q], acc[q]);
  }
}

// The same march with the lattice in global memory (read through L1): the
// chunk's cells and stacked targets lie ST elements apart from base + offset.
template <int LC, int ST>
__device__ __forceinline__ void march_chunks_global(const float4 *__restrict__ rec, int chunks,
                                                    const float *__restrict__ base, float (&acc)[kR]) {
  constexpr int RS = (LC + 4) / 4;
#pragma unroll 1
  for (int c = 0; c < chunks; ++c, rec += RS) {
    float w[4 * RS];
#pragma unroll
    for (int i = 0; i < RS; ++i) {
      const float4 f = __ldg(rec + i);
      w[4 * i] = f.x;
      w[4 * i + 1] = f.y;
      w[4 * i + 2] = f.z;
      w[4 * i + 3] = f.w;
    }
    const float *p = base + __float_as_int(w[0]);
    float v[LC + kR - 1];
#pragma unroll
    for (int m = 0; m < LC + kR - 1; ++m) v[m] = __ldg(p + ST * m);
#pragma unroll
    for (int t = 0; t < LC; ++t)
#pragma unroll
      for (int q = 0; q < kR; ++q) acc[q] = fmaf(w[1 + t], v[t + q], acc[q]);
  }
}

// Integer add whose old value nobody reads: the reduction form, with no
// value coming back to the issuing warp.  No memory clobber, so the compiler
// may still move the (read-only) source loads around it; the sums are read
// only by a later launch.
__device__ __forceinline__ void red_add(unsigned long long *p, unsigned long long v) {
  asm volatile("red.global.add.u64 [%0], %1;" ::"l"(p), "l"(v));
}

template <int ST>
__device__ __forceinline__ void march_unit(int lc, const float4 *__restrict__ rec, int chunks, unsigned base,
                                           int st, float (&acc)[kR]) {
  switch (lc) {
    case 2: march_chunks<2, ST>(rec, chunks, base, st, acc); break;
    case 3: march_chunks<3, ST>(rec, chunks, base, st, acc); break;
    case 4: march_chunks<4, ST>(rec, chunks, base, st, acc); break;
    case 6: march_chunks<6, ST>(rec, chunks, base, st, acc); break;
    default: march_chunks<8, ST>(rec, chunks, base, st, acc); break;
  }
}

template <int ST>
__device__ __forceinline__ void march_unit_global(int lc, const float4 *__restrict__ rec, int chunks,
                                                  const float *__restrict__ base, float (&acc)[kR]) {
  switch (lc) {
    case 2: march_chunks_global<2, ST>(rec, chunks, base, acc); break;
    case 3: march_chunks_global<3, ST>(rec, chunks, base, acc); break;
    case 4: march_chunks_global<4, ST>(rec, chunks, base, acc); break;
    case 6: march_chunks_global<6, ST>(rec, chunks, base, acc); break;
    default: march_chunks_global<8, ST>(rec, chunks, base, acc); break;
  }
}

}  // namespace dmarch
}  // namespace vie
