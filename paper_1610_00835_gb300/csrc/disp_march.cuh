// March of one work unit of the displacement-major pair kernels (2D and 3D):
// the chunked per-displacement stencils, kR targets stacked along the run
// axis in one thread.  Shared by k_pairs_disp.cu and k_pairs_disp3.cu.
#pragma once

#include <cuda_runtime.h>

namespace vie {
namespace dmarch {

constexpr int kR = 8;          // targets per thread, stacked along the run axis
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

// ---- 2D march: chunks of their own length, stacked targets in FP32 pairs.
//
// A run of the stencil is cut into chunks of equal length lc <= kMaxChunk,
// so no chunk carries zero weights (record layout below).  The lc + R - 1
// lattice values v[0 ..) of a chunk are held as aligned register pairs
// P[i] = (v[2i], v[2i+1]), and the R (even) stacked sums as pairs too:
//   even t: (acc[2p], acc[2p+1])   += w[t] (v[t+2p], v[t+2p+1])   p < R/2
//   odd t:  (b[2p+1], b[2p+2])     += w[t] (v[t+2p+1], v[t+2p+2]) p < R/2 - 1
//           acc[0] (c0), acc[R-1] (cl) += w[t] v[t], w[t] v[t+R-1]
// so every product is one lane of a packed fma.rn.f32x2 (the same rounding as
// fmaf) on pairs whose first index is even: no register moves.  The odd-t
// partial sums b and c0, cl join acc at the end, in a fixed order.
typedef unsigned long long u64;

__device__ __forceinline__ u64 pack2(float a, float b) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void unpack2(u64 r, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ void ffma2(u64 &d, u64 a, u64 b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}

template <int R>
struct Acc2 {
  static_assert(R % 2 == 0 && R >= 4, "stacked targets in pairs");
  u64 a[R / 2];       // (acc[0], acc[1]) .. (acc[R-2], acc[R-1]): even t
  u64 b[R / 2 - 1];   // (acc[1], acc[2]) .. (acc[R-3], acc[R-2]): odd t
  float c0, cl;       // acc[0], acc[R-1]: odd t
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int p = 0; p < R / 2; ++p) a[p] = 0ull;
#pragma unroll
    for (int p = 0; p < R / 2 - 1; ++p) b[p] = 0ull;
    c0 = cl = 0.f;
  }
  __device__ __forceinline__ void sum(float (&acc)[R]) const {
    float al[R / 2], ah[R / 2], bl[R / 2 - 1], bh[R / 2 - 1];
#pragma unroll
    for (int p = 0; p < R / 2; ++p) unpack2(a[p], al[p], ah[p]);
#pragma unroll
    for (int p = 0; p < R / 2 - 1; ++p) unpack2(b[p], bl[p], bh[p]);
    acc[0] = al[0] + c0;
#pragma unroll
    for (int p = 0; p < R / 2 - 1; ++p) {
      acc[2 * p + 1] = ah[p] + bl[p];
      acc[2 * p + 2] = al[p + 1] + bh[p];
    }
    acc[R - 1] = ah[R / 2 - 1] + cl;
  }
};

// the taps of one chunk: w[0 .. LC), v[0 .. LC + R - 1)
template <int LC, int R>
__device__ __forceinline__ void taps2(const float *w, const float *v, Acc2<R> &s) {
  constexpr int NV = LC + R - 1, NP = NV / 2;
  u64 P[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) P[i] = pack2(v[2 * i], v[2 * i + 1]);
#pragma unroll
  for (int t = 0; t < LC; ++t) {
    const u64 W = pack2(w[t], w[t]);
    if ((t & 1) == 0) {
#pragma unroll
      for (int p = 0; p < R / 2; ++p) ffma2(s.a[p], W, P[t / 2 + p]);
    } else {
#pragma unroll
      for (int p = 0; p < R / 2 - 1; ++p) ffma2(s.b[p], W, P[(t + 1) / 2 + p]);
      s.c0 = fmaf(w[t], v[t], s.c0);
      s.cl = fmaf(w[t], v[t + R - 1], s.cl);
    }
  }
}


// A D's chunk records, grouped by chunk length: one header float4 whose four
// words hold the number of chunks of each length lc = 1..8 (16 bits per
// length: lengths 1, 2 in .x, 3, 4 in .y, 5, 6 in .z, 7, 8 in .w), then the
// chunks of length 1, those of length 2, and so on.  A chunk of length LC is
// (LC + 4) / 4 float4s: the offset of its first cell from the target in
// lattice elements (int bits), then its LC weights.  Each length runs in its
// own loop, unrolled for that length: no per-chunk dispatch.
template <int LC>
__device__ __forceinline__ int chunk_count(const float4 &hdr) {
  const float f = LC <= 2 ? hdr.x : LC <= 4 ? hdr.y : LC <= 6 ? hdr.z : hdr.w;
  return (int)((__float_as_uint(f) >> (16 * ((LC - 1) & 1))) & 0xffffu);
}

template <int LC>
__device__ __forceinline__ void load_chunk(const float4 *__restrict__ rec, int &off, float (&w)[LC]) {
  constexpr int RS = (LC + 4) / 4;
  float all[4 * RS];
#pragma unroll
  for (int i = 0; i < RS; ++i) {
    const float4 f = __ldg(rec + i);
    all[4 * i] = f.x; all[4 * i + 1] = f.y; all[4 * i + 2] = f.z; all[4 * i + 3] = f.w;
  }
  off = __float_as_int(all[0]);
#pragma unroll
  for (int t = 0; t < LC; ++t) w[t] = all[1 + t];
}

template <int LC, int ST, int R>
__device__ __forceinline__ const float4 *chunks2_smem(const float4 *__restrict__ rec, int cnt, unsigned base,
                                                      int st, Acc2<R> &s) {
  constexpr int RS = (LC + 4) / 4;
#pragma unroll 1
  for (int c = 0; c < cnt; ++c, rec += RS) {
    int off;
    float w[LC];
    load_chunk<LC>(rec, off, w);
    float v[LC + R - 1];
    LoadRun<ST, 0, LC + R - 1>::go(base + 4u * (unsigned)off, st, v);
    taps2<LC, R>(w, v, s);
  }
  return rec;
}

template <int LC, int ST, int R>
__device__ __forceinline__ const float4 *chunks2_global(const float4 *__restrict__ rec, int cnt,
                                                        const float *__restrict__ base, Acc2<R> &s) {
  constexpr int RS = (LC + 4) / 4;
#pragma unroll 1
  for (int c = 0; c < cnt; ++c, rec += RS) {
    int off;
    float w[LC];
    load_chunk<LC>(rec, off, w);
    const float *p = base + off;
    float v[LC + R - 1];
#pragma unroll
    for (int m = 0; m < LC + R - 1; ++m) v[m] = __ldg(p + ST * m);
    taps2<LC, R>(w, v, s);
  }
  return rec;
}

// acc[q] = sum over the chunks of one unit of w(c) sigma[target q + c], the
// lattice in shared memory (base: the first stacked target's byte address).
template <int ST, int R>
__device__ __forceinline__ void march_runs(const float4 *__restrict__ rec, unsigned base, int st,
                                           float (&acc)[R]) {
  Acc2<R> s;
  s.zero();
  const float4 hdr = __ldg(rec);
  ++rec;
  int c;
  if ((c = chunk_count<1>(hdr)) > 0) rec = chunks2_smem<1, ST, R>(rec, c, base, st, s);
  if ((c = chunk_count<2>(hdr)) > 0) rec = chunks2_smem<2, ST, R>(rec, c, base, st, s);
  if ((c = chunk_count<3>(hdr)) > 0) rec = chunks2_smem<3, ST, R>(rec, c, base, st, s);
  if ((c = chunk_count<4>(hdr)) > 0) rec = chunks2_smem<4, ST, R>(rec, c, base, st, s);
  if ((c = chunk_count<5>(hdr)) > 0) rec = chunks2_smem<5, ST, R>(rec, c, base, st, s);
  if ((c = chunk_count<6>(hdr)) > 0) rec = chunks2_smem<6, ST, R>(rec, c, base, st, s);
  if ((c = chunk_count<7>(hdr)) > 0) rec = chunks2_smem<7, ST, R>(rec, c, base, st, s);
  if ((c = chunk_count<8>(hdr)) > 0) rec = chunks2_smem<8, ST, R>(rec, c, base, st, s);
  s.sum(acc);
}

// The same with the lattice in global memory (read through L1): the chunk's
// cells and stacked targets lie ST elements apart from base + offset.
template <int ST, int R>
__device__ __forceinline__ void march_runs_global(const float4 *__restrict__ rec, const float *__restrict__ base,
                                                  float (&acc)[R]) {
  Acc2<R> s;
  s.zero();
  const float4 hdr = __ldg(rec);
  ++rec;
  int c;
  if ((c = chunk_count<1>(hdr)) > 0) rec = chunks2_global<1, ST, R>(rec, c, base, s);
  if ((c = chunk_count<2>(hdr)) > 0) rec = chunks2_global<2, ST, R>(rec, c, base, s);
  if ((c = chunk_count<3>(hdr)) > 0) rec = chunks2_global<3, ST, R>(rec, c, base, s);
  if ((c = chunk_count<4>(hdr)) > 0) rec = chunks2_global<4, ST, R>(rec, c, base, s);
  if ((c = chunk_count<5>(hdr)) > 0) rec = chunks2_global<5, ST, R>(rec, c, base, s);
  if ((c = chunk_count<6>(hdr)) > 0) rec = chunks2_global<6, ST, R>(rec, c, base, s);
  if ((c = chunk_count<7>(hdr)) > 0) rec = chunks2_global<7, ST, R>(rec, c, base, s);
  if ((c = chunk_count<8>(hdr)) > 0) rec = chunks2_global<8, ST, R>(rec, c, base, s);
  s.sum(acc);
}

// Integer add whose old value nobody reads: the reduction form, with no
// value coming back to the issuing warp.  No memory clobber, so the compiler
// may still move the (read-only) source loads around it; the sums are read
// only by a later launch.
__device__ __forceinline__ void red_add(unsigned long long *p, unsigned long long v) {
  asm volatile("red.global.add.u64 [%0], %1;" ::"l"(p), "l"(v));
}

}  // namespace dmarch
}  // namespace vie
