// Products with the assembled operator (Section 3.2, K = [K_jk omega_k]).
//
// * k_gemv: y = K g for one right-hand side on the CUDA cores, K in FP32 or
//   BF16 hi/lo (4 bytes per entry either way); bandwidth bound.
// * k_gemm_bf16x3: Y = K G for R right-hand sides on the 5th-generation
//   tensor cores.  K = Khi + Klo is the BF16 split of the assembled FP32
//   operator (a fixed matrix); G is split three ways, G = Ghi + Gmid + Glo,
//   which represents its FP32 values exactly, so the product applies that
//   fixed matrix to FP32 G: the kept terms Khi Ghi, Khi Gmid, Klo Ghi,
//   Khi Glo and Klo Gmid leave out only Klo Glo (below 2^-24 of |K||G|).
//   A product whose error depended on how G rounds would not be a linear
//   operator, and GMRES could not drive its residual below that error.  The
//   terms accumulate in FP32 in tensor memory.  One CTA computes a 128-row
//   tile of Y for all R columns over one K-range (split-K); a TMA producer
//   thread streams 64-wide K slices of Khi, Klo, Ghi, Gmid, Glo into a
//   shared-memory ring of up to 4 stages (128-byte swizzle), one thread
//   issues tcgen05.mma and the four warps read the accumulators back with
//   tcgen05.ld.  Per 16-wide K step three instructions (M = 128, K = 16):
//   Khi Ghi (N = R), and the cross terms as two N = 2R products into one
//   block of 2R columns, Khi [Gmid; Glo] and Klo [Ghi; Gmid] (the G slices
//   sit back to back in the stage, so each pair is one operand).  Each
//   instruction has a fixed cost beside its math, so three wide ones take
//   less time than five N = R ones on the same operands.
//   The tensor cores do not round their FP32 accumulation to nearest, so a
//   long chain of products into one accumulator drifts low (measured: 3e-5
//   relative after ~770 chained MMAs; the drift grows with the chain, about
//   2^-25 per MMA).  The dominant Khi Ghi product therefore rotates over up
//   to seven accumulators (as many as tensor memory holds beside the cross
//   block), split-K keeps every chain at or below kMaxChain MMAs, and the
//   accumulators are added in FP32 in the epilogue, and across splits as an
//   FP32 hi + lo pair (error-free additions) converted once to FP64.
//   At most 128 right-hand sides per product (three G slices per stage).
//   Every mbarrier wait is bounded by a clock limit; on expiry the CTA sets
//   an error word, stops issuing work, waits for its issued copies and
//   products (again bounded), frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "tcgen05.cuh"
#include "vie_internal.cuh"

namespace vie {

namespace {

using namespace tc;

// ------------------------------------------------------------------ GEMV

template <bool BF16>
__global__ void __launch_bounds__(256) k_gemv(const void *__restrict__ K, const void *__restrict__ Klo,
                                              long ldk, long N, const float *__restrict__ g32,
                                              const double *__restrict__ g64, int op,
                                              double *__restrict__ y) {
  const int lane = threadIdx.x & 31;
  const long warp = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
  const long nwarps = ((long)gridDim.x * blockDim.x) >> 5;
  for (long row = warp; row < N; row += nwarps) {
    float acc0 = 0.f, acc1 = 0.f;
    if (BF16) {
      const uint4 *hi = reinterpret_cast<const uint4 *>((const __nv_bfloat16 *)K + row * ldk);
      const uint4 *lo = reinterpret_cast<const uint4 *>((const __nv_bfloat16 *)Klo + row * ldk);
      const long nchunk = ldk / 8;
      for (long c = lane; c < nchunk; c += 32) {
        const uint4 h = __ldcs(hi + c), l = __ldcs(lo + c);
        const float4 ga = __ldg(reinterpret_cast<const float4 *>(g32) + 2 * c);
        const float4 gb = __ldg(reinterpret_cast<const float4 *>(g32) + 2 * c + 1);
        const __nv_bfloat162 *hp = reinterpret_cast<const __nv_bfloat162 *>(&h);
        const __nv_bfloat162 *lp = reinterpret_cast<const __nv_bfloat162 *>(&l);
        const float gv[8] = {ga.x, ga.y, ga.z, ga.w, gb.x, gb.y, gb.z, gb.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float2 hf = __bfloat1622float2(hp[e]);
          const float2 lf = __bfloat1622float2(lp[e]);
          acc0 = fmaf(hf.x + lf.x, gv[2 * e], acc0);
          acc1 = fmaf(hf.y + lf.y, gv[2 * e + 1], acc1);
        }
      }
    } else {
      const float4 *kr = reinterpret_cast<const float4 *>((const float *)K + row * ldk);
      const long nchunk = ldk / 4;
      for (long c = lane; c < nchunk; c += 32) {
        const float4 kv = __ldcs(kr + c);
        const float4 gv = __ldg(reinterpret_cast<const float4 *>(g32) + c);
        acc0 = fmaf(kv.x, gv.x, fmaf(kv.z, gv.z, acc0));
        acc1 = fmaf(kv.y, gv.y, fmaf(kv.w, gv.w, acc1));
      }
    }
    double s = (double)acc0 + (double)acc1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = op == VIE_OP_I_MINUS_K ? g64[row] - s : s;
  }
}

__global__ void k_divide(long N, const double *__restrict__ a, const double *__restrict__ b,
                         double *__restrict__ out) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x)
    out[i] = a[i] / b[i];
}

// out[r][i] = a[r][i] / b[i] for R columns (column r of a at r lda, of out at r ldo)
__global__ void k_divide_cols(long N, int R, const double *__restrict__ a, long lda, const double *__restrict__ b,
                              double *__restrict__ out, long ldo) {
  const long total = (long)R * N;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const long r = t / N, i = t - r * N;
    out[r * ldo + i] = a[r * lda + i] / b[i];
  }
}

// g (FP64 [nrhs][N]) -> FP32 [nrhs][ldk], zero padded
__global__ void k_to_f32_padded(const double *__restrict__ g, long N, long ldk, int nrhs,
                                float *__restrict__ out) {
  const long total = (long)nrhs * ldk;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long r = i / ldk, c = i % ldk;
    out[i] = c < N ? (float)g[r * N + c] : 0.f;
  }
}

// G (FP64, column r at g + r ldg) -> FP32 -> BF16 hi + mid + lo [rpad][ldk],
// zero padded.  hi = bf16(v), mid = bf16(v - hi), lo = bf16(v - hi - mid):
// each remainder is exact in FP32 and has 8 fewer significant bits, so
// hi + mid + lo = v (FP32 v in the BF16 exponent range).  Row r = blockIdx.y,
// two columns per thread (ldk is a multiple of 64).
__device__ __forceinline__ void split3(float v, __nv_bfloat16 &h, __nv_bfloat16 &m, __nv_bfloat16 &l) {
  h = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(h);
  m = __float2bfloat16_rn(r1);
  l = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

__global__ void k_split_bf16(const double *__restrict__ g, long ldg, long N, long ldk, int nrhs,
                             __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ mid,
                             __nv_bfloat16 *__restrict__ lo) {
  const int r = blockIdx.y;
  const double *gr = g + (long)r * ldg;
  const long row = (long)r * ldk;
  for (long c = 2 * (blockIdx.x * (long)blockDim.x + threadIdx.x); c < ldk; c += 2L * gridDim.x * blockDim.x) {
    const float v0 = (r < nrhs && c < N) ? (float)gr[c] : 0.f;
    const float v1 = (r < nrhs && c + 1 < N) ? (float)gr[c + 1] : 0.f;
    __nv_bfloat162 h, m, l;
    split3(v0, h.x, m.x, l.x);
    split3(v1, h.y, m.y, l.y);
    *(__nv_bfloat162 *)(hi + row + c) = h;
    *(__nv_bfloat162 *)(mid + row + c) = m;
    *(__nv_bfloat162 *)(lo + row + c) = l;
  }
}

// Error-free FP32 addition (Knuth's TwoSum): s + e = a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}

// Running sum of FP32 partials as an unevaluated pair hi + lo: hi is the
// rounded sum, lo collects the rounding errors (error ~2^-48 relative).
struct PairSum {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float v) {
    float e;
    two_sum(hi, v, hi, e);
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// y[r][j] = sum_split part[split][r][j]  (then the operator); column r of g
// and y at r ldg and r ldy.  The splits are added in split order as an FP32
// hi + lo pair and converted once: GB300's FP64 pipe is narrow, and a
// conversion and an FP64 add per split made this kernel FP64-bound.  Row
// r = blockIdx.y, four columns per thread (16-byte loads of the partials
// when N is a multiple of 4).  A product that gave up on a bounded wait
// (*err != 0) turns y into NaN, which the Krylov driver reports as
// VIE_ERR_NONFINITE.
__global__ void k_gemm_finish(const float *__restrict__ part, int splits, int nrhs, long N,
                              const double *__restrict__ g, long ldg, int op, const int *__restrict__ err,
                              double *__restrict__ y, long ldy) {
  const long total = (long)nrhs * N;
  const bool failed = *err != 0;
  const int r = blockIdx.y;
  const float *pr = part + (long)r * N;
  for (long j0 = 4 * (blockIdx.x * (long)blockDim.x + threadIdx.x); j0 < N; j0 += 4L * gridDim.x * blockDim.x) {
    PairSum s[4];
    if ((N & 3) == 0) {
      int p = 0;
      for (; p + 4 <= splits; p += 4) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = __ldg((const float4 *)(pr + (long)(p + u) * total + j0));
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          s[0].add(v[u].x);
          s[1].add(v[u].y);
          s[2].add(v[u].z);
          s[3].add(v[u].w);
        }
      }
      for (; p < splits; ++p) {
        const float4 v = __ldg((const float4 *)(pr + (long)p * total + j0));
        s[0].add(v.x);
        s[1].add(v.y);
        s[2].add(v.z);
        s[3].add(v.w);
      }
    } else {
      for (int p = 0; p < splits; ++p)
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (j0 + e < N) s[e].add(pr[(long)p * total + j0 + e]);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const long j = j0 + e;
      if (j < N) {
        const double v = s[e].value();
        y[(long)r * ldy + j] = failed ? __longlong_as_double(0x7ff8000000000000LL)
                                      : (op == VIE_OP_I_MINUS_K ? g[(long)r * ldg + j] - v : v);
      }
    }
  }
}

// ------------------------------------------------------------------ GEMM

constexpr int BM = 128;          // rows of Y per CTA (MMA M)
constexpr int BK = 64;           // K elements per stage: 128 bytes of BF16
constexpr int MAX_STAGES = 4;
constexpr int UMMA_K = 16;       // K per tcgen05.mma kind::f16

struct GemmArgs {
  int stages;        // shared-memory ring depth (2..4)
  int rpad;          // N of the MMA (multiple of 16, <= 256)
  int nrhs;          // valid columns
  long N;            // rows of K and Y
  int kblocks_total; // ldk / BK
  int kblocks_per_split;
  int tmem_cols;     // allocated tensor-memory columns (512)
  int n_main;        // accumulators that take the Khi Ghi product in turn
  float *part;       // [splits][nrhs][N]
  int *err;          // error word (0 = ok)
  WaitLimits wl;     // bounded waits (clock cycles)
};


__global__ void __launch_bounds__(128, 1)
    k_gemm_bf16x3(const __grid_constant__ CUtensorMap map_khi, const __grid_constant__ CUtensorMap map_klo,
                  const __grid_constant__ CUtensorMap map_ghi, const __grid_constant__ CUtensorMap map_gmid,
                  const __grid_constant__ CUtensorMap map_glo, GemmArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment for the swizzle atoms
  unsigned char *smem = (unsigned char *)(((size_t)smem_raw + 1023) & ~(size_t)1023);
  const int a_bytes = BM * BK * 2;            // 16 KB per K operand slice
  const int b_bytes = a.rpad * BK * 2;        // rpad * 128 B per G operand slice
  const int stage_bytes = 2 * a_bytes + 3 * b_bytes;
  const int STAGES = a.stages;
  unsigned char *stages = smem;
  unsigned long long *bars = (unsigned long long *)(smem + STAGES * stage_bytes);
  // bars[0..S) full, [S..2S) empty, [2S] done
  unsigned *tmem_slot = (unsigned *)(bars + 2 * STAGES + 1);
  volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int tile = blockIdx.x, split = blockIdx.y;
  const int kb0 = split * a.kblocks_per_split;
  const int kb1 = min(a.kblocks_total, kb0 + a.kblocks_per_split);
  const int nkb = max(0, kb1 - kb0);

  if (threadIdx.x == 0) {
    for (int s = 0; s < 2 * STAGES + 1; ++s) mbar_init(su32(bars + s), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *tmem_slot;
  const unsigned idesc = idesc_bf16(BM, a.rpad);
  const unsigned idesc2 = idesc_bf16(BM, 2 * a.rpad);

  int issued_loads = 0, issued_mma = 0;
  if (warp == 0 && lane == 0) {
    // TMA producer
    for (int i = 0; i < nkb; ++i) {
      const int s = i % STAGES, use = i / STAGES;
      if (use > 0 && !mbar_wait(su32(bars + STAGES + s), (use - 1) & 1, abort_flag,
                                use == 1 && s == 0 ? a.wl.first : a.wl.limit)) {
        atomicExch(a.err, 1);
        *abort_flag = 1;
        break;
      }
      unsigned char *st = stages + s * stage_bytes;
      const unsigned full = su32(bars + s);
      mbar_arrive_expect_tx(full, (unsigned)stage_bytes);
      const int kx = (kb0 + i) * BK;
      tma_load_2d(su32(st), &map_khi, full, kx, tile * BM);
      tma_load_2d(su32(st + a_bytes), &map_klo, full, kx, tile * BM);
      tma_load_2d(su32(st + 2 * a_bytes), &map_ghi, full, kx, 0);
      tma_load_2d(su32(st + 2 * a_bytes + b_bytes), &map_gmid, full, kx, 0);
      tma_load_2d(su32(st + 2 * a_bytes + 2 * b_bytes), &map_glo, full, kx, 0);
      ++issued_loads;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    for (int i = 0; i < nkb; ++i) {
      const int s = i % STAGES, use = i / STAGES;
      if (!mbar_wait(su32(bars + s), use & 1, abort_flag, i == 0 ? a.wl.first : a.wl.limit)) {
        atomicExch(a.err, 2);
        *abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      unsigned char *st = stages + s * stage_bytes;
      const unsigned a_hi = su32(st), a_lo = su32(st + a_bytes);
      const unsigned b_hi = su32(st + 2 * a_bytes), b_mid = su32(st + 2 * a_bytes + b_bytes);
      const unsigned b_lo = su32(st + 2 * a_bytes + 2 * b_bytes);
      // accumulator columns: main_q at q * rpad (q < n_main); after them the
      // cross block of 2 rpad columns, [Khi Gmid + Klo Ghi | Khi Glo + Klo Gmid]
      const int q = i % a.n_main;
      const unsigned d_main = tmem + (unsigned)(q * a.rpad);
      const unsigned d_cross = tmem + (unsigned)(a.n_main * a.rpad);
#pragma unroll
      for (int kk = 0; kk < BK / UMMA_K; ++kk) {
        const unsigned off = kk * UMMA_K * 2;  // bytes along the swizzled row
        const unsigned first_main = (i < a.n_main && kk == 0) ? 0u : 1u;
        const unsigned first_cross = (i == 0 && kk == 0) ? 0u : 1u;
        mma_bf16(d_main, smem_desc_sw128(a_hi + off), smem_desc_sw128(b_hi + off), idesc, first_main);
        // the G slices sit back to back, so [Gmid; Glo] and [Ghi; Gmid] are
        // operands of 2 rpad rows: one instruction each for Khi and Klo
        mma_bf16(d_cross, smem_desc_sw128(a_hi + off), smem_desc_sw128(b_mid + off), idesc2, first_cross);
        mma_bf16(d_cross, smem_desc_sw128(a_lo + off), smem_desc_sw128(b_hi + off), idesc2, 1u);
      }
      mma_commit(su32(bars + STAGES + s));  // frees the stage once these MMAs finish
      ++issued_mma;
    }
    mma_commit(su32(bars + 2 * STAGES));    // accumulator complete
  }
  __syncwarp();

  // Epilogue: every warp reads its 32 TMEM lanes (rows) x rpad columns.
  bool ok = nkb > 0 && mbar_wait(su32(bars + 2 * STAGES), 0, abort_flag, a.wl.limit);
  ok = __syncthreads_and(ok) != 0;  // tcgen05.ld below must be warp-uniform
  if (!ok && nkb > 0 && threadIdx.x == 0) {
    atomicExch(a.err, 3);
    *abort_flag = 1;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const long row = (long)tile * BM + warp * 32 + lane;
  float *out = a.part + (long)split * a.nrhs * a.N;
  if (ok) {
    const unsigned lane_base = tmem + ((unsigned)(warp * 32) << 16);
    const int used = min(nkb, a.n_main);  // main accumulators that were written
    for (int c0 = 0; c0 < a.rpad; c0 += 16) {
      float v[16], w[16];
      tmem_ld16(lane_base + (unsigned)(a.n_main * a.rpad + c0), v);
      tmem_ld16(lane_base + (unsigned)((a.n_main + 1) * a.rpad + c0), w);
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] += w[i];
      for (int q = 0; q < used; ++q) {
        tmem_ld16(lane_base + (unsigned)(q * a.rpad + c0), w);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] += w[i];
      }
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (row < a.N && c0 + i < a.nrhs) out[(long)(c0 + i) * a.N + row] = v[i];
    }
  } else if (nkb == 0) {
    for (int c = 0; c < a.nrhs; ++c)
      if (row < a.N) out[(long)c * a.N + row] = 0.f;
  }
  // Before the CTA frees its shared and tensor memory, everything it issued
  // has landed, whether the run was normal (every wait below then returns at
  // once) or aborted: the producer waits for the last load of each stage (a
  // barrier's earlier phases cannot be told apart from its later ones), the
  // issuer for the accumulator commit that follows its last product.  Both
  // bounded by the full limit.
  if (warp == 0 && lane == 0) {
    const long long t0 = clock64();
    for (int s = 0; s < STAGES && s < issued_loads; ++s) {
      const int use = (issued_loads - 1 - s) / STAGES;
      while (!mbar_test(su32(bars + s), use & 1) && clock64() - t0 < a.wl.limit) {
      }
    }
  }
  if (warp == 1 && lane == 0) {
    const long long t0 = clock64();
    while (!mbar_test(su32(bars + 2 * STAGES), 0) && clock64() - t0 < a.wl.limit) {
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols)
                 : "memory");
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// 2D BF16 tensor [rows][ld] (ld elements per row), box {64, box_rows}, 128B swizzle.
vie_status make_map(CUtensorMap *m, const void *base, long ld, long rows, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled unavailable");
    return VIE_ERR_CUDA;
  }
  cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box,
                  estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed");
    return VIE_ERR_CUDA;
  }
  return VIE_OK;
}

int grid_for(long n, int threads) {
  long b = (n + threads - 1) / threads;
  return (int)std::max(1L, std::min(b, 8192L));
}

}  // namespace

// A BF16 tensor map of `rank` dimensions (dims[0] innermost, strides in bytes
// for dims 1..rank-1), box `box`, 64- or 128-byte swizzle, zero fill outside.
vie_status encode_bf16_map(CUtensorMap *m, int rank, const void *base, const unsigned long long *dims,
                           const unsigned long long *strides, const unsigned *box, int swizzle_bytes) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled unavailable");
    return VIE_ERR_CUDA;
  }
  cuuint64_t d[5], st[4];
  cuuint32_t b[5], e[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    b[i] = box[i];
    e[i] = 1;
    if (i > 0) st[i - 1] = strides[i - 1];
  }
  const CUtensorMapSwizzle sw = swizzle_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                : swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                      : CU_TENSOR_MAP_SWIZZLE_NONE;
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void *>(base), d, st, b, e,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed");
    return VIE_ERR_CUDA;
  }
  return VIE_OK;
}

vie_status launch_divide_cols(long N, int R, const double *a, long lda, const double *b, double *out, long ldo,
                              cudaStream_t st) {
  k_divide_cols<<<grid_for((long)R * N, 256), 256, 0, st>>>(N, R, a, lda, b, out, ldo);
  VIE_CHECK_LAUNCH("k_divide_cols");
  return VIE_OK;
}

vie_status launch_divide(long N, const double *a, const double *b, double *out, cudaStream_t st) {
  k_divide<<<grid_for(N, 256), 256, 0, st>>>(N, a, b, out);
  VIE_CHECK_LAUNCH("k_divide");
  return VIE_OK;
}

vie_status launch_gemv(const void *k, const void *klo, int bf16, long ldk, long N, const double *g,
                       float *g32, int op, double *y, cudaStream_t st) {
  k_to_f32_padded<<<grid_for(ldk, 256), 256, 0, st>>>(g, N, ldk, 1, g32);
  VIE_CHECK_LAUNCH("k_to_f32_padded");
  const int blocks = (int)std::min<long>((N + 7) / 8, 152L * 16);
  if (bf16)
    k_gemv<true><<<blocks, 256, 0, st>>>(k, klo, ldk, N, g32, g, op, y);
  else
    k_gemv<false><<<blocks, 256, 0, st>>>(k, nullptr, ldk, N, g32, g, op, y);
  VIE_CHECK_LAUNCH("k_gemv");
  return VIE_OK;
}

// FP32 split-K partials, rounded up so the BF16 G operands after them start on
// a 256-byte boundary (TMA wants 16).
static size_t part_region_bytes(int splits, int nrhs, long N) {
  return ((sizeof(float) * (size_t)splits * nrhs * N) + 255) & ~(size_t)255;
}

// Main accumulators for a given width: they and the cross block (2 rpad
// columns) fill at most the 512 tensor-memory columns.
static int n_main_for(int rpad) { return std::max(1, std::min(7, 512 / rpad - 2)); }
// Longest chain of MMAs into one accumulator (a drift of ~1e-6 relative).
constexpr int kMaxChain = 32;

size_t gemm_workspace_bytes(long N, long ldk, int nrhs, int *splits_out, int sms) {
  const long tiles = (N + BM - 1) / BM;
  const int kblocks = (int)(ldk / BK);
  const int rpad = (nrhs + 15) / 16 * 16;
  const int nm = n_main_for(rpad);
  // At most kMaxChain chained MMAs per accumulator; above that bound, the
  // split count whose CTAs (one per SM) stream K in the fewest bytes-times:
  // waves x the K slices of one split, plus the FP32 partials each split
  // writes and the finish kernel reads back.
  const long by_chain = (4L * kblocks + (long)nm * kMaxChain - 1) / ((long)nm * kMaxChain);
  const long s0 = std::max(1L, std::min<long>(kblocks, by_chain));
  long splits_best = s0;
  double cost_best = 0.0;
  for (long s = s0; s <= std::min<long>(kblocks, s0 + 64); ++s) {
    const long per = (kblocks + s - 1) / s;
    if (s > s0 && (s - 1) * per >= kblocks) continue;  // a split would be empty
    const double waves = (double)((tiles * s + sms - 1) / sms);
    const double cost = waves * sms * per * (2.0 * BM * BK * 2) + s * 8.0 * nrhs * N;
    if (s == s0 || cost < cost_best) {
      cost_best = cost;
      splits_best = s;
    }
  }
  int splits = (int)splits_best;
  if (splits_out) *splits_out = splits;
  return part_region_bytes(splits, nrhs, N) + 3 * sizeof(short) * (size_t)rpad * ldk;
}

vie_status launch_gemm_bf16x3(const void *khi, const void *klo, long ldk, long N, const double *g, long ldg,
                              int nrhs, int op, double *y, long ldy, void *workspace, int *err,
                              cudaStream_t st) {
  if (nrhs < 1 || nrhs > kGemmMaxRhs) {
    set_error("BF16 product: 1 <= nrhs <= 128");
    return VIE_ERR_INVALID_ARG;
  }
  int dev = 0, sms = 0;
  VIE_CUDA(cudaGetDevice(&dev));
  VIE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int splits = 1;
  gemm_workspace_bytes(N, ldk, nrhs, &splits, sms);
  const int rpad = (nrhs + 15) / 16 * 16;
  float *part = (float *)workspace;
  __nv_bfloat16 *ghi = (__nv_bfloat16 *)((unsigned char *)workspace + part_region_bytes(splits, nrhs, N));
  __nv_bfloat16 *gmid = ghi + (size_t)rpad * ldk, *glo = gmid + (size_t)rpad * ldk;
  k_split_bf16<<<dim3((unsigned)std::min<long>((ldk / 2 + 255) / 256, 1024L), (unsigned)rpad), 256, 0, st>>>(
      g, ldg, N, ldk, nrhs, ghi, gmid, glo);
  VIE_CHECK_LAUNCH("k_split_bf16");
  CUtensorMap mkhi, mklo, mghi, mgmid, mglo;
  vie_status s;
  if ((s = make_map(&mkhi, khi, ldk, N, BM)) != VIE_OK) return s;
  if ((s = make_map(&mklo, klo, ldk, N, BM)) != VIE_OK) return s;
  if ((s = make_map(&mghi, ghi, ldk, rpad, rpad)) != VIE_OK) return s;
  if ((s = make_map(&mgmid, gmid, ldk, rpad, rpad)) != VIE_OK) return s;
  if ((s = make_map(&mglo, glo, ldk, rpad, rpad)) != VIE_OK) return s;
  GemmArgs a;
  a.rpad = rpad;
  a.nrhs = nrhs;
  a.N = N;
  a.kblocks_total = (int)(ldk / BK);
  a.kblocks_per_split = (a.kblocks_total + splits - 1) / splits;
  a.n_main = n_main_for(rpad);
  a.tmem_cols = 512;  // one CTA per SM (shared memory), so the whole TMEM is free
  a.part = part;
  a.err = err;
  a.wl = wait_limits(dev);
  const size_t stage_bytes = (size_t)(2 * BM * BK * 2 + 3 * rpad * BK * 2);
  int optin = 0;
  VIE_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  a.stages = (int)std::min<size_t>(MAX_STAGES, ((size_t)optin - 1024 - 256) / stage_bytes);
  if (a.stages < 2) {
    set_error("BF16 product: not enough shared memory for two stages");
    return VIE_ERR_UNSUPPORTED;
  }
  const size_t smem = 1024 + a.stages * stage_bytes + 256;
  VIE_TRY(raise_smem_limit((const void *)k_gemm_bf16x3, (size_t)((int)smem)));
  dim3 grid((unsigned)((N + BM - 1) / BM), (unsigned)splits);
  k_gemm_bf16x3<<<grid, 128, smem, st>>>(mkhi, mklo, mghi, mgmid, mglo, a);
  VIE_CHECK_LAUNCH("k_gemm_bf16x3");
  k_gemm_finish<<<dim3((unsigned)std::min<long>((N + 1023) / 1024, 1024L), (unsigned)nrhs), 256, 0, st>>>(
      part, splits, nrhs, N, g, ldg, op, err, y, ldy);
  VIE_CHECK_LAUNCH("k_gemm_finish");
  return VIE_OK;
}

}  // namespace vie
