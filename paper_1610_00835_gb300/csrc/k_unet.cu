// Learned right preconditioner: a small convolutional U-Net, trained and
// evaluated with this library's own kernels.  The paper preconditions its
// Krylov solve with FFT and diffusion solvers (Section 4.4); here a network
// maps (sigma_t, sigma_s, b) to the smooth part of (I - K)^{-1} b, and FGMRES
// (vie_solve_gmres with a preconditioner set) absorbs that it is nonlinear.
//
// Network (L levels, C channels; tensors FP32 NCHW, weights [Co][Ci][k][k]):
//   encoder l = 0..L-1: a_l = relu(conv3(x_l)), e_l = relu(conv3(a_l)),
//                       x_0 = input (3 channels), x_l = avgpool2(e_{l-1});
//   decoder l = L-2..0: c_l = [upsample2(d_{l+1}), e_l], b_l = relu(conv3(c_l)),
//                       d_l = relu(conv3(b_l)), d_{L-1} = e_{L-1};
//   output  o = conv1(d_0).
// e_l (l < L-1) is written straight into the second half of c_l's channels.
// Training minimises mean((o - t)^2) with Adam; inference can use a BF16 copy
// of the weights (FP32 accumulation either way).
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <type_traits>
#include <string>
#include <vector>

#include "tcgen05.cuh"
#include "vie_internal.cuh"

namespace vie {

namespace {

constexpr int TX = 32;            // output tile width of the 3x3 convolution kernels
constexpr int CIB = 8;            // input channels staged per step
constexpr int COB = 32;           // output channels per CTA of the weight-gradient kernel

// ------------------------------------------------------------ kernels

// 3x3 convolution, zero padding 1, + bias (+ relu).  A CTA computes a TX x TY
// pixel tile for COBC output channels; thread (tx, ty), ty in 0..7, owns the
// pixels (x0 + tx, y0 + ty + 8 k), k < TY / 8, for all COBC outputs.  Every
// output sums its input channels and taps in the same order whatever TY and
// COBC are, so the tile shape changes no result bit.
template <bool RELU, typename WT, int TY, int COBC>
__global__ void __launch_bounds__(256) k_conv3(const float *__restrict__ in, long in_bs, int Ci,
                                               const WT *__restrict__ w, const float *__restrict__ bias,
                                               float *__restrict__ out, long out_bs, int Co, int H,
                                               int W, int co_blocks) {
  static_assert(TY % 8 == 0 && COBC % 4 == 0, "tile shape");
  constexpr int PY = TY / 8;
  __shared__ float in_s[CIB][TY + 2][TX + 2];
  __shared__ __align__(16) float w_s[CIB][9][COBC];
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;  // ty in 0..7
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int b = blockIdx.z / co_blocks, cb = blockIdx.z % co_blocks;
  const int co0 = cb * COBC;
  float acc[PY][COBC];
#pragma unroll
  for (int k = 0; k < PY; ++k)
#pragma unroll
    for (int c = 0; c < COBC; ++c) acc[k][c] = 0.f;
  const float *inb = in + b * in_bs;
  const long plane = (long)H * W;
  // Each step stages CIB input channels: the padded pixel tile through
  // asynchronous 4-byte copies (zero-filled outside the image), the weights
  // through registers, all loads in flight together.  Flat index i of a
  // staging array is its shared-memory offset.
  constexpr int IN_N = CIB * (TY + 2) * (TX + 2);
  constexpr int W_N = CIB * 9 * COBC, W_K = (W_N + 255) / 256;
  const unsigned in_s0 = (unsigned)__cvta_generic_to_shared(&in_s[0][0][0]);
  for (int ci0 = 0; ci0 < Ci; ci0 += CIB) {
    __syncthreads();
    for (int i = threadIdx.x; i < IN_N; i += 256) {
      const int c = i / ((TY + 2) * (TX + 2)), r = i % ((TY + 2) * (TX + 2));
      const int gy = y0 - 1 + r / (TX + 2), gx = x0 - 1 + r % (TX + 2);
      const bool ok = ci0 + c < Ci && gy >= 0 && gy < H && gx >= 0 && gx < W;
      const float *src = ok ? inb + (ci0 + c) * plane + (long)gy * W + gx : inb;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(in_s0 + 4u * i), "l"(src),
                   "r"(ok ? 4 : 0)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    float pwt[W_K];
#pragma unroll
    for (int k = 0; k < W_K; ++k) {
      const int i = threadIdx.x + 256 * k;
      const int c = i / (9 * COBC), r = i % (9 * COBC);
      const int tap = r / COBC, co = r % COBC;
      pwt[k] = i < W_N && ci0 + c < Ci && co0 + co < Co
                   ? (float)w[((long)(co0 + co) * Ci + ci0 + c) * 9 + tap]
                   : 0.f;
    }
#pragma unroll
    for (int k = 0; k < W_K; ++k)
      if (threadIdx.x + 256 * k < W_N) (&w_s[0][0][0])[threadIdx.x + 256 * k] = pwt[k];
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
#pragma unroll 1
    for (int c = 0; c < CIB; ++c) {
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3, dx = tap % 3;
        float v[PY];
#pragma unroll
        for (int k = 0; k < PY; ++k) v[k] = in_s[c][ty + 8 * k + dy][tx + dx];
        const float4 *wr = reinterpret_cast<const float4 *>(&w_s[c][tap][0]);
#pragma unroll
        for (int q = 0; q < COBC / 4; ++q) {
          const float4 wv = wr[q];
#pragma unroll
          for (int k = 0; k < PY; ++k) {
            acc[k][4 * q + 0] = fmaf(v[k], wv.x, acc[k][4 * q + 0]);
            acc[k][4 * q + 1] = fmaf(v[k], wv.y, acc[k][4 * q + 1]);
            acc[k][4 * q + 2] = fmaf(v[k], wv.z, acc[k][4 * q + 2]);
            acc[k][4 * q + 3] = fmaf(v[k], wv.w, acc[k][4 * q + 3]);
          }
        }
      }
    }
  }
  const int x = x0 + tx;
  float *ob = out + b * out_bs;
#pragma unroll
  for (int c = 0; c < COBC; ++c) {
    const int co = co0 + c;
    if (co >= Co || x >= W) continue;
    const float bv = bias ? bias[co] : 0.f;
#pragma unroll
    for (int k = 0; k < PY; ++k) {
      const int yk = y0 + ty + 8 * k;
      float vk = acc[k][c] + bv;
      if (RELU) vk = fmaxf(vk, 0.f);
      if (yk < H) ob[co * plane + (long)yk * W + x] = vk;
    }
  }
}

// Tensor-core convolution tiles: 128 TMEM lanes (pixels) per tile.
constexpr int kTcM = 128;

// The BF16 convolution as an implicit GEMM fed by the tensor memory
// accelerator.  The input is first rounded to BF16 and laid out NHWC with its
// channels padded to S slices of 32 (k_to_nhwc_bf16).  A tile is 128 TMEM
// lanes = R rows x Wb pixels of one image (Wb = min(W, 128), R = 128 / Wb);
// for each tap (dy, dx) and channel slice the A operand is the input shifted
// by the tap: one TMA box (32 channels, Wb, R, 1) at (slice, x0 + dx - 1,
// y0 + dy - 1, image), whose out-of-image part the TMA fills with zeros --
// exactly the zero padding of the convolution.  Its rows are 64 bytes (32
// BF16 along K), written with the 64-byte swizzle that the MMA's K-major
// descriptor reads.  The B operand of the same step is the weights' [Co][32]
// block of that tap and slice (packed by k_pack_tc_weights).
//
// Two CTAs per SM (half of its shared memory each) take tiles blockIdx.x,
// blockIdx.x + G, ... in a warp-specialised pipeline: the weights are loaded once; warp 4 streams the A
// boxes of its tiles into a ring of nst stages (a tile of one image row
// takes, per slice, its 3 input rows once as boxes of Wb + 2 pixels, and the
// MMAs read the 3 taps of a row at 64-byte offsets into them: a third of the
// TMA rows; other tiles take one box per tap and slice); warp 5 issues two
// tcgen05.mma (M = 128, N = Co, K = 16) per tap into one of kAcc tensor-
// memory accumulators (FP32), committing each stage back to the producer and
// each finished tile to the epilogue; warps 0-3 read their 32 lanes of a
// finished accumulator, hand it back, add the bias (and relu) and write FP32
// NCHW, while the next tiles' loads and products run.  Waits are bounded (wl;
// the first operand wait takes wl.first).  On expiry the CTA stops issuing,
// writes NaN for the tiles it has not finished, sets *err, waits (bounded by
// wl.limit) for the loads and products it issued and frees its tensor memory.
constexpr int kTmaSlice = 32;   // channels per K slice (64 bytes of BF16)
constexpr int kAcc = 4;         // tensor-memory accumulators (Co <= 32 columns each)
constexpr int kConvThreads = 192;

// one ring stage: a tap box of 128 pixels, or a halo box of Wb + 2 (Wb = 128)
// rounded up to 1024 bytes
__host__ __device__ inline int conv_stage_bytes(int Wb) { return Wb == kTcM ? 9216 : kTcM * 64; }
// ring stages of a CTA with `budget` bytes of shared memory
// (np = 2: split precision, operands in two parts)
int conv_stages(int S, int Co, int Wb, size_t budget, int np = 1) {
  const size_t b = (size_t)np * 9 * S * Co * 64, fixed = 1024 + b + 1024;
  if (budget <= fixed) return 0;
  return (int)std::min<size_t>(32, (budget - fixed) / ((size_t)np * conv_stage_bytes(Wb)));
}
size_t conv_tma_smem(int S, int Co, int Wb, int nst, int np = 1) {
  return 1024 + (size_t)np * 9 * S * Co * 64 + (size_t)nst * np * conv_stage_bytes(Wb) + 8 * (2 * nst + 2 * kAcc + 2) +
         16;
}

// NP > 1: the FP32 convolutions of training in split precision: input and
// weights each as NP BF16 parts (v = p0 + p1 [+ p2], each part the BF16
// rounding of what the earlier ones leave; map_x1 / map_w1, map_x2 / map_w2
// the later parts), every tap the products of parts i, j with i + j < NP
// into the FP32 accumulator (the terms left out are below 2^-8 NP of the
// kept ones: 2^-16 for two parts, 2^-24 for three); a stage holds the parts'
// boxes one after the other.
template <bool RELU, int NP>
__global__ void __launch_bounds__(kConvThreads, 2)
    k_conv3_tma(const __grid_constant__ CUtensorMap map_x, const __grid_constant__ CUtensorMap map_w,
                const __grid_constant__ CUtensorMap map_x1, const __grid_constant__ CUtensorMap map_w1,
                const __grid_constant__ CUtensorMap map_x2, const __grid_constant__ CUtensorMap map_w2,
                const float *__restrict__ bias, float *__restrict__ out, long out_bs, int Co, int H, int W, int S,
                int Wb, int R, int tiles_x, int tiles, int nst, WaitLimits wl, int *err,
                __nv_bfloat16 *__restrict__ out_h, long oh_bs, int oh_cp, int oh_c0) {
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = (unsigned char *)(((size_t)smem_raw + 1023) & ~(size_t)1023);
  // halo: tiles of one image row take, per slice, the 3 input rows once
  // (Wb + 2 pixels each) and the 3 taps of a row as 64-byte offsets into
  // that box; other tiles take one box per tap and slice
  const bool halo = R == 1;
  const int steps = (halo ? 3 : 9) * S, taps_step = halo ? 3 : 1;
  const int tiles_img = tiles_x * ((H + R - 1) / R);
  const int a_part = conv_stage_bytes(Wb), a_bytes = NP * a_part, b_bytes = Co * 64;
  const size_t b_part = (size_t)9 * S * b_bytes;  // one part of the weights
  unsigned char *Bs = smem;
  unsigned char *As = smem + (size_t)NP * b_part;
  unsigned long long *full = (unsigned long long *)(As + (size_t)nst * a_bytes);
  unsigned long long *empty = full + nst, *tfull = empty + nst, *tempty = tfull + kAcc;
  unsigned long long *wbar = tempty + kAcc, *done = wbar + 1;
  unsigned *tmem_slot = (unsigned *)(done + 1);
  volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int G = gridDim.x;
  if (tid == 0) {
    for (int i = 0; i < nst; ++i) {
      mbar_init(su32(full + i), 1);
      mbar_init(su32(empty + i), 1);
    }
    for (int i = 0; i < kAcc; ++i) {
      mbar_init(su32(tfull + i), 1);
      mbar_init(su32(tempty + i), 4);  // one arrival per epilogue warp
    }
    mbar_init(su32(wbar), 1);
    mbar_init(su32(done), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(kAcc * 32)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *tmem_slot;
  const unsigned box_bytes = (unsigned)(kTmaSlice * 2 * (halo ? Wb + 2 : Wb * R));
  int issued_loads = 0;
  if (warp == 4 && lane == 0) {
    // TMA producer: the weights once, then every step's shifted input box
    mbar_arrive_expect_tx(su32(wbar), (unsigned)(NP * 9 * S * b_bytes));
    for (int k = 0; k < 9 * S; ++k) {
      tma_load_2d(su32(Bs + (size_t)k * b_bytes), &map_w, su32(wbar), 0, k * Co);
      if (NP > 1) tma_load_2d(su32(Bs + b_part + (size_t)k * b_bytes), &map_w1, su32(wbar), 0, k * Co);
      if (NP > 2) tma_load_2d(su32(Bs + 2 * b_part + (size_t)k * b_bytes), &map_w2, su32(wbar), 0, k * Co);
    }
    int g = 0;
    bool go = true;
    for (int t = blockIdx.x; t < tiles && go; t += G) {
      const int img = t / tiles_img, r = t - img * tiles_img;
      const int x0 = (r % tiles_x) * Wb, y0 = (r / tiles_x) * R;
      for (int k = 0; k < steps; ++k, ++g) {
        const int st = g % nst, use = g / nst;
        if (use > 0 && !mbar_wait(su32(empty + st), (use - 1) & 1, abort_flag, wl.limit)) {
          atomicExch(err, 1);
          *abort_flag = 1;
          go = false;
          break;
        }
        // step k: slice sl of input row dy (halo) or of tap (dy, dx)
        const int q = k / S, sl = k - q * S;
        const int dy = halo ? q : q / 3, dx = halo ? 0 : q % 3;
        mbar_arrive_expect_tx(su32(full + st), NP * box_bytes);
        tma_load_4d(su32(As + (size_t)st * a_bytes), &map_x, su32(full + st), sl * kTmaSlice, x0 + dx - 1,
                    y0 + dy - 1, img);
        if (NP > 1)
          tma_load_4d(su32(As + (size_t)st * a_bytes + a_part), &map_x1, su32(full + st), sl * kTmaSlice,
                      x0 + dx - 1, y0 + dy - 1, img);
        if (NP > 2)
          tma_load_4d(su32(As + (size_t)st * a_bytes + 2 * a_part), &map_x2, su32(full + st), sl * kTmaSlice,
                      x0 + dx - 1, y0 + dy - 1, img);
        ++issued_loads;
      }
    }
  } else if (warp == 5 && lane == 0) {
    // MMA issuer
    const unsigned idesc = idesc_bf16(kTcM, Co);
    bool go = mbar_wait(su32(wbar), 0, abort_flag, wl.first);
    int g = 0, j = 0;
    for (int t = blockIdx.x; t < tiles && go; t += G, ++j) {
      const int b = j % kAcc;
      if (j >= kAcc && !mbar_wait(su32(tempty + b), (j / kAcc - 1) & 1, abort_flag, wl.limit)) {
        go = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned d = tmem + (unsigned)(b * 32);
      for (int k = 0; k < steps; ++k, ++g) {
        const int st = g % nst;
        if (!mbar_wait(su32(full + st), (g / nst) & 1, abort_flag, g == 0 ? wl.first : wl.limit)) {
          go = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int q = k / S, sl = k - q * S;
        for (int e = 0; e < taps_step; ++e) {
          // tap (dy, dx): its weights, and its input rows e pixels into a halo box
          const int tap = halo ? 3 * q + e : q;
          const unsigned a = su32(As + (size_t)st * a_bytes) + 64u * (unsigned)e;
          const unsigned bb = su32(Bs + (size_t)(tap * S + sl) * b_bytes);
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
            // parts i of the input and j of the weights, i + j < NP
#pragma unroll
            for (int i = 0; i < NP; ++i)
#pragma unroll
              for (int j = 0; i + j < NP; ++j) {
                const unsigned ai = a + (unsigned)(i * a_part) + kk * 32;
                const unsigned bj = bb + (unsigned)(j * b_part) + kk * 32;
                mma_bf16(d, smem_desc_sw64(ai), smem_desc_sw64(bj), idesc,
                         (k > 0 || e > 0 || kk > 0 || i > 0 || j > 0) ? 1u : 0u);
              }
          }
        }
        mma_commit(su32(empty + st));  // the stage is free once these products finish
      }
      if (!go) break;
      mma_commit(su32(tfull + b));     // the tile's accumulator is complete
    }
    if (!go) {
      atomicExch(err, 1);
      *abort_flag = 1;
    }
    mma_commit(su32(done));            // every product this thread issued
  } else if (warp < 4) {
    // epilogue: warp w reads TMEM lanes 32 w .. 32 w + 31
    const int i = warp * 32 + lane;  // this thread's lane: pixel (x0 + i % Wb, y0 + i / Wb) of the tile
    const long plane = (long)H * W;
    float bv[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) bv[c] = bias && c < Co ? bias[c] : 0.f;
    int j = 0;
    for (int t = blockIdx.x; t < tiles; t += G, ++j) {
      const int b = j % kAcc;
      const int img = t / tiles_img, r = t - img * tiles_img;
      const int px = (r % tiles_x) * Wb + i % Wb, py = (r / tiles_x) * R + i / Wb;
      const bool pvalid = i < Wb * R && px < W && py < H;
      bool ok = *abort_flag == 0 && mbar_wait(su32(tfull + b), (j / kAcc) & 1, abort_flag, wl.limit);
      ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective
      float v[32];
      if (ok) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned ta = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)(b * 32);
        tmem_ld16(ta, v);
        if (Co > 16) tmem_ld16(ta + 16, v + 16);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(su32(tempty + b));  // the accumulator may be overwritten
      } else if (lane == 0) {
        atomicExch(err, 1);
        *abort_flag = 1;
      }
      float *ob = out + img * out_bs + (long)py * W + px;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        float x = ok ? v[c] + bv[c] : __int_as_float(0x7fc00000);
        if (RELU && ok) x = fmaxf(x, 0.f);
        v[c] = x;
        if (c < Co && pvalid) ob[(long)c * plane] = x;
      }
      if (out_h && pvalid) {
        // the same values in BF16 for the next convolution's NHWC input:
        // channels oh_c0 .. oh_c0 + Co of this pixel, 16 bytes at a time
        uint4 *hp = reinterpret_cast<uint4 *>(out_h + img * oh_bs + ((long)py * W + px) * oh_cp + oh_c0);
#pragma unroll
        for (int g8 = 0; g8 < 4; ++g8) {
          if (8 * g8 >= Co) break;
          unsigned w4[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const __nv_bfloat162 q2 = __floats2bfloat162_rn(v[8 * g8 + 2 * e], v[8 * g8 + 2 * e + 1]);
            w4[e] = *reinterpret_cast<const unsigned *>(&q2);
          }
          hp[g8] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        }
      }
    }
  }
  __syncwarp();
  // everything issued has landed before shared and tensor memory are released
  // (bounded by the full limit): the producer waits for the weights and for
  // the last load into each stage, the issuer for its last commit
  if (warp == 4 && lane == 0) {
    const long long t0 = clock64();
    while (!mbar_test(su32(wbar), 0) && clock64() - t0 < wl.limit) {
    }
    for (int s = 0; s < nst && s < issued_loads; ++s) {
      const int use = (issued_loads - 1 - s) / nst;
      while (!mbar_test(su32(full + s), use & 1) && clock64() - t0 < wl.limit) {
      }
    }
  }
  if (warp == 5 && lane == 0) {
    const long long t0 = clock64();
    while (!mbar_test(su32(done), 0) && clock64() - t0 < wl.limit) {
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 5) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kAcc * 32) : "memory");
  }
}

// in: FP32 [B][Ci][plane] (image stride in_bs) -> BF16 [B][plane][Cp], rounded
// to nearest even, channels Ci..Cp-1 zero.  One thread per (image, pixel):
// a warp reads 32 consecutive pixels of a channel plane at a time and writes
// its pixels' Cp channels as 16-byte groups.
__global__ void k_to_nhwc_bf16(const float *__restrict__ in, long in_bs, int Ci, long plane, int Cp, int B,
                               __nv_bfloat16 *__restrict__ out) {
  const long total = (long)B * plane;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const long b = t / plane, p = t - b * plane;
    const float *src = in + b * in_bs + p;
    uint4 *dst = reinterpret_cast<uint4 *>(out + t * Cp);
    for (int gq = 0; gq < Cp / 8; ++gq) {
      unsigned w[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int c = gq * 8 + 2 * e;
        const float lo = c < Ci ? src[(long)c * plane] : 0.f, hi = c + 1 < Ci ? src[(long)(c + 1) * plane] : 0.f;
        const __nv_bfloat162 q = __floats2bfloat162_rn(lo, hi);
        w[e] = *reinterpret_cast<const unsigned *>(&q);
      }
      dst[gq] = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// Weights of one 3x3 convolution, FP32 [Co][Ci][9] -> BF16 [9 S][Co][32]:
// block k = tap S + slice holds w[co][slice 32 + c][tap] (zero past Ci).
__global__ void k_pack_tc_weights(const float *__restrict__ w, int Co, int Ci, int S,
                                  __nv_bfloat16 *__restrict__ out) {
  const long total = (long)9 * S * Co * kTmaSlice;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int c = (int)(t % kTmaSlice);
    const long r = t / kTmaSlice;
    const int co = (int)(r % Co);
    const int k = (int)(r / Co);
    const int tap = k / S, ci = (k - tap * S) * kTmaSlice + c;
    out[t] = __float2bfloat16_rn(ci < Ci ? w[((long)co * Ci + ci) * 9 + tap] : 0.f);
  }
}

// The split-precision operands of training: v = p0 + p1 [+ p2], p0 = bf16(v),
// each later part the BF16 rounding of what the earlier ones leave (exact in
// FP32): 16 significant bits for two parts, 24 (all of FP32's) for three.
__device__ __forceinline__ void split_parts(float v, int np, __nv_bfloat16 (&part)[3]) {
  float r = v;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    part[q] = __float2bfloat16_rn(q < np ? r : 0.f);
    r -= __bfloat162float(part[q]);
  }
}

// Input: FP32 [B][Ci][plane] -> NP BF16 parts [B][plane][Cp] (out0, out1,
// out2), one thread per (image, pixel) as in k_to_nhwc_bf16.
template <int NP>
__global__ void k_to_nhwc_split(const float *__restrict__ in, long in_bs, int Ci, long plane, int Cp, int B,
                                __nv_bfloat16 *__restrict__ out0, __nv_bfloat16 *__restrict__ out1,
                                __nv_bfloat16 *__restrict__ out2) {
  const long total = (long)B * plane;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const long b = t / plane, p = t - b * plane;
    const float *src = in + b * in_bs + p;
    for (int gq = 0; gq < Cp / 8; ++gq) {
      unsigned w[3][4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int c = gq * 8 + 2 * e;
        __nv_bfloat16 p0[3], p1[3];
        split_parts(c < Ci ? src[(long)c * plane] : 0.f, NP, p0);
        split_parts(c + 1 < Ci ? src[(long)(c + 1) * plane] : 0.f, NP, p1);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const __nv_bfloat162 h2 = __halves2bfloat162(p0[q], p1[q]);
          w[q][e] = *reinterpret_cast<const unsigned *>(&h2);
        }
      }
      reinterpret_cast<uint4 *>(out0 + t * Cp)[gq] = make_uint4(w[0][0], w[0][1], w[0][2], w[0][3]);
      if (NP > 1) reinterpret_cast<uint4 *>(out1 + t * Cp)[gq] = make_uint4(w[1][0], w[1][1], w[1][2], w[1][3]);
      if (NP > 2) reinterpret_cast<uint4 *>(out2 + t * Cp)[gq] = make_uint4(w[2][0], w[2][1], w[2][2], w[2][3]);
    }
  }
}

// Weights FP32 [Co][Ci][9], output channels co0 .. co0 + cb -> np BF16 parts
// [9 S][cb][32] in k_pack_tc_weights's block order.
__global__ void k_pack_split_weights(const float *__restrict__ w, int Co, int Ci, int S, int co0, int cb, int np,
                                     __nv_bfloat16 *__restrict__ w0, __nv_bfloat16 *__restrict__ w1,
                                     __nv_bfloat16 *__restrict__ w2) {
  const long total = (long)9 * S * cb * kTmaSlice;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int c = (int)(t % kTmaSlice);
    const long r = t / kTmaSlice;
    const int co = co0 + (int)(r % cb);
    const int k = (int)(r / cb);
    const int tap = k / S, ci = (k - tap * S) * kTmaSlice + c;
    __nv_bfloat16 part[3];
    split_parts(ci < Ci && co < Co ? w[((long)co * Ci + ci) * 9 + tap] : 0.f, np, part);
    w0[t] = part[0];
    if (np > 1) w1[t] = part[1];
    if (np > 2) w2[t] = part[2];
  }
}

// Gradient of a 3x3 convolution's weights and bias over one 32 x 8 pixel tile
// of images b0 .. b1 and 8 input channels; thread (co, ci) keeps its 9 taps
// over those images and adds them into dw with atomics once.  A 3 x 3 window
// of the input slides along x in registers.
constexpr int WY = 8;
__global__ void __launch_bounds__(256, 3) k_conv3_dw(const float *__restrict__ x, long x_bs, int Ci,
                                                  const float *__restrict__ gy, long g_bs, int Co,
                                                  int H, int W, float *__restrict__ dw,
                                                  float *__restrict__ db, int ci_blocks,
                                                  int co_blocks, int B, int b_splits) {
  __shared__ float g_s[COB][WY * TX + 1];
  __shared__ float x_s[CIB][WY + 2][TX + 2];
  const int co_l = threadIdx.x % 32, ci_l = threadIdx.x / 32;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * WY;
  int z = blockIdx.z;
  const int cib = z % ci_blocks;
  z /= ci_blocks;
  const int cob = z % co_blocks;
  const int bs = z / co_blocks;
  const int ci0 = cib * CIB, co0 = cob * COB;
  const long plane = (long)H * W;
  float acc[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) acc[t] = 0.f;
  float bsum = 0.f;
  const int b_lo = (int)((long)B * bs / b_splits), b_hi = (int)((long)B * (bs + 1) / b_splits);
  for (int b = b_lo; b < b_hi; ++b) {
  if (b > b_lo) __syncthreads();  // the previous image's tiles are consumed
  for (int i = threadIdx.x; i < COB * WY * TX; i += 256) {
    const int c = i / (WY * TX), p = i % (WY * TX);
    const int yy = p / TX, xx = p % TX;
    const int gyy = y0 + yy, gxx = x0 + xx;
    float v = 0.f;
    if (co0 + c < Co && gyy < H && gxx < W) v = gy[b * g_bs + (co0 + c) * plane + (long)gyy * W + gxx];
    g_s[c][p] = v;
  }
  for (int i = threadIdx.x; i < CIB * (WY + 2) * (TX + 2); i += 256) {
    const int c = i / ((WY + 2) * (TX + 2)), r = i % ((WY + 2) * (TX + 2));
    const int yy = r / (TX + 2), xx = r % (TX + 2);
    const int gyy = y0 - 1 + yy, gxx = x0 - 1 + xx;
    float v = 0.f;
    if (ci0 + c < Ci && gyy >= 0 && gyy < H && gxx >= 0 && gxx < W)
      v = x[b * x_bs + (ci0 + c) * plane + (long)gyy * W + gxx];
    x_s[c][yy][xx] = v;
  }
  __syncthreads();
  for (int yy = 0; yy < WY; ++yy) {
    float win[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      win[r][0] = x_s[ci_l][yy + r][0];
      win[r][1] = x_s[ci_l][yy + r][1];
    }
    // unrolled by four along the row: the window's shift is register
    // renaming within each group
#pragma unroll 4
    for (int xx = 0; xx < TX; ++xx) {
#pragma unroll
      for (int r = 0; r < 3; ++r) win[r][2] = x_s[ci_l][yy + r][xx + 2];
      const float g = g_s[co_l][yy * TX + xx];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[r * 3 + c] = fmaf(g, win[r][c], acc[r * 3 + c]);
      if (ci_l == 0) bsum += g;  // the bias gradient: warp 0 alone adds it
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        win[r][0] = win[r][1];
        win[r][1] = win[r][2];
      }
    }
  }
  }
  const int co = co0 + co_l, ci = ci0 + ci_l;
  if (co < Co && ci < Ci) {
#pragma unroll
    for (int t = 0; t < 9; ++t) atomicAdd(&dw[((long)co * Ci + ci) * 9 + t], acc[t]);
  }
  if (db && cib == 0 && ci_l == 0 && co < Co) atomicAdd(&db[co], bsum);
}

// wt[ci][co][8 - tap] = w[co][ci][tap]: the adjoint of a 3x3 convolution with
// zero padding is the convolution with the flipped, transposed kernel.
__global__ void k_flip(const float *__restrict__ w, int Co, int Ci, float *__restrict__ wt) {
  const long total = (long)Co * Ci * 9;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long co = i / (Ci * 9), r = i % (Ci * 9), ci = r / 9, tap = r % 9;
    wt[(ci * Co + co) * 9 + (8 - tap)] = w[i];
  }
}

// 1x1 convolution to one channel: o = sum_c w_c d_c + b
template <typename WT>
__global__ void k_head(const float *__restrict__ d, long d_bs, int C, const WT *__restrict__ w,
                       const float *__restrict__ bias, float *__restrict__ o, long plane, int B) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < (long)B * plane; i += (long)gridDim.x * blockDim.x) {
    const long b = i / plane, p = i % plane;
    float s = bias[0];
    for (int c = 0; c < C; ++c) s = fmaf((float)w[c], d[b * d_bs + c * plane + p], s);
    o[i] = s;
  }
}

// head backward: dd_c = w_c go (written), dw_c += sum go d_c, db += sum go
__global__ void k_head_bwd_data(const float *__restrict__ go, int C, const float *__restrict__ w,
                                float *__restrict__ dd, long dd_bs, long plane, int B) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < (long)B * plane * C; i += (long)gridDim.x * blockDim.x) {
    const long b = i / (plane * C), r = i % (plane * C), c = r / plane, p = r % plane;
    dd[b * dd_bs + c * plane + p] = w[c] * go[b * plane + p];
  }
}

// Gradient of the 1x1 head's weights and bias in two passes, deterministic:
// block (c, k) sums channel c's products (c == C: the bias) over the k-th of
// gridDim.y slices of the B planes into part[c][k]; k_head_bwd_w_finish adds
// each channel's slices in order.
__global__ void k_head_bwd_w(const float *__restrict__ go, const float *__restrict__ d, long d_bs, int C,
                             long plane, int B, double *__restrict__ part) {
  __shared__ double red[256];
  const int c = blockIdx.x, k = blockIdx.y, K = gridDim.y;
  const long total = (long)B * plane, i0 = total * k / K, i1 = total * (k + 1) / K;
  float s = 0.f;  // a few dozen terms per thread in FP32; the block's sum in FP64
  for (long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const long b = i / plane, p = i - b * plane;
    s += go[i] * (c < C ? d[b * d_bs + c * plane + p] : 1.f);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[c * K + k] = red[0];
}

__global__ void k_head_bwd_w_finish(const double *__restrict__ part, int C, int K, float *__restrict__ dw,
                                    float *__restrict__ db) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c > C) return;
  double s = 0.0;
  for (int k = 0; k < K; ++k) s += part[c * K + k];
  if (c < C)
    dw[c] += (float)s;
  else
    db[0] += (float)s;
}

// The 2x2 pooling and upsampling kernels take one thread per coarse pixel of
// one plane (blockIdx.y = b C + c): 32-bit pixel arithmetic, the fine pixels
// of a row pair as float2.  H, W: the fine size (even).
__device__ __forceinline__ bool coarse_pixel(int H, int W, int C, int &b, int &c, int &y, int &x, int &q) {
  const int Wo = W / 2;
  q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (H / 2) * Wo) return false;
  b = blockIdx.y / C;
  c = blockIdx.y - b * C;
  y = q / Wo;
  x = q - y * Wo;
  return true;
}
dim3 coarse_grid(int H, int W, int C, int B) { return dim3((unsigned)(((H / 2) * (W / 2) + 255) / 256), (unsigned)(B * C)); }

__global__ void k_avgpool(const float *__restrict__ in, long in_bs, float *__restrict__ out, long out_bs,
                          int C, int H, int W, int B) {
  int b, c, y, x, q;
  if (!coarse_pixel(H, W, C, b, c, y, x, q)) return;
  const float *p = in + b * in_bs + (long)c * H * W + (long)(2 * y) * W + 2 * x;
  const float2 r0 = *reinterpret_cast<const float2 *>(p), r1 = *reinterpret_cast<const float2 *>(p + W);
  out[b * out_bs + (long)c * (H / 2) * (W / 2) + q] = 0.25f * (r0.x + r0.y + r1.x + r1.y);
}

// grad of avgpool: g_in (+)= g_out / 4 on each 2x2 block
__global__ void k_avgpool_bwd(const float *__restrict__ go, long go_bs, float *__restrict__ gi, long gi_bs,
                              int C, int H, int W, int B, int accumulate) {
  int b, c, y, x, q;
  if (!coarse_pixel(H, W, C, b, c, y, x, q)) return;
  const float v = 0.25f * go[b * go_bs + (long)c * (H / 2) * (W / 2) + q];
  float2 *d0 = reinterpret_cast<float2 *>(gi + b * gi_bs + (long)c * H * W + (long)(2 * y) * W + 2 * x);
  float2 *d1 = reinterpret_cast<float2 *>(reinterpret_cast<float *>(d0) + W);
  if (accumulate) {
    const float2 a0 = *d0, a1 = *d1;
    *d0 = make_float2(a0.x + v, a0.y + v);
    *d1 = make_float2(a1.x + v, a1.y + v);
  } else {
    *d0 = make_float2(v, v);
    *d1 = make_float2(v, v);
  }
}

__global__ void k_upsample(const float *__restrict__ in, long in_bs, float *__restrict__ out, long out_bs,
                           int C, int H, int W, int B) {  // H, W: output size
  int b, c, y, x, q;
  if (!coarse_pixel(H, W, C, b, c, y, x, q)) return;
  const float v = in[b * in_bs + (long)c * (H / 2) * (W / 2) + q];
  float *o = out + b * out_bs + (long)c * H * W + (long)(2 * y) * W + 2 * x;
  *reinterpret_cast<float2 *>(o) = make_float2(v, v);
  *reinterpret_cast<float2 *>(o + W) = make_float2(v, v);
}

__global__ void k_upsample_bwd(const float *__restrict__ go, long go_bs, float *__restrict__ gi, long gi_bs,
                               int C, int H, int W, int B) {  // H, W: upsampled size
  int b, c, y, x, q;
  if (!coarse_pixel(H, W, C, b, c, y, x, q)) return;
  const float *p = go + b * go_bs + (long)c * H * W + (long)(2 * y) * W + 2 * x;
  const float2 r0 = *reinterpret_cast<const float2 *>(p), r1 = *reinterpret_cast<const float2 *>(p + W);
  gi[b * gi_bs + (long)c * (H / 2) * (W / 2) + q] = r0.x + r0.y + r1.x + r1.y;
}

// The decoder's upsampled half straight into its BF16 NHWC concatenation:
// coarse FP32 planes (image stride in_bs) -> channels 0 .. C (C a multiple of
// 8) of the 4 fine pixels of each coarse pixel, pixels o_cp channels apart.
// One thread per (image, coarse pixel, group of 8 channels), the groups
// fastest, so a warp's stores cover whole 16-byte runs of each fine pixel.
// H, W: the fine size.
__global__ void k_upsample_nhwc(const float *__restrict__ in, long in_bs, int C, int H, int W, int B,
                                __nv_bfloat16 *__restrict__ out, long o_bs, int o_cp) {
  const int Wc = W / 2, G8 = C / 8;
  const long per = (long)(H / 2) * Wc;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < (long)B * per * G8;
       t += (long)gridDim.x * blockDim.x) {
    const long pq = t / G8;
    const int g8 = (int)(t - pq * G8);
    const long b = pq / per;
    const int q = (int)(pq - b * per), y = q / Wc, x = q - y * Wc;
    const float *src = in + b * in_bs + (long)(8 * g8) * per + q;
    unsigned w4[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const __nv_bfloat162 q2 = __floats2bfloat162_rn(src[(long)(2 * e) * per], src[(long)(2 * e + 1) * per]);
      w4[e] = *reinterpret_cast<const unsigned *>(&q2);
    }
    const uint4 v = make_uint4(w4[0], w4[1], w4[2], w4[3]);
    __nv_bfloat16 *o = out + b * o_bs + ((long)(2 * y) * W + 2 * x) * o_cp + 8 * g8;
    *reinterpret_cast<uint4 *>(o) = v;
    *reinterpret_cast<uint4 *>(o + o_cp) = v;
    *reinterpret_cast<uint4 *>(o + (long)W * o_cp) = v;
    *reinterpret_cast<uint4 *>(o + (long)(W + 1) * o_cp) = v;
  }
}

// g *= (a > 0): relu backward through a stored activation
__global__ void k_relu_mask(float *__restrict__ g, long g_bs, const float *__restrict__ a, long a_bs,
                            long per, int B) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < (long)B * per; i += (long)gridDim.x * blockDim.x) {
    const long b = i / per, r = i % per;
    if (!(a[b * a_bs + r] > 0.f)) g[b * g_bs + r] = 0.f;
  }
}

// loss = mean(w_b (o - t)^2) (block partials in double), go = 2 w_b (o - t) / n;
// w_b = sample weight of image b (1 without weights), plane pixels per image
__global__ void k_mse(const float *__restrict__ o, const float *__restrict__ t, long n, long plane,
                      const float *__restrict__ wts, float *__restrict__ go, double *__restrict__ part) {
  __shared__ double red[256];
  double s = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float d = o[i] - t[i];
    const float wb = wts ? wts[i / plane] : 1.f;
    s += (double)wb * d * d;
    go[i] = 2.f * wb * d / (float)n;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, __nv_bfloat16 *__restrict__ pb, long n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    pb[i] = __float2bfloat16_rn(pi);
  }
}

__global__ void k_to_bf16(const float *__restrict__ p, __nv_bfloat16 *__restrict__ pb, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    pb[i] = __float2bfloat16_rn(p[i]);
}

// Preconditioner input [1][3][n][n]: (sigma_t / s_ref, sigma_s / s_ref, v / rms(v))
__global__ void k_net_input(const double *__restrict__ st, const double *__restrict__ ss,
                            const double *__restrict__ v, const double *__restrict__ vnorm2, long N,
                            float inv_ref, float *__restrict__ x) {
  const double rms = sqrt(*vnorm2 / (double)N);
  const double inv = rms > 0.0 ? 1.0 / rms : 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    x[i] = (float)st[i] * inv_ref;
    x[N + i] = (float)ss[i] * inv_ref;
    x[2 * N + i] = (float)(v[i] * inv);
  }
}

// z = base + rms(v) o (base: v itself, or another preconditioner's z_0 = M_0 v)
__global__ void k_net_output(const double *__restrict__ base, const double *__restrict__ vnorm2,
                             const float *__restrict__ o, long N, double *__restrict__ z) {
  const double rms = sqrt(*vnorm2 / (double)N);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x)
    z[i] = base[i] + rms * (double)o[i];
}

int gridn(long n) { return (int)std::max(1L, std::min((n + 255) / 256, 8192L)); }

// The same for R vectors at once (blockIdx.y = r): v_r at v + r ldv, ||v_r||^2
// at scal[8 r + slot], input image r at x + 3 r N, z_r at z + r ldz.
__global__ void k_net_input_b(const double *__restrict__ st, const double *__restrict__ ss,
                              const double *__restrict__ v, long ldv, const double *__restrict__ scal, int slot,
                              long N, float inv_ref, float *__restrict__ x) {
  const int r = blockIdx.y;
  const double rms = sqrt(scal[8 * r + slot] / (double)N);
  const double inv = rms > 0.0 ? 1.0 / rms : 0.0;
  const double *vr = v + (long)r * ldv;
  float *xr = x + 3L * r * N;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    xr[i] = (float)st[i] * inv_ref;
    xr[N + i] = (float)ss[i] * inv_ref;
    xr[2 * N + i] = (float)(vr[i] * inv);
  }
}

__global__ void k_net_output_b(const double *__restrict__ base, long ldb, const double *__restrict__ scal, int slot,
                               const float *__restrict__ o, long N, double *__restrict__ z, long ldz) {
  const int r = blockIdx.y;
  const double rms = sqrt(scal[8 * r + slot] / (double)N);
  const double *br = base + (long)r * ldb;
  const float *orr = o + (long)r * N;
  double *zr = z + (long)r * ldz;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x)
    zr[i] = br[i] + rms * (double)orr[i];
}

}  // namespace

// ------------------------------------------------------------ network host

struct ConvLayer {
  int co, ci, k;
  long w_off, b_off;  // into the flat parameter array
  long tc_off;        // 3x3 layers: their packed BF16 weights [9 S][co][32] in UnetImpl::ptc
};

// A cached TMA descriptor (encoding one costs host time on every launch).
struct MapEntry {
  const void *base;
  unsigned long long key[4];
  CUtensorMap map;
};

struct UnetImpl {
  int L = 4, C = 32, device = 0;
  std::vector<ConvLayer> layers;
  long nparams = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr, *wt = nullptr;
  __nv_bfloat16 *pb = nullptr;
  long step = 0;
  // activations for (B, n)
  int B = 0, n = 0;
  std::vector<float *> xin, a, cat, bl, dl, ebot;  // per level
  std::vector<float *> gx, ga, gcat, gbl, gdl, gebot;
  float *o = nullptr, *go = nullptr;
  double *part = nullptr, *h_part = nullptr;
  float *xin0_owned = nullptr;
  int *dev_err = nullptr;  // set by a tensor-core convolution whose bounded wait gave up
  // BF16 tensor-core forward: packed weights (rebuilt when the parameters
  // change), the NHWC BF16 copy of the current convolution's input, cached maps
  __nv_bfloat16 *ptc = nullptr;
  long ptc_elems = 0;
  bool ptc_dirty = true;
  __nv_bfloat16 *nhwc = nullptr;
  // BF16 NHWC inputs written by the convolutions themselves: hx, a level's
  // second convolution's input (C channels padded to slices); hcat[l], the
  // decoder's concatenation at level l (the upsampled half, then the skip)
  __nv_bfloat16 *hx = nullptr;
  std::vector<__nv_bfloat16 *> hcat;
  // the input-gradient convolutions of training on the tensor cores (split
  // precision): the lo half of the converted input, the split weights of
  // one 32-channel output block
  int train_tc = 0;  // operand parts of the training convolutions on the tensor cores (0: CUDA cores)
  __nv_bfloat16 *nhwc_lo = nullptr, *nhwc_p2 = nullptr, *wsp_hi = nullptr, *wsp_lo = nullptr, *wsp_p2 = nullptr;
  std::vector<MapEntry> maps;
};

namespace {

void free_acts(UnetImpl *u) {
  auto fr = [](std::vector<float *> &vv) {
    for (float *&q : vv)
      if (q) vie_free(q);
    vv.clear();
  };
  fr(u->xin); fr(u->a); fr(u->cat); fr(u->bl); fr(u->dl); fr(u->ebot);
  fr(u->gx); fr(u->ga); fr(u->gcat); fr(u->gbl); fr(u->gdl); fr(u->gebot);
  if (u->o) vie_free(u->o);
  if (u->go) vie_free(u->go);
  if (u->part) vie_free(u->part);
  if (u->h_part) vie_free_host(u->h_part);
  if (u->nhwc) vie_free(u->nhwc);
  u->nhwc = nullptr;
  if (u->hx) vie_free(u->hx);
  u->hx = nullptr;
  for (__nv_bfloat16 **q : {&u->nhwc_lo, &u->nhwc_p2, &u->wsp_hi, &u->wsp_lo, &u->wsp_p2}) {
    if (*q) vie_free(*q);
    *q = nullptr;
  }
  for (__nv_bfloat16 *q : u->hcat)
    if (q) vie_free(q);
  u->hcat.clear();
  u->maps.clear();
  u->o = u->go = nullptr;
  u->part = nullptr;
  u->h_part = nullptr;
  u->B = u->n = 0;
}

vie_status ensure_acts(UnetImpl *u, int B, int n) {
  if (u->B >= B && u->n == n) return VIE_OK;
  free_acts(u);
  const int L = u->L, C = u->C;
  auto al = [](float **q, long count) -> vie_status {
    VIE_CUDA(vie_malloc((void **)q, sizeof(float) * std::max(1L, count)));
    return VIE_OK;
  };
  u->xin.assign(L, nullptr); u->a.assign(L, nullptr); u->cat.assign(L, nullptr);
  u->bl.assign(L, nullptr); u->dl.assign(L, nullptr); u->ebot.assign(1, nullptr);
  u->gx.assign(L, nullptr); u->ga.assign(L, nullptr); u->gcat.assign(L, nullptr);
  u->gbl.assign(L, nullptr); u->gdl.assign(L, nullptr); u->gebot.assign(1, nullptr);
  vie_status s;
  for (int l = 0; l < L; ++l) {
    const long hw = (long)(n >> l) * (n >> l);
    const int cin = l == 0 ? 3 : C;
    if ((s = al(&u->xin[l], (long)B * cin * hw)) != VIE_OK) return s;
    if ((s = al(&u->a[l], (long)B * C * hw)) != VIE_OK) return s;
    if ((s = al(&u->gx[l], (long)B * cin * hw)) != VIE_OK) return s;
    if ((s = al(&u->ga[l], (long)B * C * hw)) != VIE_OK) return s;
    if (l < L - 1) {
      if ((s = al(&u->cat[l], (long)B * 2 * C * hw)) != VIE_OK) return s;
      if ((s = al(&u->bl[l], (long)B * C * hw)) != VIE_OK) return s;
      if ((s = al(&u->dl[l], (long)B * C * hw)) != VIE_OK) return s;
      if ((s = al(&u->gcat[l], (long)B * 2 * C * hw)) != VIE_OK) return s;
      if ((s = al(&u->gbl[l], (long)B * C * hw)) != VIE_OK) return s;
      if ((s = al(&u->gdl[l], (long)B * C * hw)) != VIE_OK) return s;
    }
  }
  const long hwb = (long)(n >> (L - 1)) * (n >> (L - 1));
  if ((s = al(&u->ebot[0], (long)B * C * hwb)) != VIE_OK) return s;
  if ((s = al(&u->gebot[0], (long)B * C * hwb)) != VIE_OK) return s;
  if ((s = al(&u->o, (long)B * n * n)) != VIE_OK) return s;
  if ((s = al(&u->go, (long)B * n * n)) != VIE_OK) return s;
  VIE_CUDA(vie_malloc((void **)&u->part, sizeof(double) * 1024));
  VIE_CUDA(vie_malloc_host((void **)&u->h_part, sizeof(double) * 1024));
  // the widest convolution input: 2 C channels (a decoder's concatenation), padded to slices
  VIE_CUDA(vie_malloc((void **)&u->nhwc,
                      sizeof(__nv_bfloat16) * (size_t)B * n * n * (size_t)(((2 * C + 31) / 32) * 32)));
  VIE_CUDA(vie_malloc((void **)&u->nhwc_lo,
                      sizeof(__nv_bfloat16) * (size_t)B * n * n * (size_t)(((2 * C + 31) / 32) * 32)));
  VIE_CUDA(vie_malloc((void **)&u->nhwc_p2,
                      sizeof(__nv_bfloat16) * (size_t)B * n * n * (size_t)(((2 * C + 31) / 32) * 32)));
  {
    const size_t wsp = (size_t)9 * ((2 * C + 31) / 32) * 32 * 32;  // 9 S blocks of [32][32]
    VIE_CUDA(vie_malloc((void **)&u->wsp_hi, sizeof(__nv_bfloat16) * wsp));
    VIE_CUDA(vie_malloc((void **)&u->wsp_lo, sizeof(__nv_bfloat16) * wsp));
    VIE_CUDA(vie_malloc((void **)&u->wsp_p2, sizeof(__nv_bfloat16) * wsp));
  }
  // the hand-off buffers, zeroed once: their padding channels are never written
  const size_t cp1 = (size_t)((C + 31) / 32) * 32, cp2 = (size_t)((2 * C + 31) / 32) * 32;
  VIE_CUDA(vie_malloc((void **)&u->hx, sizeof(__nv_bfloat16) * (size_t)B * n * n * cp1));
  VIE_CUDA(cudaMemset(u->hx, 0, sizeof(__nv_bfloat16) * (size_t)B * n * n * cp1));
  u->hcat.assign(L, nullptr);
  for (int l = 0; l < L - 1; ++l) {
    const size_t bytes = sizeof(__nv_bfloat16) * (size_t)B * (n >> l) * (n >> l) * cp2;
    VIE_CUDA(vie_malloc((void **)&u->hcat[l], bytes));
    VIE_CUDA(cudaMemset(u->hcat[l], 0, bytes));
  }
  u->B = B;
  u->n = n;
  return VIE_OK;
}

template <bool RELU, typename WT, int TY, int COBC>
void launch_conv3(const float *in, long in_bs, int Ci, const WT *w, const float *bias, float *out, long out_bs,
                  int Co, int H, int W, int B, cudaStream_t st) {
  const int cob = (Co + COBC - 1) / COBC;
  dim3 grid((W + TX - 1) / TX, (H + TY - 1) / TY, B * cob);
  k_conv3<RELU, WT, TY, COBC><<<grid, 256, 0, st>>>(in, in_bs, Ci, w, bias, out, out_bs, Co, H, W, cob);
}

// Tile shapes by decreasing work per thread: (TY, COBC) = (16, 32), (16, 16),
// (8, 16), (8, 8).  The first whose grid covers two CTAs per SM is taken, the
// smallest otherwise: the coarse U-Net levels have too few pixels to fill the
// GPU with 64 outputs per thread.
template <bool RELU, typename WT>
void conv3_shape(const float *in, long in_bs, int Ci, const WT *w, const float *bias, float *out, long out_bs,
                 int Co, int H, int W, int B, cudaStream_t st) {
  const long tx = (W + TX - 1) / TX;
  auto ctas = [&](int ty, int cobc) { return tx * ((H + ty - 1) / ty) * B * ((Co + cobc - 1) / cobc); };
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long want = 2L * (sms > 0 ? sms : 1);
  if (ctas(16, 32) >= want)
    launch_conv3<RELU, WT, 16, 32>(in, in_bs, Ci, w, bias, out, out_bs, Co, H, W, B, st);
  else if (ctas(16, 16) >= want)
    launch_conv3<RELU, WT, 16, 16>(in, in_bs, Ci, w, bias, out, out_bs, Co, H, W, B, st);
  else if (ctas(8, 16) >= want)
    launch_conv3<RELU, WT, 8, 16>(in, in_bs, Ci, w, bias, out, out_bs, Co, H, W, B, st);
  else
    launch_conv3<RELU, WT, 8, 8>(in, in_bs, Ci, w, bias, out, out_bs, Co, H, W, B, st);
}

// the tensor map for (base, key), encoded on first use and copied out by
// value (the cache may grow, and move its entries, on a later call)
vie_status cached_map(UnetImpl *u, const void *base, const unsigned long long (&key)[4], int rank,
                      const unsigned long long *dims, const unsigned long long *strides, const unsigned *box,
                      CUtensorMap *out) {
  for (const MapEntry &e : u->maps)
    if (e.base == base && e.key[0] == key[0] && e.key[1] == key[1] && e.key[2] == key[2] && e.key[3] == key[3]) {
      *out = e.map;
      return VIE_OK;
    }
  MapEntry e{base, {key[0], key[1], key[2], key[3]}, CUtensorMap{}};
  VIE_TRY(encode_bf16_map(&e.map, rank, base, dims, strides, box, 64));
  if (u->maps.size() >= 256) u->maps.clear();
  u->maps.push_back(e);
  *out = e.map;
  return VIE_OK;
}

// the BF16 convolutions the tensor-core kernel takes
bool conv_on_tensor_cores(const void *wtc, int Ci, int Co, const float *bias) {
  return wtc && Co % 16 == 0 && Co >= 16 && Co <= 32 && Ci <= 2 * kTmaSlice && bias;
}

// The BF16 3x3 convolution on the tensor cores (k_conv3_tma): input to BF16
// NHWC, then the implicit GEMM.  wtc: the layer's packed weights.
// Fused NHWC hand-off between convolutions (all optional): in_h, the input
// already in BF16 NHWC with S 32-channel slices (else `in` is converted);
// out_h, a second output in BF16 NHWC at channel oh_c0 of pixels oh_cp
// channels apart (image stride oh_bs elements).
struct NhwcIo {
  const __nv_bfloat16 *in_h = nullptr;
  __nv_bfloat16 *out_h = nullptr;
  long oh_bs = 0;
  int oh_cp = 0, oh_c0 = 0;
  bool wrote = false;  // set when out_h was written
};

// the input's tensor map: NHWC BF16 at src, S slices; tiles of one row load
// halo boxes of Wb + 2 pixels (the kernel's halo mode)
vie_status conv_input_map(UnetImpl *u, const __nv_bfloat16 *src, int S, int H, int W, int B, CUtensorMap *mx) {
  const int Cp = S * kTmaSlice, Wb = std::min(W, kTcM), R = std::min(kTcM / Wb, H);
  const unsigned bw = R == 1 ? (unsigned)Wb + 2 : (unsigned)Wb;
  const unsigned long long key[4] = {(unsigned long long)Cp | ((unsigned long long)bw << 32), (unsigned long long)W,
                                     (unsigned long long)H, (unsigned long long)B};
  const unsigned long long dims[4] = {(unsigned long long)Cp, (unsigned long long)W, (unsigned long long)H,
                                      (unsigned long long)B};
  const unsigned long long strides[3] = {2ull * Cp, 2ull * Cp * W, 2ull * Cp * W * H};
  const unsigned box[4] = {(unsigned)kTmaSlice, bw, (unsigned)R, 1u};
  return cached_map(u, src, key, 4, dims, strides, box, mx);
}

// packed weights [9 S][Co][32] at wtc
vie_status conv_weight_map(UnetImpl *u, const __nv_bfloat16 *wtc, int S, int Co, CUtensorMap *mw) {
  const unsigned long long key[4] = {(unsigned long long)S, (unsigned long long)Co, 0ull, 1ull};
  const unsigned long long dims[2] = {(unsigned long long)kTmaSlice, 9ull * S * Co};
  const unsigned long long strides[1] = {2ull * kTmaSlice};
  const unsigned box[2] = {(unsigned)kTmaSlice, (unsigned)Co};
  return cached_map(u, wtc, key, 2, dims, strides, box, mw);
}

// Launch k_conv3_tma with np operand parts (maps mx[p], mw[p]; np > 1: the
// split-precision form).
vie_status launch_conv_tma(UnetImpl *u, const CUtensorMap *mx, const CUtensorMap *mw, int np, const float *bias,
                           float *out, long out_bs, int Co, int H, int W, int S, int B, bool relu, cudaStream_t st,
                           NhwcIo *io) {
  const int Wb = std::min(W, kTcM), R = std::min(kTcM / Wb, H);
  const int tiles_x = (W + Wb - 1) / Wb, tiles_y = (H + R - 1) / R;
  int dev = 0;
  VIE_CUDA(cudaGetDevice(&dev));
  DevProps prop;
  VIE_TRY(get_dev_props(dev, &prop));
  // two CTAs per SM (two epilogues and issuers in flight), each with half of
  // the SM's shared memory less the per-CTA reserve, where three stages fit;
  // else one with all of it.  Measured with 64 images at 128^2: one CTA per
  // SM 1.69 ms per forward, two 1.25, three 1.42, four 1.45.  (The occupancy
  // query reports one CTA per SM for this kernel at any shared-memory size;
  // two run side by side all the same, and a grid they could not share would
  // only run in two waves, each CTA taking every G-th tile.)
  const size_t optin = (size_t)prop.sharedMemPerBlockOptin;
  int per_sm = 2, nst = conv_stages(S, Co, Wb, (optin + 1024) / 2 - 1024, np);
  if (nst < 3) {
    per_sm = 1;
    nst = conv_stages(S, Co, Wb, optin, np);
  }
  if (nst < 2) {
    set_error("BF16 convolution: not enough shared memory for two stages");
    return VIE_ERR_UNSUPPORTED;
  }
  const size_t smem = conv_tma_smem(S, Co, Wb, nst, np);
  const void *k = np == 3   ? (relu ? (const void *)k_conv3_tma<true, 3> : (const void *)k_conv3_tma<false, 3>)
                  : np == 2 ? (relu ? (const void *)k_conv3_tma<true, 2> : (const void *)k_conv3_tma<false, 2>)
                            : (relu ? (const void *)k_conv3_tma<true, 1> : (const void *)k_conv3_tma<false, 1>);
  VIE_TRY(raise_smem_limit(k, smem));
  // all of the SM's unified memory as shared memory, so that two CTAs fit
  VIE_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  WaitLimits wl = wait_limits(dev);
  // per_sm CTAs per SM, each taking every G-th tile
  int tiles = tiles_x * tiles_y * B;
  const int grid = std::min(tiles, per_sm * prop.multiProcessorCount);
  __nv_bfloat16 *oh = io ? io->out_h : nullptr;
  long oh_bs = io ? io->oh_bs : 0;
  int oh_cp = io ? io->oh_cp : 0, oh_c0 = io ? io->oh_c0 : 0;
  int nst_i = nst, S_i = S, Co_i = Co, H_i = H, W_i = W, Wb_i = Wb, R_i = R, tx_i = tiles_x;
  int *err = u->dev_err;
  // maps of the parts past np: copies of part 0 (not read)
  const CUtensorMap *x1 = np > 1 ? mx + 1 : mx, *w1 = np > 1 ? mw + 1 : mw;
  const CUtensorMap *x2 = np > 2 ? mx + 2 : mx, *w2 = np > 2 ? mw + 2 : mw;
  void *args[] = {(void *)mx, (void *)mw, (void *)x1, (void *)w1, (void *)x2, (void *)w2, (void *)&bias, (void *)&out,
                  (void *)&out_bs, (void *)&Co_i, (void *)&H_i, (void *)&W_i, (void *)&S_i, (void *)&Wb_i,
                  (void *)&R_i, (void *)&tx_i, (void *)&tiles, (void *)&nst_i, (void *)&wl, (void *)&err,
                  (void *)&oh, (void *)&oh_bs, (void *)&oh_cp, (void *)&oh_c0};
  VIE_CUDA(cudaLaunchKernel(k, dim3((unsigned)grid), dim3(kConvThreads), args, smem, st));
  if (io) io->wrote = oh != nullptr;
  VIE_CHECK_LAUNCH("k_conv3_tma");
  return VIE_OK;
}

vie_status conv3_tma(UnetImpl *u, const float *in, long in_bs, int Ci, const __nv_bfloat16 *wtc, const float *bias,
                     float *out, long out_bs, int Co, int H, int W, int B, bool relu, cudaStream_t st, NhwcIo *io) {
  const int S = (Ci + kTmaSlice - 1) / kTmaSlice, Cp = S * kTmaSlice;
  const long plane = (long)H * W;
  const __nv_bfloat16 *src = io && io->in_h ? io->in_h : u->nhwc;
  if (src == u->nhwc) {
    k_to_nhwc_bf16<<<gridn((long)B * plane), 256, 0, st>>>(in, in_bs, Ci, plane, Cp, B, u->nhwc);
    VIE_CHECK_LAUNCH("k_to_nhwc_bf16");
  }
  CUtensorMap mx, mw;
  VIE_TRY(conv_input_map(u, src, S, H, W, B, &mx));
  VIE_TRY(conv_weight_map(u, wtc, S, Co, &mw));
  return launch_conv_tma(u, &mx, &mw, 1, bias, out, out_bs, Co, H, W, S, B, relu, st, io);
}

// The FP32 convolution of training on the tensor cores in split precision:
// the input split into np BF16 NHWC parts, the FP32 weights [Co][Ci][9] split
// and packed per block of 32 output channels, one launch per block.
bool conv_split_ok(int Ci, int Co) { return Ci <= 2 * kTmaSlice && Co % 32 == 0 && Co <= 64; }

vie_status conv3_split(UnetImpl *u, const float *in, long in_bs, int Ci, const float *w, const float *bias,
                       float *out, long out_bs, int Co, int H, int W, int B, bool relu, int np, cudaStream_t st) {
  const int S = (Ci + kTmaSlice - 1) / kTmaSlice, Cp = S * kTmaSlice;
  const long plane = (long)H * W;
  __nv_bfloat16 *xin[3] = {u->nhwc, u->nhwc_lo, u->nhwc_p2}, *wsp[3] = {u->wsp_hi, u->wsp_lo, u->wsp_p2};
  if (np == 3)
    k_to_nhwc_split<3><<<gridn((long)B * plane), 256, 0, st>>>(in, in_bs, Ci, plane, Cp, B, xin[0], xin[1], xin[2]);
  else
    k_to_nhwc_split<2><<<gridn((long)B * plane), 256, 0, st>>>(in, in_bs, Ci, plane, Cp, B, xin[0], xin[1], xin[2]);
  VIE_CHECK_LAUNCH("k_to_nhwc_split");
  CUtensorMap mx[3], mw[3];
  for (int q = 0; q < np; ++q) {
    VIE_TRY(conv_input_map(u, xin[q], S, H, W, B, &mx[q]));
    VIE_TRY(conv_weight_map(u, wsp[q], S, 32, &mw[q]));
  }
  for (int co0 = 0; co0 < Co; co0 += 32) {
    k_pack_split_weights<<<gridn(9L * S * 32 * kTmaSlice), 256, 0, st>>>(w, Co, Ci, S, co0, 32, np, wsp[0], wsp[1],
                                                                         wsp[2]);
    VIE_CHECK_LAUNCH("k_pack_split_weights");
    VIE_TRY(launch_conv_tma(u, mx, mw, np, bias ? bias + co0 : nullptr, out + co0 * plane, out_bs, 32, H, W, S, B,
                            relu, st, nullptr));
  }
  return VIE_OK;
}

// io (tensor-core path only; ignored, with io->wrote false, on the CUDA cores)
template <typename WT>
vie_status conv3(UnetImpl *u, const float *in, long in_bs, int Ci, const WT *w, const __nv_bfloat16 *wtc,
                 const float *bias, float *out, long out_bs, int Co, int H, int W, int B, bool relu,
                 cudaStream_t st, NhwcIo *io = nullptr) {
  if (io) io->wrote = false;
  if constexpr (std::is_same<WT, __nv_bfloat16>::value) {
    if (conv_on_tensor_cores(wtc, Ci, Co, bias))
      return conv3_tma(u, in, in_bs, Ci, wtc, bias, out, out_bs, Co, H, W, B, relu, st, io);
  } else {
    if (u->train_tc > 1 && conv_split_ok(Ci, Co))
      return conv3_split(u, in, in_bs, Ci, w, bias, out, out_bs, Co, H, W, B, relu, u->train_tc, st);
  }
  if (relu)
    conv3_shape<true, WT>(in, in_bs, Ci, w, bias, out, out_bs, Co, H, W, B, st);
  else
    conv3_shape<false, WT>(in, in_bs, Ci, w, bias, out, out_bs, Co, H, W, B, st);
  VIE_CHECK_LAUNCH("k_conv3");
  return VIE_OK;
}

// Forward through the network; weights FP32 (pw) or BF16 (pbw).
// the packed BF16 weights of every 3x3 layer, from the FP32 parameters
vie_status pack_tc_weights(UnetImpl *u, cudaStream_t st) {
  if (!u->ptc_dirty) return VIE_OK;
  for (const ConvLayer &c : u->layers) {
    if (c.k != 3) continue;
    const int S = (c.ci + kTmaSlice - 1) / kTmaSlice;
    k_pack_tc_weights<<<gridn(9L * S * c.co * kTmaSlice), 256, 0, st>>>(u->p + c.w_off, c.co, c.ci, S,
                                                                       u->ptc + c.tc_off);
    VIE_CHECK_LAUNCH("k_pack_tc_weights");
  }
  u->ptc_dirty = false;
  return VIE_OK;
}

template <typename WT>
vie_status forward(UnetImpl *u, const WT *pw, const float *x, int B, int n, cudaStream_t st) {
  const int L = u->L, C = u->C;
  vie_status s;
  int li = 0;
  const bool tc = std::is_same<WT, __nv_bfloat16>::value;
  if (tc && (s = pack_tc_weights(u, st)) != VIE_OK) return s;
  auto wtc = [&](const ConvLayer &c) { return tc ? u->ptc + c.tc_off : nullptr; };
  const float *xl = x;
  long xl_bs = 3L * n * n;
  // BF16 NHWC hand-off (tensor-core path): each convolution also writes the
  // next one's input, and the encoder's second convolution its skip into the
  // decoder's concatenation
  const int cp1 = ((C + 31) / 32) * 32, cp2 = ((2 * C + 31) / 32) * 32;
  const bool handoff = tc && C % 8 == 0;
  std::vector<char> skip_h(L, 0);
  for (int l = 0; l < L; ++l) {
    const int H = n >> l;
    const long hw = (long)H * H;
    const ConvLayer &c1 = u->layers[li++], &c2 = u->layers[li++];
    NhwcIo io1;
    if (handoff) {
      io1.out_h = u->hx;
      io1.oh_bs = hw * cp1;
      io1.oh_cp = cp1;
    }
    if ((s = conv3(u, xl, xl_bs, c1.ci, pw + c1.w_off, wtc(c1), u->p + c1.b_off, u->a[l], (long)C * hw, C, H,
                   H, B, true, st, &io1)) != VIE_OK)
      return s;
    float *e = l < L - 1 ? u->cat[l] + (long)C * hw : u->ebot[0];
    const long e_bs = l < L - 1 ? 2L * C * hw : (long)C * hw;
    NhwcIo io2;
    io2.in_h = io1.wrote ? u->hx : nullptr;
    if (handoff && l < L - 1) {
      io2.out_h = u->hcat[l];
      io2.oh_bs = hw * cp2;
      io2.oh_cp = cp2;
      io2.oh_c0 = C;
    }
    if ((s = conv3(u, u->a[l], (long)C * hw, C, pw + c2.w_off, wtc(c2), u->p + c2.b_off, e, e_bs, C, H, H, B,
                   true, st, &io2)) != VIE_OK)
      return s;
    skip_h[l] = io2.wrote;
    if (l < L - 1) {
      k_avgpool<<<coarse_grid(H, H, C, B), 256, 0, st>>>(e, e_bs, u->xin[l + 1], (long)C * hw / 4, C, H,
                                                             H, B);
      VIE_CHECK_LAUNCH("k_avgpool");
      xl = u->xin[l + 1];
      xl_bs = (long)C * hw / 4;
    }
  }
  const float *d = u->ebot[0];
  long d_bs = (long)C * (n >> (L - 1)) * (n >> (L - 1));
  for (int l = L - 2; l >= 0; --l) {
    const int H = n >> l;
    const long hw = (long)H * H;
    const ConvLayer &c1 = u->layers[li++], &c2 = u->layers[li++];
    NhwcIo io1, io2;
    if (skip_h[l] && conv_on_tensor_cores(wtc(c1), c1.ci, c1.co, u->p + c1.b_off)) {
      // the upsampled half in BF16 beside the skip the encoder wrote; the FP32
      // concatenation's first half is not written (vie_unet_layer_io rebuilds it)
      const long per = hw / 4;
      k_upsample_nhwc<<<gridn((long)B * per * (C / 8)), 256, 0, st>>>(d, d_bs, C, H, H, B, u->hcat[l], hw * cp2,
                                                                      cp2);
      VIE_CHECK_LAUNCH("k_upsample_nhwc");
      io1.in_h = u->hcat[l];
    } else {
      k_upsample<<<coarse_grid(H, H, C, B), 256, 0, st>>>(d, d_bs, u->cat[l], 2L * C * hw, C, H, H, B);
      VIE_CHECK_LAUNCH("k_upsample");
    }
    if (handoff) {
      io1.out_h = u->hx;
      io1.oh_bs = hw * cp1;
      io1.oh_cp = cp1;
    }
    if ((s = conv3(u, u->cat[l], 2L * C * hw, 2 * C, pw + c1.w_off, wtc(c1), u->p + c1.b_off, u->bl[l],
                   (long)C * hw, C, H, H, B, true, st, &io1)) != VIE_OK)
      return s;
    io2.in_h = io1.wrote ? u->hx : nullptr;
    if ((s = conv3(u, u->bl[l], (long)C * hw, C, pw + c2.w_off, wtc(c2), u->p + c2.b_off, u->dl[l],
                   (long)C * hw, C, H, H, B, true, st, &io2)) != VIE_OK)
      return s;
    d = u->dl[l];
    d_bs = (long)C * hw;
  }
  const ConvLayer &hd = u->layers[li];
  k_head<WT><<<gridn((long)B * n * n), 256, 0, st>>>(d, d_bs, C, pw + hd.w_off, u->p + hd.b_off, u->o,
                                                     (long)n * n, B);
  VIE_CHECK_LAUNCH("k_head");
  return VIE_OK;
}

// dw/db of a 3x3 convolution and, if gin, the input gradient (adjoint conv).
vie_status conv3_backward(UnetImpl *u, const ConvLayer &c, const float *in, long in_bs, const float *gout,
                          long g_bs, float *gin, long gin_bs, int H, int B, cudaStream_t st) {
  const int cib = (c.ci + CIB - 1) / CIB, cob = (c.co + COB - 1) / COB;
  // images per CTA: about four CTAs per SM in all, each adding its sums once
  const long per_split = (long)((H + TX - 1) / TX) * ((H + WY - 1) / WY) * cob * cib;
  int sms = 0, dev = 0;
  VIE_CUDA(cudaGetDevice(&dev));
  DevProps prop;
  VIE_TRY(get_dev_props(dev, &prop));
  sms = prop.multiProcessorCount;
  const int splits = (int)std::max(1L, std::min<long>(B, (4L * sms + per_split - 1) / per_split));
  dim3 grid((H + TX - 1) / TX, (H + WY - 1) / WY, splits * cob * cib);
  k_conv3_dw<<<grid, 256, 0, st>>>(in, in_bs, c.ci, gout, g_bs, c.co, H, H, u->g + c.w_off, u->g + c.b_off,
                                  cib, cob, B, splits);
  VIE_CHECK_LAUNCH("k_conv3_dw");
  if (gin) {
    k_flip<<<gridn((long)c.co * c.ci * 9), 256, 0, st>>>(u->p + c.w_off, c.co, c.ci, u->wt);
    VIE_CHECK_LAUNCH("k_flip");
    vie_status s = conv3<float>(u, gout, g_bs, c.co, u->wt, nullptr, nullptr, gin, gin_bs, c.ci, H, H, B, false,
                                st);
    if (s != VIE_OK) return s;
  }
  return VIE_OK;
}

vie_status relu_mask(float *g, long g_bs, const float *a, long a_bs, long per, int B, cudaStream_t st) {
  k_relu_mask<<<gridn((long)B * per), 256, 0, st>>>(g, g_bs, a, a_bs, per, B);
  VIE_CHECK_LAUNCH("k_relu_mask");
  return VIE_OK;
}

// Backward pass from go (d loss / d o); gradients accumulate into u->g.
vie_status backward(UnetImpl *u, const float *x, int B, int n, cudaStream_t st) {
  const int L = u->L, C = u->C;
  vie_status s;
  int li = (int)u->layers.size() - 1;
  const ConvLayer &hd = u->layers[li];
  const float *d = L > 1 ? u->dl[0] : u->ebot[0];
  float *gd = L > 1 ? u->gdl[0] : u->gebot[0];
  const long plane0 = (long)n * n;
  {
    // (C + 1) x K blocks, K slices of the pixels (the partials fit u->part's 1024 doubles)
    const int K = std::max(1, std::min(1024 / (C + 1), (int)std::min(64L, (long)B * plane0 / 4096 + 1)));
    k_head_bwd_w<<<dim3((unsigned)(C + 1), (unsigned)K), 256, 0, st>>>(u->go, d, (long)C * plane0, C, plane0, B,
                                                                      u->part);
    VIE_CHECK_LAUNCH("k_head_bwd_w");
    k_head_bwd_w_finish<<<1, ((C + 1 + 31) / 32) * 32, 0, st>>>(u->part, C, K, u->g + hd.w_off, u->g + hd.b_off);
    VIE_CHECK_LAUNCH("k_head_bwd_w_finish");
  }
  k_head_bwd_data<<<gridn((long)B * C * plane0), 256, 0, st>>>(u->go, C, u->p + hd.w_off, gd, (long)C * plane0,
                                                                plane0, B);
  VIE_CHECK_LAUNCH("k_head_bwd_data");
  --li;
  // decoder, l = 0 .. L-2 (reverse of the forward order)
  for (int l = 0; l <= L - 2; ++l) {
    const int H = n >> l;
    const long hw = (long)H * H;
    const ConvLayer &c2 = u->layers[li--];
    const ConvLayer &c1 = u->layers[li--];
    if ((s = relu_mask(u->gdl[l], (long)C * hw, u->dl[l], (long)C * hw, (long)C * hw, B, st)) != VIE_OK) return s;
    if ((s = conv3_backward(u, c2, u->bl[l], (long)C * hw, u->gdl[l], (long)C * hw, u->gbl[l], (long)C * hw, H, B,
                            st)) != VIE_OK)
      return s;
    if ((s = relu_mask(u->gbl[l], (long)C * hw, u->bl[l], (long)C * hw, (long)C * hw, B, st)) != VIE_OK) return s;
    if ((s = conv3_backward(u, c1, u->cat[l], 2L * C * hw, u->gbl[l], (long)C * hw, u->gcat[l], 2L * C * hw, H, B,
                            st)) != VIE_OK)
      return s;
    // upsample part of the concat -> gradient of d_{l+1}
    float *gnext = (l + 1 <= L - 2) ? u->gdl[l + 1] : u->gebot[0];
    k_upsample_bwd<<<coarse_grid(H, H, C, B), 256, 0, st>>>(u->gcat[l], 2L * C * hw, gnext, (long)C * hw / 4,
                                                                 C, H, H, B);
    VIE_CHECK_LAUNCH("k_upsample_bwd");
  }
  // encoder, l = L-1 .. 0; grad of e_l: concat slice (l < L-1) + pool path
  for (int l = L - 1; l >= 0; --l) {
    const int H = n >> l;
    const long hw = (long)H * H;
    const ConvLayer &c1 = u->layers[2 * l], &c2 = u->layers[2 * l + 1];
    float *ge;
    long ge_bs;
    const float *e;
    long e_bs;
    if (l < L - 1) {
      ge = u->gcat[l] + (long)C * hw;
      ge_bs = 2L * C * hw;
      e = u->cat[l] + (long)C * hw;
      e_bs = 2L * C * hw;
      // + pool path from level l+1's input gradient
      k_avgpool_bwd<<<coarse_grid(H, H, C, B), 256, 0, st>>>(u->gx[l + 1], (long)C * hw / 4, ge, ge_bs, C, H, H,
                                                              B, 1);
      VIE_CHECK_LAUNCH("k_avgpool_bwd");
    } else {
      ge = u->gebot[0];
      ge_bs = (long)C * hw;
      e = u->ebot[0];
      e_bs = (long)C * hw;
    }
    if ((s = relu_mask(ge, ge_bs, e, e_bs, (long)C * hw, B, st)) != VIE_OK) return s;
    if ((s = conv3_backward(u, c2, u->a[l], (long)C * hw, ge, ge_bs, u->ga[l], (long)C * hw, H, B, st)) != VIE_OK)
      return s;
    if ((s = relu_mask(u->ga[l], (long)C * hw, u->a[l], (long)C * hw, (long)C * hw, B, st)) != VIE_OK) return s;
    const float *xl = l == 0 ? x : u->xin[l];
    const long xl_bs = l == 0 ? 3L * hw : (long)C * hw;
    if ((s = conv3_backward(u, c1, xl, xl_bs, u->ga[l], (long)C * hw, l > 0 ? u->gx[l] : nullptr,
                            (long)C * hw, H, B, st)) != VIE_OK)
      return s;
  }
  return VIE_OK;
}

vie_status loss_grad(UnetImpl *u, const float *x, const float *t, const float *wts, int B, int n, double *loss,
                     cudaStream_t st) {
  vie_status s;
  if ((s = ensure_acts(u, B, n)) != VIE_OK) return s;
  // the training convolutions on the tensor cores in split precision: the
  // forward in three parts (24 significant bits, FP32's own: in two parts its
  // ~1e-5 relative error flipped the ReLU masks of pre-activations near zero,
  // each flip moving a gradient entry by a whole term, 3.6e-3 relative
  // against the FP64 reference, 1e-4 allowed), the input gradients in two
  struct TrainTc {
    UnetImpl *u;
    TrainTc(UnetImpl *q, int np) : u(q) { u->train_tc = np; }
    ~TrainTc() { u->train_tc = 0; }
  };
  {
    TrainTc tc3(u, 3);
    if ((s = forward<float>(u, u->p, x, B, n, st)) != VIE_OK) return s;
  }
  const long cnt = (long)B * n * n;
  const int blocks = 512;
  k_mse<<<blocks, 256, 0, st>>>(u->o, t, cnt, (long)n * n, wts, u->go, u->part);
  VIE_CHECK_LAUNCH("k_mse");
  // the loss partials leave u->part before the backward pass reuses it
  VIE_CUDA(cudaMemcpyAsync(u->h_part, u->part, sizeof(double) * blocks, cudaMemcpyDeviceToHost, st));
  VIE_CUDA(cudaMemsetAsync(u->g, 0, sizeof(float) * u->nparams, st));
  {
    TrainTc tc2(u, 2);
    if ((s = backward(u, x, B, n, st)) != VIE_OK) return s;
  }
  VIE_CUDA(cudaStreamSynchronize(st));
  double sum = 0.0;
  for (int i = 0; i < blocks; ++i) sum += u->h_part[i];
  *loss = sum / (double)cnt;
  return VIE_OK;
}

}  // namespace

// ---- used by the FGMRES driver (vie_api.cu)
vie_status unet_precondition(UnetImpl *u, const double *sigma_t, const double *sigma_s, double inv_ref,
                             const double *v, const double *vnorm2, int n, float *xbuf, const double *base,
                             double *z, cudaStream_t st) {
  vie_status s;
  if ((s = ensure_acts(u, 1, n)) != VIE_OK) return s;
  const long N = (long)n * n;
  k_net_input<<<gridn(N), 256, 0, st>>>(sigma_t, sigma_s, v, vnorm2, N, (float)inv_ref, xbuf);
  VIE_CHECK_LAUNCH("k_net_input");
  if ((s = forward<__nv_bfloat16>(u, u->pb, xbuf, 1, n, st)) != VIE_OK) return s;
  k_net_output<<<gridn(N), 256, 0, st>>>(base ? base : v, vnorm2, u->o, N, z);
  VIE_CHECK_LAUNCH("k_net_output");
  return VIE_OK;
}

// R preconditioner applications in one forward pass of R images (the batched
// FGMRES driver): z_r = base_r + rms(v_r) Net(sigma_t / s_ref, sigma_s / s_ref,
// v_r / rms(v_r)), BF16 weights; base_r = v_r, or (base non-null) another
// preconditioner's result that the network corrects.
vie_status unet_precondition_batch(UnetImpl *u, const double *sigma_t, const double *sigma_s, double inv_ref,
                                   const double *v, long ldv, const double *scal, int slot, int R, int n,
                                   float *xbuf, const double *base, long ldb, double *z, long ldz, cudaStream_t st) {
  vie_status s;
  if ((s = ensure_acts(u, R, n)) != VIE_OK) return s;
  const long N = (long)n * n;
  const dim3 grid((unsigned)std::max(1L, std::min((N + 255) / 256, 1024L)), (unsigned)R);
  k_net_input_b<<<grid, 256, 0, st>>>(sigma_t, sigma_s, v, ldv, scal, slot, N, (float)inv_ref, xbuf);
  VIE_CHECK_LAUNCH("k_net_input_b");
  if ((s = forward<__nv_bfloat16>(u, u->pb, xbuf, R, n, st)) != VIE_OK) return s;
  k_net_output_b<<<grid, 256, 0, st>>>(base ? base : v, base ? ldb : ldv, scal, slot, u->o, N, z, ldz);
  VIE_CHECK_LAUNCH("k_net_output_b");
  return VIE_OK;
}

// VIE_ERR_TIMEOUT (and the word cleared) if a tensor-core convolution of this
// network gave up on a bounded wait since the last check; synchronises `st`.
vie_status unet_take_error(UnetImpl *u, cudaStream_t st) {
  int e = 0;
  VIE_CUDA(cudaMemcpyAsync(&e, u->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  VIE_CUDA(cudaStreamSynchronize(st));
  if (e == 0) return VIE_OK;
  VIE_CUDA(cudaMemsetAsync(u->dev_err, 0, sizeof(int), st));
  set_error("a tensor-core convolution gave up on a bounded device wait (its output is NaN)");
  return VIE_ERR_TIMEOUT;
}

int *unet_error_word(UnetImpl *u) { return u->dev_err; }

}  // namespace vie

using namespace vie;

struct vie_unet {
  UnetImpl impl;
};

namespace vie {
UnetImpl *unet_impl(vie_unet *u) { return &u->impl; }
int unet_levels(vie_unet *u) { return u->impl.L; }
}  // namespace vie

extern "C" {

vie_status vie_unet_create(vie_unet **out, int levels, int channels, unsigned long long seed, int device) {
  if (!out || levels < 1 || levels > 6 || channels < 1 || channels > 32) {
    set_error("vie_unet_create: 1 <= levels <= 6, 1 <= channels <= 32");
    return VIE_ERR_INVALID_ARG;
  }
  *out = nullptr;
  int prev = -1;
  cudaGetDevice(&prev);
  VIE_CUDA(cudaSetDevice(device));
  vie_unet *u = new vie_unet();
  UnetImpl &U = u->impl;
  U.L = levels;
  U.C = channels;
  U.device = device;
  long off = 0;
  long tc = 0;  // packed BF16 weights of the 3x3 layers
  auto add = [&](int co, int ci, int k) {
    ConvLayer c{co, ci, k, off, off + (long)co * ci * k * k, tc};
    off = c.b_off + co;
    if (k == 3) tc += 9L * ((ci + kTmaSlice - 1) / kTmaSlice) * co * kTmaSlice;
    U.layers.push_back(c);
  };
  for (int l = 0; l < levels; ++l) {
    add(channels, l == 0 ? 3 : channels, 3);
    add(channels, channels, 3);
  }
  for (int l = levels - 2; l >= 0; --l) {
    add(channels, 2 * channels, 3);
    add(channels, channels, 3);
  }
  add(1, channels, 1);
  U.nparams = off;
  U.ptc_elems = tc;
  long max_w = 0;
  for (auto &c : U.layers) max_w = std::max(max_w, (long)c.co * c.ci * c.k * c.k);
  // He initialisation from SplitMix64 + Box-Muller, biases zero
  std::vector<float> h(off, 0.f);
  unsigned long long state = seed;
  auto next = [&]() {
    state += 0x9E3779B97F4A7C15ull;
    unsigned long long z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  };
  for (auto &c : U.layers) {
    const double std = sqrt(2.0 / (c.ci * c.k * c.k));
    for (long i = 0; i < (long)c.co * c.ci * c.k * c.k; ++i) {
      const double u1 = next(), u2 = next();
      h[c.w_off + i] = (float)(std * sqrt(-2.0 * log(u1)) * cos(2.0 * kPi * u2));
    }
  }
  vie_status s = VIE_OK;
  cudaError_t e = cudaSuccess;
  for (float **q : {&U.p, &U.g, &U.m, &U.v})
    if (e == cudaSuccess) e = vie_malloc((void **)q, sizeof(float) * off);
  if (e == cudaSuccess) e = vie_malloc((void **)&U.wt, sizeof(float) * max_w);
  if (e == cudaSuccess) e = vie_malloc((void **)&U.pb, sizeof(__nv_bfloat16) * off);
  if (e == cudaSuccess) e = vie_malloc((void **)&U.dev_err, sizeof(int));
  if (e == cudaSuccess) e = vie_malloc((void **)&U.ptc, sizeof(__nv_bfloat16) * std::max(1L, U.ptc_elems));
  if (e == cudaSuccess) e = cudaMemset(U.dev_err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(U.p, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(U.m, 0, sizeof(float) * off);
  if (e == cudaSuccess) e = cudaMemset(U.v, 0, sizeof(float) * off);
  if (e != cudaSuccess) s = cuda_fail(e, "vie_unet_create");
  if (s == VIE_OK) {
    k_to_bf16<<<gridn(off), 256>>>(U.p, U.pb, off);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) s = cuda_fail(e, "vie_unet_create");
  }
  if (prev >= 0) cudaSetDevice(prev);
  if (s != VIE_OK) {
    for (void *q : {(void *)U.p, (void *)U.g, (void *)U.m, (void *)U.v, (void *)U.wt, (void *)U.pb,
                    (void *)U.dev_err, (void *)U.ptc})
      if (q) vie_free(q);
    delete u;
    return s;
  }
  *out = u;
  return VIE_OK;
}

vie_status vie_unet_destroy(vie_unet *u) {
  if (!u) return VIE_OK;
  cudaSetDevice(u->impl.device);
  cudaDeviceSynchronize();
  free_acts(&u->impl);
  for (void *q : {(void *)u->impl.p, (void *)u->impl.g, (void *)u->impl.m, (void *)u->impl.v,
                  (void *)u->impl.wt, (void *)u->impl.pb, (void *)u->impl.dev_err, (void *)u->impl.ptc})
    if (q) vie_free(q);
  delete u;
  return VIE_OK;
}

vie_status vie_unet_num_params(vie_unet *u, long long *n) {
  if (!u || !n) return VIE_ERR_INVALID_ARG;
  *n = u->impl.nparams;
  return VIE_OK;
}

vie_status vie_unet_get_params(vie_unet *u, float *host) {
  if (!u || !host) return VIE_ERR_INVALID_ARG;
  VIE_CUDA(cudaSetDevice(u->impl.device));
  VIE_CUDA(cudaMemcpy(host, u->impl.p, sizeof(float) * u->impl.nparams, cudaMemcpyDeviceToHost));
  return VIE_OK;
}

vie_status vie_unet_set_params(vie_unet *u, const float *host) {
  if (!u || !host) return VIE_ERR_INVALID_ARG;
  VIE_CUDA(cudaSetDevice(u->impl.device));
  VIE_CUDA(cudaMemcpy(u->impl.p, host, sizeof(float) * u->impl.nparams, cudaMemcpyHostToDevice));
  u->impl.ptc_dirty = true;
  k_to_bf16<<<gridn(u->impl.nparams), 256>>>(u->impl.p, u->impl.pb, u->impl.nparams);
  VIE_CHECK_LAUNCH("k_to_bf16");
  VIE_CUDA(cudaDeviceSynchronize());
  return VIE_OK;
}

vie_status vie_unet_forward(vie_unet *u, const float *x, float *o, int B, int n, int use_bf16, void *stream) {
  if (!u || !x || !o || B < 1 || n < 1 || (n % (1 << (u->impl.L - 1))) != 0) {
    set_error("vie_unet_forward: n must be divisible by 2^(levels-1)");
    return VIE_ERR_INVALID_ARG;
  }
  VIE_CUDA(cudaSetDevice(u->impl.device));
  cudaStream_t st = (cudaStream_t)stream;
  vie_status s = ensure_acts(&u->impl, B, n);
  if (s != VIE_OK) return s;
  s = use_bf16 ? forward<__nv_bfloat16>(&u->impl, u->impl.pb, x, B, n, st)
               : forward<float>(&u->impl, u->impl.p, x, B, n, st);
  if (s != VIE_OK) return s;
  VIE_CUDA(cudaMemcpyAsync(o, u->impl.o, sizeof(float) * (long)B * n * n, cudaMemcpyDeviceToDevice, st));
  // the tensor-core convolutions report a bounded wait that gave up here
  if (use_bf16) return unet_take_error(&u->impl, st);
  return VIE_OK;
}

vie_status vie_unet_layer_io(vie_unet *u, int layer, float *in, float *out, void *stream) {
  if (!u || !out || layer < 0 || layer >= (int)u->impl.layers.size() || u->impl.B < 1) {
    set_error("vie_unet_layer_io: no forward yet, or layer out of range");
    return VIE_ERR_INVALID_ARG;
  }
  UnetImpl &U = u->impl;
  VIE_CUDA(cudaSetDevice(U.device));
  cudaStream_t st = (cudaStream_t)stream;
  const int L = U.L, C = U.C, B = U.B, n = U.n;
  const ConvLayer &c = U.layers[layer];
  // where the most recent forward keeps this layer's input and output
  const float *src_in = nullptr, *src_out = nullptr;
  long in_bs = 0, out_bs = 0;
  int H = n;
  if (layer < 2 * L) {  // encoder level l: a_l = conv(x_l), e_l = conv(a_l)
    const int l = layer / 2;
    H = n >> l;
    const long hw = (long)H * H;
    if (layer % 2 == 0) {
      src_in = l == 0 ? nullptr : U.xin[l];
      in_bs = (long)c.ci * hw;
      src_out = U.a[l];
      out_bs = (long)C * hw;
    } else {
      src_in = U.a[l];
      in_bs = (long)C * hw;
      src_out = l < L - 1 ? U.cat[l] + (long)C * hw : U.ebot[0];
      out_bs = l < L - 1 ? 2L * C * hw : (long)C * hw;
    }
  } else if (layer < 2 * L + 2 * (L - 1)) {  // decoder, deepest level first
    const int k = layer - 2 * L, l = L - 2 - k / 2;
    H = n >> l;
    const long hw = (long)H * H;
    if (k % 2 == 0) {
      src_in = U.cat[l];
      in_bs = 2L * C * hw;
      src_out = U.bl[l];
      if (in) {
        // the BF16 forward hands the upsampled half to the convolution in
        // BF16 only: rebuild its FP32 copy from the level below
        const float *d = l == L - 2 ? U.ebot[0] : U.dl[l + 1];
        k_upsample<<<coarse_grid(H, H, C, B), 256, 0, st>>>(d, (long)C * hw / 4, U.cat[l], 2L * C * hw, C, H, H, B);
        VIE_CHECK_LAUNCH("k_upsample");
      }
    } else {
      src_in = U.bl[l];
      in_bs = (long)C * hw;
      src_out = U.dl[l];
    }
    out_bs = (long)C * hw;
  } else {  // head
    const long hw = (long)n * n;
    src_in = L > 1 ? U.dl[0] : U.ebot[0];
    in_bs = (long)C * hw;
    src_out = U.o;
    out_bs = hw;
  }
  const long hw = (long)H * H;
  if (in && src_in)
    VIE_CUDA(cudaMemcpy2DAsync(in, sizeof(float) * c.ci * hw, src_in, sizeof(float) * in_bs, sizeof(float) * c.ci * hw,
                               B, cudaMemcpyDefault, st));
  VIE_CUDA(cudaMemcpy2DAsync(out, sizeof(float) * c.co * hw, src_out, sizeof(float) * out_bs,
                             sizeof(float) * c.co * hw, B, cudaMemcpyDefault, st));
  VIE_CUDA(cudaStreamSynchronize(st));
  return VIE_OK;
}

vie_status vie_unet_loss_grad(vie_unet *u, const float *x, const float *t, int B, int n, float *grads_host,
                              double *loss, void *stream) {
  if (!u || !x || !t || !loss || B < 1 || (n % (1 << (u->impl.L - 1))) != 0) {
    set_error("vie_unet_loss_grad: bad arguments");
    return VIE_ERR_INVALID_ARG;
  }
  VIE_CUDA(cudaSetDevice(u->impl.device));
  cudaStream_t st = (cudaStream_t)stream;
  vie_status s = loss_grad(&u->impl, x, t, nullptr, B, n, loss, st);
  if (s != VIE_OK) return s;
  if (grads_host)
    VIE_CUDA(cudaMemcpy(grads_host, u->impl.g, sizeof(float) * u->impl.nparams, cudaMemcpyDeviceToHost));
  return VIE_OK;
}

vie_status vie_unet_train_step(vie_unet *u, const float *x, const float *t, const float *weights, int B,
                               int n, float lr, double *loss, void *stream) {
  if (!u || !x || !t || !loss || B < 1 || (n % (1 << (u->impl.L - 1))) != 0 || !(lr > 0.f)) {
    set_error("vie_unet_train_step: bad arguments");
    return VIE_ERR_INVALID_ARG;
  }
  VIE_CUDA(cudaSetDevice(u->impl.device));
  cudaStream_t st = (cudaStream_t)stream;
  UnetImpl &U = u->impl;
  vie_status s = loss_grad(&U, x, t, weights, B, n, loss, st);
  if (s != VIE_OK) return s;
  U.step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)U.step), c2 = 1.f - powf(b2, (float)U.step);
  k_adam<<<gridn(U.nparams), 256, 0, st>>>(U.p, U.g, U.m, U.v, U.pb, U.nparams, lr, b1, b2, 1e-8f, c1, c2);
  VIE_CHECK_LAUNCH("k_adam");
  U.ptc_dirty = true;
  return VIE_OK;
}

// File layout: int32 header {"UNET", version, levels, channels}, int64
// parameter count np, np FP32 parameters; version 2 adds the Adam state
// (int64 step, np FP32 first moments, np FP32 second moments) so that
// training can resume where it stopped.  Version 1 files (parameters only)
// still load, with the optimizer state reset.
vie_status vie_unet_save(vie_unet *u, const char *path) {
  if (!u || !path) return VIE_ERR_INVALID_ARG;
  UnetImpl &U = u->impl;
  const long np = U.nparams;
  std::vector<float> h(np), hm(np), hv(np);
  vie_status s = vie_unet_get_params(u, h.data());
  if (s != VIE_OK) return s;
  VIE_CUDA(cudaMemcpy(hm.data(), U.m, sizeof(float) * np, cudaMemcpyDeviceToHost));
  VIE_CUDA(cudaMemcpy(hv.data(), U.v, sizeof(float) * np, cudaMemcpyDeviceToHost));
  FILE *f = fopen(path, "wb");
  if (!f) {
    set_error(std::string("vie_unet_save: cannot open ") + path);
    return VIE_ERR_INVALID_ARG;
  }
  const int hdr[4] = {0x54454e55 /* "UNET" */, 2, U.L, U.C};
  const long long n64 = np, step = U.step;
  bool ok = fwrite(hdr, sizeof hdr, 1, f) == 1 && fwrite(&n64, sizeof n64, 1, f) == 1 &&
            fwrite(h.data(), sizeof(float), h.size(), f) == h.size() && fwrite(&step, sizeof step, 1, f) == 1 &&
            fwrite(hm.data(), sizeof(float), hm.size(), f) == hm.size() &&
            fwrite(hv.data(), sizeof(float), hv.size(), f) == hv.size();
  ok = (fclose(f) == 0) && ok;
  if (!ok) {
    set_error("vie_unet_save: write failed");
    return VIE_ERR_INVALID_ARG;
  }
  return VIE_OK;
}

vie_status vie_unet_load(vie_unet *u, const char *path) {
  if (!u || !path) return VIE_ERR_INVALID_ARG;
  UnetImpl &U = u->impl;
  FILE *f = fopen(path, "rb");
  if (!f) {
    set_error(std::string("vie_unet_load: cannot open ") + path);
    return VIE_ERR_INVALID_ARG;
  }
  int hdr[4];
  long long np = 0, step = 0;
  std::vector<float> h(U.nparams), hm(U.nparams, 0.f), hv(U.nparams, 0.f);
  bool ok = fread(hdr, sizeof hdr, 1, f) == 1 && fread(&np, sizeof np, 1, f) == 1 && hdr[0] == 0x54454e55 &&
            (hdr[1] == 1 || hdr[1] == 2) && hdr[2] == U.L && hdr[3] == U.C && np == U.nparams &&
            fread(h.data(), sizeof(float), h.size(), f) == h.size();
  if (ok && hdr[1] == 2)
    ok = fread(&step, sizeof step, 1, f) == 1 && step >= 0 &&
         fread(hm.data(), sizeof(float), hm.size(), f) == hm.size() &&
         fread(hv.data(), sizeof(float), hv.size(), f) == hv.size();
  fclose(f);
  if (!ok) {
    set_error("vie_unet_load: file does not match this network");
    return VIE_ERR_INVALID_ARG;
  }
  vie_status s = vie_unet_set_params(u, h.data());
  if (s != VIE_OK) return s;
  VIE_CUDA(cudaMemcpy(U.m, hm.data(), sizeof(float) * U.nparams, cudaMemcpyHostToDevice));
  VIE_CUDA(cudaMemcpy(U.v, hv.data(), sizeof(float) * U.nparams, cudaMemcpyHostToDevice));
  U.step = (long)step;
  return VIE_OK;
}

vie_status vie_unet_train_state(vie_unet *u, long long *step) {
  if (!u || !step) return VIE_ERR_INVALID_ARG;
  *step = u->impl.step;
  return VIE_OK;
}

}  // extern "C"
