// Displacement-major pair kernel with per-displacement stencils: 2D, FP32
// tiles, S = 64 march steps.
//
// It computes the operator of k_apply.cu (Section 2, Eq. EQ:Kernel; Section
// 3.2, M-iii): y_j = sum_{k != j} A_jk s_k, the optical depth of the segment
// from cell j to cell k = j + D (D = (dx, dy) in cells) taken by the S-step
// midpoint march of the bilinear interpolant of sigma_t.  On a uniform grid
// the samples of that march sit at u_j + (i + 1/2) D / S: their integer parts
// relative to j and their bilinear weights depend on D and i only.  Summing,
// for each lattice cell c, the weights of the samples that touch it gives a
// stencil W_D with
//     sum_i sigma(u_j + (i + 1/2) D / S) = sum_c W_D(c) sigma[j + c]
// for every j: the same products, grouped by lattice cell.  W_D has at most
// 4 S cells and far fewer when |D| < S, because consecutive samples share
// cells.  It is built once per handle on the host in FP64 and stored in FP32.
//
// W_D is stored as runs of consecutive cells along one lattice axis (the one
// that makes the march cheaper, normally the axis closer to D), each run cut
// into the fewest chunks of at most kMaxChunk cells, of equal length, so no
// chunk multiplies zero weights; a D's chunks are stored grouped by length
// Lc behind a header of counts, and each length runs in its own loop.  A
// warp takes one displacement and a block of 32 x R targets: 32 consecutive
// across the run axis (one per lane) and R consecutive along it, stacked in
// one thread.  A chunk then takes Lc + R - 1 lattice loads per thread and
// R Lc multiply-adds, issued as packed FP32 pairs (fma.rn.f32x2, two
// stacked targets per instruction) in code unrolled for each Lc.  Lanes sit
// on consecutive x (runs along y) or consecutive y with an odd row pitch
// (runs along x), so every load is free of bank conflicts.
//
// Work units are (D, block of the targets j with j + D inside the grid) for D
// in a half plane (dy > 0, or dy = 0 and dx > 0): A_jk = A_kj, so each
// unordered pair is marched once and feeds y_j (weight s_{j+D}) and y_{j+D}
// (weight s_j).  Units are sorted by estimated cost, largest first, and warps
// take them four at a time from a global counter.  Every term w s is rounded
// once to a multiple of 1/scale (64-bit fixed point, scale the power of two
// at or below 2^62 / (max|s| R), R a bound on every row sum of A) and added
// with an integer reduction (red.add, no value returned) into a global int64
// array: integer sums are exact in any order, so the result is bitwise
// reproducible whatever the schedule, and the accumulation error is below
// N 2^-63 max|s| R.  k_disp_reduce converts each sum once to FP64, adds the
// self cell and clears the array for the next apply.  Shared memory holds the
// lattice alone, which leaves the rest of the SM's L1 to the chunk records.
//
// The array has two halves: targets on consecutive x (runs along y) sum into
// the first, x fastest; targets on consecutive y (runs along x) into the
// second, y fastest.  Either way a warp's 32 atomics cover contiguous words,
// and the sources come from s or its transposed copy in the same layout.
//
// Targets of a block that fall outside the rectangle (ragged blocks) are
// computed and discarded: lanes beyond it repeat the last valid target, and
// the lattice carries R - 1 extra rows and columns (repeating the
// edge) so that stacked targets beyond it stay in bounds.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "disp_march.cuh"
#include "march.cuh"
#include "vie_internal.cuh"

namespace vie {

namespace {

using march::kS;

using dmarch::kMaxChunk;
using dmarch::march_runs;
using dmarch::march_runs_global;
// R, the targets stacked along the run axis in one thread: 12 on grids of
// 96 and more, 8 below (measured per apply: 8 / 12 took 0.100 / 0.107 ms at
// 64^2, 0.550 / 0.519 at 100^2, 1.41 / 1.38 at 128^2, 42.9 / 38.3 at 256^2;
// 16 took 1.47 at 128^2, with fewer warps resident; a last block of 4 or 8
// for the rest of a rectangle, as its own code path, 1.62).  The lattice
// carries R - 1 extra rows and columns: the stacked targets of a block that
// reach past the rectangle of targets (chunks carry no padding).
using dmarch::red_add;
constexpr int kThreads = 1024;
__host__ __device__ constexpr int disp_depth(int n) { return n >= 96 ? 12 : 8; }
// lattice pitch: room for R - 1 stacked targets past the grid, odd so that
// 32 consecutive rows of one column fall in 32 different banks
__host__ __device__ constexpr int disp_pitch(int n, int R) { return (n + R) | 1; }
// Lane groups of a ragged lane block sit s blocks apart along the stack, s R
// rows of an odd pitch: s R = 16 (mod 32) for pairs and 8 or 24 for quads,
// so the groups load from disjoint banks.
__host__ __device__ constexpr int group_stride(int R, int lg) { return lg == 1 ? (R == 8 ? 2 : 4) : (R == 8 ? 1 : 2); }
// Grids whose lattice does not fit in shared memory read it from global
// memory: a square lattice of pitch disp_pitch(kGlobalMaxN, R) (odd, like the
// shared one, so that the lane groups of a ragged block get the same
// strides), for n <= kGlobalMaxN.
constexpr int kGlobalMaxN = 258;

struct DispArgs {
  const float *lat;            // [n + R][ldp] sigma_t on the cell lattice, edge repeated
  const float *lat_t;          // global-lattice kernels: the same lattice with y fastest
  const float4 *stencil;       // chunk records of every W_D
  const float *src;            // s_k, FP32 [N]
  const float *src_t;          // s transposed: s at (x, y) is src_t[x n + y]
  const float *wtab;           // M-ii: h / (2 pi) times the cell integral of 1/|z| per D
                               // of the half plane (disp_index order); null for M-iii
  unsigned *smax;              // bits of max |s_k| (set by the source kernel)
  double *scale_out;           // fixed-point scale of this apply (for the reduce)
  double rbound;               // bound on sum_k A_jk for every j
  unsigned long long *yacc;    // [2 N] int64 sums (x fastest, then y fastest), zero between applies
  const int4 *units;           // {the D's record header (float4 index), dx | dy << 16,
                               //  lane block | stack block << 16,
                               //  runs along y | lane groups << 1 | record float4s << 12}
  int *counter;                // [2]
  float *wbuf;                 // stored weights (store: written, stream: read)
  const long long *doff;       // first stored weight of each D of the half plane
  long n_units;
  int n, ldp;
  long lat_elems;
  float tau_scale2, wcoef;
};

// What one launch does with the pairs of its units.
enum DispMode {
  kApply = 0,   // march, then y_j += w s_k and y_k += w s_j (fixed point)
  kStore = 1,   // march, then store w (FP32, displacement-major) for later applies
  kStream = 2   // read the stored w, then y_j += w s_k and y_k += w s_j
};

// index of D = (dx, dy) in the half plane, in the order the geometry lists them
__device__ __forceinline__ int disp_index(int dx, int dy, int n) {
  return dy == 0 ? dx - 1 : (n - 1) + (dy - 1) * (2 * n - 1) + (dx + n - 1);
}

// GLAT: the lattice stays in global memory (read through L1).  Units whose
// runs go along y read lat from (x, y) on, the others lat_t from (y, x) on:
// in both the run axis has stride LDP and the lanes are consecutive elements,
// and the records of the runs along x carry their offsets in lat_t's layout.
template <int LDP, int MODE, bool GLAT, int R>
__device__ __forceinline__ void disp_body(const DispArgs &a) {
  extern __shared__ float4 smem4[];
  const int n = a.n;
  const long N = (long)n * n;
  // shared memory: the lattice (none when streaming)
  float *lat = reinterpret_cast<float *>(smem4);
  const int tid = threadIdx.x, lane = tid & 31;
  if constexpr (MODE != kStream && !GLAT) {
    const float4 *g4 = reinterpret_cast<const float4 *>(a.lat);
    float4 *l4 = reinterpret_cast<float4 *>(lat);
    const long n4 = a.lat_elems / 4;
    for (long i = tid; i < n4; i += kThreads) l4[i] = g4[i];
    for (long i = n4 * 4 + tid; i < a.lat_elems; i += kThreads) lat[i] = a.lat[i];
  }
  __syncthreads();
  // power-of-two scale: 2^k <= 2^62 / (max|s| R), so w * scale is exact
  double scale_d = 1.0;
  if constexpr (MODE != kStore) {
    const float smax = __uint_as_float(*a.smax);
    if (smax > 0.f) scale_d = ldexp(1.0, ilogb(4.611686018427387904e18 / ((double)smax * a.rbound)));
  }
  const float scale = (float)scale_d;
  const int ldp = LDP > 0 ? LDP : a.ldp;
  const unsigned lat_base = (unsigned)__cvta_generic_to_shared(lat);
  long u0 = 0, u_end = 0;
  for (;;) {
    if (u0 >= u_end) {
      long got = 0;
      if (lane == 0) got = atomicAdd(a.counter, 4);
      got = __shfl_sync(0xffffffffu, got, 0);
      if (got >= a.n_units) break;
      u0 = got;
      u_end = min(got + 4, a.n_units);
    }
    const int4 un = a.units[u0++];
    {
    const int dx = (short)(un.y & 0xffff), dy = un.y >> 16;
    const int lb = un.z & 0xffff, row0 = un.z >> 16;
    const int xlo = dx < 0 ? -dx : 0, xhi = dx > 0 ? n - dx : n;
    const int ylo = dy < 0 ? -dy : 0, yhi = dy > 0 ? n - dy : n;
    const bool along_y = (un.w & 1) != 0;
    const int lg = (un.w >> 1) & 3, nrec = un.w >> 12;
    // lane groups: 1, 2 or 4 groups of 32 >> lg lanes, group g on the block
    // starting R s g rows after row0 (s = group_stride); a group past the
    // last block is masked off
    const int gw = 32 >> lg, g = lane >> (5 - lg), lig = lane & (gw - 1);
    const int stack = along_y ? yhi - ylo : xhi - xlo;
    int row = row0 + R * group_stride(R, lg) * g;
    bool lvalid = row < stack;
    if (!lvalid) row = row0;
    // lane coordinate (clamped to the rectangle) and the first stacked target
    int x, y;
    if (along_y) {
      const int xr = xlo + 32 * lb + lig;
      lvalid = lvalid && xr < xhi;
      x = xr < xhi ? xr : xhi - 1;
      y = ylo + row;
    } else {
      const int yr = ylo + 32 * lb + lig;
      lvalid = lvalid && yr < yhi;
      y = yr < yhi ? yr : yhi - 1;
      x = xlo + row;
    }
    float acc[R];
#pragma unroll
    for (int q = 0; q < R; ++q) acc[q] = 0.f;
    if constexpr (MODE != kStream) {
      const unsigned base = lat_base + 4u * (unsigned)(x + ldp * y);
      {
        // bring this D's chunk records into L1 (one 128-byte line per lane)
        const char *r0 = reinterpret_cast<const char *>(a.stencil + un.x);
        const int lines = (int)(((reinterpret_cast<size_t>(r0) & 127) + 16L * nrec + 127) >> 7);
        for (int l = lane; l < lines; l += 32) asm volatile("prefetch.global.L1 [%0];" ::"l"(r0 + 128L * l));
      }
      if constexpr (GLAT) {
        const float *gb = along_y ? a.lat + (x + (long)LDP * y) : a.lat_t + (y + (long)LDP * x);
        march_runs_global<LDP, R>(a.stencil + un.x, gb, acc);
      } else if (along_y) {
        march_runs<LDP, R>(a.stencil + un.x, base, ldp, acc);
      } else {
        march_runs<1, R>(a.stencil + un.x, base, 1, acc);
      }
    }
    const float r2 = (float)(dx * dx + dy * dy);
    const float inv_r = rsqrtf(r2);
    const float tscale = -a.tau_scale2 * r2 * inv_r;  // -(h/S) log2(e) r
    // M-iii: h^2 / (2 pi r) = (h / 2 pi) / |D|; M-ii: the closed-form cell
    // integral of |x_j - z|^{-1} over T_k (Remark REM: NEW KERNEL), per D
    const float wk = a.wtab ? __ldg(a.wtab + disp_index(dx, dy, n)) : a.wcoef * inv_r;
    // stored weights of D: its rectangle of targets, row-major (lanes along x
    // write 128 contiguous bytes; lanes along y each write their R targets)
    long woff = 0;
    if constexpr (MODE != kApply) woff = a.doff[disp_index(dx, dy, n)];
    const int wx = xhi - xlo;
    // sums of targets on consecutive x (runs along y) go to yacc with x
    // fastest, those on consecutive y (runs along x) to its second half with
    // y fastest, so a warp's atomics cover contiguous words; s and its
    // transpose follow the same layouts.  Stacked targets are n apart in both.
    const float *sv = along_y ? a.src : a.src_t;
    unsigned long long *ya = along_y ? a.yacc : a.yacc + N;
    const long j0 = along_y ? (long)y * n + x : (long)x * n + y;
    const long dk = along_y ? (long)dy * n + dx : (long)dx * n + dy;
    if constexpr (MODE == kStream) {
      // four targets at a time: their global loads are issued before their atomics
#pragma unroll
      for (int q0 = 0; q0 < R; q0 += 4) {
        float wv[4], sjv[4], skv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int q = q0 + i;
          const int xq = along_y ? x : x + q, yq = along_y ? y + q : y;
          wv[i] = sjv[i] = skv[i] = 0.f;
          if (lvalid && (along_y ? yq < yhi : xq < xhi)) {
            const long wi = woff + (long)(yq - ylo) * wx + (xq - xlo);
            wv[i] = __ldcs(a.wbuf + wi);
            sjv[i] = __ldg(sv + j0 + (long)q * n);
            skv[i] = __ldg(sv + j0 + (long)q * n + dk);
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int q = q0 + i;
          const int xq = along_y ? x : x + q, yq = along_y ? y + q : y;
          if (lvalid && (along_y ? yq < yhi : xq < xhi)) {
            const float w = wv[i] * scale;
            const long j = j0 + (long)q * n;
            red_add(ya + j, (unsigned long long)__float2ll_rn(w * skv[i]));
            red_add(ya + j + dk, (unsigned long long)__float2ll_rn(w * sjv[i]));
          }
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int xq = along_y ? x : x + q, yq = along_y ? y + q : y;
        if (lvalid && (along_y ? yq < yhi : xq < xhi)) {
          const float wq = wk * exp2f(tscale * acc[q]);
          if constexpr (MODE == kStore) {
            a.wbuf[woff + (long)(yq - ylo) * wx + (xq - xlo)] = wq;
          } else {
            const long j = j0 + (long)q * n;
            const float sj = __ldg(sv + j), sk = __ldg(sv + j + dk);
            const float w = wq * scale;
            red_add(ya + j, (unsigned long long)__float2ll_rn(w * sk));
            red_add(ya + j + dk, (unsigned long long)__float2ll_rn(w * sj));
          }
        }
      }
    }
    }
  }
  // every warp of this CTA is past its last unit before the CTA counts as done
  // (the last CTA resets the unit counter for the next launch)
  __syncthreads();
  if constexpr (MODE != kStore) {
    if (blockIdx.x == 0 && tid == 0) *a.scale_out = scale_d;
  }
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(a.counter + 1, 1) == (int)gridDim.x - 1) {
      a.counter[0] = 0;
      a.counter[1] = 0;
      if (MODE != kStore) *a.smax = 0u;  // every CTA read it before this, the next source kernel sets it
      __threadfence();
    }
  }
}

template <int LDP, int R>
__global__ void __launch_bounds__(kThreads, 1) k_pairs_disp(DispArgs a) {
  disp_body<LDP, kApply, false, R>(a);
}

template <int LDP, int R>
__global__ void __launch_bounds__(kThreads, 1) k_store_disp(DispArgs a) {
  disp_body<LDP, kStore, false, R>(a);
}

template <int R>
__global__ void __launch_bounds__(kThreads, 1) k_stream_disp(DispArgs a) {
  disp_body<1, kStream, false, R>(a);
}

template <int R>
__global__ void __launch_bounds__(kThreads, 1) k_pairs_disp_global(DispArgs a) {
  disp_body<disp_pitch(kGlobalMaxN, R), kApply, true, R>(a);
}

template <int R>
__global__ void __launch_bounds__(kThreads, 1) k_store_disp_global(DispArgs a) {
  disp_body<disp_pitch(kGlobalMaxN, R), kStore, true, R>(a);
}


// output forms of the expansion
enum ExpandOut {
  kDenseF32 = 0,   // K row-major, FP32
  kDenseBF16 = 1,  // K row-major, BF16 hi + lo
  kSymBlocks = 2   // A (no sigma_s) in the n (n + 1) / 2 blocks of grid-row pairs yj <= yk
};

template <int OUT>
__device__ __forceinline__ void put_entry(long idx, float v, float *k32, unsigned short *khi, unsigned short *klo) {
  if constexpr (OUT == kDenseBF16) {
    const unsigned short hi = bf16_bits_rn(v);
    khi[idx] = hi;
    klo[idx] = bf16_bits_rn(v - __uint_as_float((unsigned)hi << 16));
  } else {
    k32[idx] = v;
  }
}

// K_jk = A_jk sigma_s,k (j != k) and K_jj = d_j sigma_s,j, row-major N x ldk
// (FP32, or BF16 hi + lo with lo = bf16(v - hi)), from the stored pair
// weights, each read once.  An item is (dy, target row yj): the stored rows
// "D = (dx, dy), targets (., yj)" of every dx go to shared memory
// (T[dx + n - 1][xj]), then
//   K[j][k]  = T sigma_s,k  for j = (xj, yj), k = (xk, yj + dy), and
//   K[k][j]  = T sigma_s,j  for the same pairs seen from k,
// each written as whole row segments of n columns.  Every ordered pair is
// written once: by its own D when D is in the half plane, else from -D.  For
// dy = 0 the row of j gets its columns k > j from the first part and k < j
// from the second, and the diagonal K_jj = d_j sigma_s,j.

//
// kSymBlocks writes A itself (A_jk = A_kj, no sigma_s): block t = item (dy, yj),
// n x n row-major at t n^2, row xj, column xk; only the first part (and for
// dy = 0 the whole block with its diagonal d_j).
template <int OUT>
__global__ void __launch_bounds__(1024, 1) k_expand_pairs(int n, const float *__restrict__ w,
                                                          const long long *__restrict__ doff,
                                                          const float *__restrict__ ss,
                                                          const double *__restrict__ diag,
                                                          const double *__restrict__ ss64, long ldk, float *k32,
                                                          unsigned short *khi, unsigned short *klo) {
  extern __shared__ float T[];  // [2n - 1][p]
  const int p = n + 2;           // strides p and 1 - p: at most one is even (2-way conflicts)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, warps = blockDim.x >> 5;
  const int items = n * (n + 1) / 2;
  // item t -> (dy, yj), rows of dy holding n - dy items; advanced by gridDim.x per step
  int dy = 0, yj = blockIdx.x;
  while (dy < n && yj >= n - dy) {
    yj -= n - dy;
    ++dy;
  }
  for (int t = blockIdx.x; t < items; t += gridDim.x) {
    if (t != (int)blockIdx.x) {
      yj += gridDim.x;
      while (dy < n && yj >= n - dy) {
        yj -= n - dy;
        ++dy;
      }
    }
    const int yk = yj + dy;
    for (int dx = -(n - 1) + warp; dx < n; dx += warps) {
      if (dy == 0 && dx <= 0) continue;
      const int xlo = dx < 0 ? -dx : 0, wx = n - (dx < 0 ? -dx : dx);
      const float *row = w + doff[disp_index(dx, dy, n)] + (long)yj * wx;
      float *trow = T + (dx + n - 1) * p + xlo;
      for (int x = lane; x < wx; x += 32) trow[x] = __ldcs(row + x);
    }
    __syncthreads();
    const long jrow = (long)n * yj, krow = (long)n * yk;
    const float *ssj = ss + jrow, *ssk = ss + krow;
    if constexpr (OUT == kSymBlocks) {
      float *blk = k32 + (long)t * n * n;
      for (int xj = warp; xj < n; xj += warps) {
        float *out = blk + (long)xj * n;
        for (int xk = lane; xk < n; xk += 32) {
          const int dx = xk - xj;
          float v;
          if (dy > 0 || dx > 0)
            v = T[(dx + n - 1) * p + xj];
          else if (dx < 0)
            v = T[(-dx + n - 1) * p + xk];  // A_jk = A_kj, stored under (-dx, 0) for target xk
          else
            v = (float)diag[jrow + xj];
          out[xk] = v;
        }
      }
    } else if (dy > 0) {
      // every (xj, xk) is a pair of this item
      for (int xj = warp; xj < n; xj += warps) {
        const float *tb = T + (n - 1 - xj) * p + xj;  // T[(xk - xj + n - 1) p + xj]
        const long rb = (jrow + xj) * ldk + krow;
        for (int xk = lane; xk < n; xk += 32) put_entry<OUT>(rb + xk, tb[xk * p] * ssk[xk], k32, khi, klo);
      }
      for (int xk = warp; xk < n; xk += warps) {
        const float *tb = T + (xk + n - 1) * p;  // T[(xk - xj + n - 1) p + xj]
        const long rb = (krow + xk) * ldk + jrow;
        for (int xj = lane; xj < n; xj += 32) put_entry<OUT>(rb + xj, tb[xj * (1 - p)] * ssj[xj], k32, khi, klo);
      }
    } else {
      // one grid row: columns right of the diagonal from j, left of it from k
      for (int r = warp; r < n; r += warps) {
        const long rb = (jrow + r) * ldk + jrow;
        for (int x = lane; x < n; x += 32) {
          if (x == r) continue;
          const float v = x > r ? T[(x - r + n - 1) * p + r] : T[(r - x + n - 1) * p + x];
          put_entry<OUT>(rb + x, v * ssj[x], k32, khi, klo);
        }
      }
      for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const long j = jrow + r;
        put_entry<OUT>(j * ldk + j, (float)(diag[j] * ss64[j]), k32, khi, klo);
      }
    }
    __syncthreads();
  }
}

// ---- applies of A stored as symmetric blocks (the kSymBlocks expansion)
//
// y = A s with s = sigma_s g (or g): block t = (dy, yj) holds A_jk for j on
// grid row yj, k on grid row yj + dy.  k_symv_blocks reads each block once and
// writes P[t][0, n) = its row sums against s on row yj + dy and, for dy > 0,
// P[t][n, 2n) = its column sums against s on row yj (A_kj = A_jk); all sums
// in a fixed order.  k_symv_reduce adds, for each target, the partials of the
// n blocks that touch its grid row, in block order.
constexpr int kSymvCols = 5;  // columns per lane: n <= 32 kSymvCols

__device__ __forceinline__ int symv_item(int dy, int yj, int n) { return dy * n - dy * (dy - 1) / 2 + yj; }

__global__ void __launch_bounds__(256) k_symv_blocks(int n, const float *__restrict__ A, const float *__restrict__ s,
                                                     float *__restrict__ P) {
  __shared__ float colpart[8][32 * kSymvCols];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int items = n * (n + 1) / 2;
  int dy = 0, yj = blockIdx.x;
  while (dy < n && yj >= n - dy) {
    yj -= n - dy;
    ++dy;
  }
  for (int t = blockIdx.x; t < items; t += gridDim.x) {
    if (t != (int)blockIdx.x) {
      yj += gridDim.x;
      while (dy < n && yj >= n - dy) {
        yj -= n - dy;
        ++dy;
      }
    }
    const float *blk = A + (long)t * n * n;
    const float *sJ = s + (long)n * yj, *sK = s + (long)n * (yj + dy);
    float sk[kSymvCols], ca[kSymvCols];
#pragma unroll
    for (int i = 0; i < kSymvCols; ++i) {
      const int c = lane + 32 * i;
      sk[i] = c < n ? sK[c] : 0.f;
      ca[i] = 0.f;
    }
    // four rows of the block per warp in flight
    for (int r0 = 4 * warp; r0 < n; r0 += 32) {
      float a[4][kSymvCols];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int i = 0; i < kSymvCols; ++i) {
          const int r = r0 + u, c = lane + 32 * i;
          a[u][i] = r < n && c < n ? __ldcs(blk + (long)r * n + c) : 0.f;
        }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = r0 + u;
        const float sjr = r < n ? sJ[r] : 0.f;
        float rs = 0.f;
#pragma unroll
        for (int i = 0; i < kSymvCols; ++i) {
          rs = fmaf(a[u][i], sk[i], rs);
          ca[i] = fmaf(a[u][i], sjr, ca[i]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
        if (lane == 0 && r < n) P[(long)t * 2 * n + r] = rs;
      }
    }
    if (dy > 0) {  // uniform over the CTA
#pragma unroll
      for (int i = 0; i < kSymvCols; ++i) colpart[warp][lane + 32 * i] = ca[i];
      __syncthreads();
      for (int c = threadIdx.x; c < n; c += blockDim.x) {
        float v = 0.f;
#pragma unroll
        for (int w8 = 0; w8 < 8; ++w8) v += colpart[w8][c];
        P[(long)t * 2 * n + n + c] = v;
      }
      __syncthreads();
    }
  }
}

// four threads per target (one quarter of its n block sums each, 64 targets per
// CTA), their sums added in part order
__global__ void __launch_bounds__(256) k_symv_reduce(int n, int op, const float *__restrict__ P,
                                                     const double *__restrict__ g, double *__restrict__ y) {
  __shared__ double part[4][64];
  const long N = (long)n * n;
  const int tx = threadIdx.x & 63, q = threadIdx.x >> 6;
  for (long j0 = blockIdx.x * 64L; j0 < N; j0 += gridDim.x * 64L) {
    const long j = j0 + tx;
    double acc = 0.0;
    if (j < N) {
      const int x = (int)(j % n), yl = (int)(j / n);
      // the target's n blocks: (yl, yl + dy) for dy < n - yl (row sums), then
      // (yl - dy, yl) for 1 <= dy <= yl (column sums); part q takes every 4th
      for (int b = q; b < n; b += 4) {
        const int dy = b < n - yl ? b : b - (n - yl) + 1;
        acc += b < n - yl ? P[(long)symv_item(dy, yl, n) * 2 * n + x]
                          : P[(long)symv_item(dy, yl - dy, n) * 2 * n + n + x];
      }
    }
    part[q][tx] = acc;
    __syncthreads();
    if (q == 0 && j < N) {
      const double v = ((part[0][tx] + part[1][tx]) + part[2][tx]) + part[3][tx];
      y[j] = op == VIE_OP_I_MINUS_K ? g[j] - v : v;
    }
    __syncthreads();
  }
}

__global__ void k_symv_source(long N, int op, const double *__restrict__ ss, const double *__restrict__ g,
                              float *__restrict__ s) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x)
    s[i] = (float)(op == VIE_OP_A_RAW ? g[i] : ss[i] * g[i]);
}

// FP32 copy of sigma_s (the expansion multiplies in FP32, as the on-the-fly
// kernels do)
__global__ void k_to_f32(long N, const double *__restrict__ x, float *__restrict__ y) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

// the padded FP32 lattice (pitch P = n + 1) extended to rows x ldp, repeating
// its last row and column; transposed: element i = x ldp + y holds point (x, y)
__global__ void k_make_lattice(int n, const float *__restrict__ pad, int rows, int ldp, int transposed,
                               float *__restrict__ out) {
  const int P = n + 1;
  const long total = (long)rows * ldp;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int r = (int)(i / ldp), c = (int)(i % ldp);
    const int y = transposed ? c : r, x = transposed ? r : c;
    out[i] = pad[(long)min(y, P - 1) * P + min(x, P - 1)];
  }
}

// y_j = (both sums of j) / scale + d_j s_j, and yacc back to zero for the
// next apply.  yacc holds N sums with x fastest, then N with y fastest.
__global__ void k_disp_reduce(long N, int n, int op, unsigned long long *__restrict__ yacc,
                              const double *__restrict__ scale, const double *__restrict__ diag,
                              const double *__restrict__ ss, const double *__restrict__ g,
                              double *__restrict__ y) {
  const double inv = 1.0 / *scale;
  for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < N; j += (long)gridDim.x * blockDim.x) {
    const long jt = N + (j % n) * n + j / n;
    const unsigned long long acc = yacc[j] + yacc[jt];
    yacc[j] = 0ull;
    yacc[jt] = 0ull;
    const double sj = op == VIE_OP_A_RAW ? g[j] : ss[j] * g[j];
    const double v = (double)(long long)acc * inv + diag[j] * sj;
    y[j] = op == VIE_OP_I_MINUS_K ? g[j] - v : v;
  }
}

// s = sigma_s g (or g) in FP32, its transpose, and max |s| (float bits, atomicMax)
__global__ void k_disp_source(long N, int n, int op, const double *__restrict__ ss, const double *__restrict__ g,
                              float *__restrict__ s, float *__restrict__ s_t, unsigned *__restrict__ smax) {
  unsigned m = 0u;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    const float v = (float)(op == VIE_OP_A_RAW ? g[i] : ss[i] * g[i]);
    s[i] = v;
    s_t[(i % n) * n + i / n] = v;
    m = max(m, __float_as_uint(fabsf(v)));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(smax, m);
}

typedef void (*DispKernel)(DispArgs);

// compile-time lattice pitches of the 64^2 and 128^2 grids (stack depths
// disp_depth(64) = 8 and disp_depth(128) = 12)
constexpr int kLdp64 = disp_pitch(64, disp_depth(64)), kLdp128 = disp_pitch(128, disp_depth(128));

// the shared-lattice apply (store) kernel of lattice pitch ldp, depth R
DispKernel pick_disp(int ldp, int R, bool store) {
  if (R == 8) {
    if (ldp == kLdp64) return store ? k_store_disp<kLdp64, 8> : k_pairs_disp<kLdp64, 8>;
    return store ? k_store_disp<0, 8> : k_pairs_disp<0, 8>;
  }
  if (ldp == kLdp128) return store ? k_store_disp<kLdp128, 12> : k_pairs_disp<kLdp128, 12>;
  return store ? k_store_disp<0, 12> : k_pairs_disp<0, 12>;
}


struct Cell {
  int cx, cy;
  double w;
};

// W_D: the bilinear weights of the S midpoint samples (i + 1/2) D / S summed
// per lattice cell (Section 3.2, M-iii), cells with zero weight left out;
// sorted by (cx, cy) when runs go along y, by (cy, cx) when they go along x
void stencil_cells(int dx, int dy, bool along_y, std::vector<Cell> &out) {
  std::vector<Cell> raw;
  raw.reserve(4 * kS);
  for (int i = 0; i < kS; ++i) {
    const double px = (i + 0.5) * dx / kS, py = (i + 0.5) * dy / kS;
    const double fx = floor(px), fy = floor(py), ax = px - fx, ay = py - fy;
    const int ix = (int)fx, iy = (int)fy;
    const double w[4] = {(1.0 - ax) * (1.0 - ay), ax * (1.0 - ay), (1.0 - ax) * ay, ax * ay};
    for (int c = 0; c < 4; ++c)
      if (w[c] != 0.0) raw.push_back({ix + (c & 1), iy + (c >> 1), w[c]});
  }
  std::sort(raw.begin(), raw.end(), [along_y](const Cell &p, const Cell &q) {
    return along_y ? (p.cx != q.cx ? p.cx < q.cx : p.cy < q.cy) : (p.cy != q.cy ? p.cy < q.cy : p.cx < q.cx);
  });
  out.clear();
  for (const Cell &c : raw) {
    if (!out.empty() && out.back().cx == c.cx && out.back().cy == c.cy)
      out.back().w += c.w;
    else
      out.push_back(c);
  }
}

// run lengths of sorted cells (a run: consecutive cells along the run axis)
void stencil_runs(const std::vector<Cell> &cells, bool along_y, std::vector<int> &starts) {
  starts.clear();
  for (size_t i = 0; i < cells.size(); ++i) {
    const bool cont = i > 0 && (along_y ? cells[i].cx == cells[i - 1].cx && cells[i].cy == cells[i - 1].cy + 1
                                        : cells[i].cy == cells[i - 1].cy && cells[i].cx == cells[i - 1].cx + 1);
    if (!cont) starts.push_back((int)i);
  }
  starts.push_back((int)cells.size());
}

// A run of L cells is cut into ceil(L / kMaxChunk) chunks of equal length
// (their lengths differ by at most one).  Estimated instructions per thread of
// one unit of stack depth R: per chunk its record loads and loop, Lc + R - 1
// lattice loads, the packed multiply-adds (R / 2 per even tap, R / 2 + 1 per
// odd one) and a weight broadcast per tap; per unit the epilogue.
struct Plan {
  long chunks, recs, cost;
};
long chunk_cost(int lc, int R) {
  return 4 + (lc + 4) / 4 + (lc + R - 1) + ((lc + 1) / 2) * (R / 2) + (lc / 2) * (R / 2 + 1) + lc;
}
// estimated cost of all units of one D for stack `stack` across `lanes` lanes
long axis_cost(const Plan &p, int lanes, int stack, int R) {
  return (long)((lanes + 31) / 32) * ((stack + R - 1) / R) * p.cost;
}
template <typename F>
void for_each_chunk(const std::vector<int> &starts, F f) {
  for (size_t r = 0; r + 1 < starts.size(); ++r) {
    const int L = starts[r + 1] - starts[r], nch = (L + kMaxChunk - 1) / kMaxChunk;
    int c0 = starts[r];
    for (int c = 0; c < nch; ++c) {
      const int lc = L / nch + (c < L % nch ? 1 : 0);
      f(c0, lc);
      c0 += lc;
    }
  }
}
Plan chunk_plan(const std::vector<int> &starts, int R) {
  Plan p{0, 0, 12L * R + 40};
  for_each_chunk(starts, [&](int, int lc) {
    ++p.chunks;
    p.recs += (lc + 4) / 4;
    p.cost += chunk_cost(lc, R);
  });
  return p;
}

}  // namespace

// the expansion's sheared tile: 2 n - 1 diagonals of n + 2 floats
static size_t expand_smem_bytes(int n) { return sizeof(float) * (size_t)(2 * n - 1) * (n + 2); }

bool disp_expand_fits(int n, int device) {
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) return false;
  return expand_smem_bytes(n) <= (size_t)optin;
}

size_t disp_smem_bytes(int n, int R) {
  const long rows = n + R;
  return sizeof(float) * (size_t)rows * disp_pitch(n, R) + 16;
}

namespace {

// The stencils and the sorted work units depend on n only, not on the
// medium: they are built once per (device, n) and shared by every handle of
// that size (kept after the last handle goes, at most kGeoKeep unused ones).
struct Geometry {
  int device = -1, n = 0, ldp = 0, global = 0, depth = 0, refs = 0;
  int4 *units = nullptr;
  float *stencil = nullptr;
  long long *doff = nullptr;  // first stored weight of each D (displacement-major storage)
  long n_units = 0;
  size_t stencil_bytes = 0;
  double taps = 0.0;
  double inv_r_sum = 0.0;  // sum over the nonzero displacements D of 1 / |D|
};
std::mutex g_geo_mu;
std::vector<Geometry *> g_geo;
constexpr int kGeoKeep = 4;

void geometry_free(Geometry *g) {
  if (g->units) vie_free(g->units);
  if (g->stencil) vie_free(g->stencil);
  if (g->doff) vie_free(g->doff);
  delete g;
}

// drop the oldest unused entries beyond kGeoKeep (caller holds g_geo_mu)
void geometry_trim() {
  int unused = 0;
  for (Geometry *g : g_geo) unused += g->refs == 0;
  for (size_t i = 0; i < g_geo.size() && unused > kGeoKeep;) {
    if (g_geo[i]->refs == 0) {
      geometry_free(g_geo[i]);
      g_geo.erase(g_geo.begin() + i);
      --unused;
    } else {
      ++i;
    }
  }
}

// global: the lattice-in-global-memory layout (runs along x address lat_t)
vie_status geometry_build(int n, int ldp, bool global, int R, Geometry *geo) {
  // stencils and work units, the run axis of each D chosen by estimated cost
  struct U {
    int4 u;
    long cost;
  };
  // first stored weight of each D, in the half plane's order
  std::vector<long long> doff;
  long long stored = 0;
  for (int dy = 0; dy < n; ++dy)
    for (int dx = -(n - 1); dx < n; ++dx) {
      if (dy == 0 && dx <= 0) continue;
      doff.push_back(stored);
      stored += (long long)(n - std::abs(dx)) * (n - dy);
    }
  // each row dy of displacements into its own lists (record offsets local to
  // the row), the rows spread over host threads, then joined in row order
  struct Row {
    std::vector<U> units;
    std::vector<float> rec;
    double taps = 0.0;
    vie_status s = VIE_OK;
  };
  std::vector<Row> rows(n);
  auto build_row = [&](int dy, Row &o) {
    std::vector<U> &units = o.units;
    std::vector<float> &rec = o.rec;
    double &taps = o.taps;
    std::vector<Cell> cy_cells, cx_cells;
    std::vector<int> cy_runs, cx_runs;
    for (int dx = -(n - 1); dx < n; ++dx) {
      if (dy == 0 && dx <= 0) continue;
      const int wx = n - std::abs(dx), wy = n - dy;
      stencil_cells(dx, dy, true, cy_cells);
      stencil_runs(cy_cells, true, cy_runs);
      stencil_cells(dx, dy, false, cx_cells);
      stencil_runs(cx_cells, false, cx_runs);
      const Plan py = chunk_plan(cy_runs, R), px = chunk_plan(cx_runs, R);
      const bool along_y = axis_cost(py, wx, wy, R) <= axis_cost(px, wy, wx, R);
      const std::vector<Cell> &cells = along_y ? cy_cells : cx_cells;
      taps += (double)cells.size() * wx * wy;
      const std::vector<int> &runs = along_y ? cy_runs : cx_runs;
      const Plan &pl = along_y ? py : px;
      const int off = (int)(rec.size() / 4);
      // header: chunks per length (16 bits per length 1..8), then the chunks
      // grouped by length, each group in run order
      unsigned counts[4] = {0u, 0u, 0u, 0u};
      for_each_chunk(runs, [&](int, int lc) { counts[(lc - 1) >> 1] += 1u << (16 * ((lc - 1) & 1)); });
      float hbits[4];
      memcpy(hbits, counts, sizeof hbits);
      for (float f : hbits) rec.push_back(f);
      for (int len = 1; len <= kMaxChunk; ++len)
        for_each_chunk(runs, [&](int c0, int lc) {
          if (lc != len) return;
          const int eoff =
              global && !along_y ? cells[c0].cy + ldp * cells[c0].cx : cells[c0].cx + ldp * cells[c0].cy;
          float obits;
          memcpy(&obits, &eoff, sizeof obits);
          rec.push_back(obits);
          for (int i = 0; i < lc; ++i) rec.push_back((float)cells[c0 + i].w);
          for (int i = lc + 1; i < 4 * ((lc + 4) / 4); ++i) rec.push_back(0.f);
        });
      int per_len[kMaxChunk + 1] = {};
      for_each_chunk(runs, [&](int, int lc) { ++per_len[lc]; });
      if (*std::max_element(per_len, per_len + kMaxChunk + 1) > 65535 || pl.recs + 1 > 524287) {
        o.s = VIE_ERR_UNSUPPORTED;
        return;
      }
      const int lanes = along_y ? wx : wy, stack = along_y ? wy : wx;
      // blocks of R stacked targets (the last one ragged); a unit carries
      // its first row (offset along the stack)
      const int nfb = (stack + R - 1) / R, full = lanes / 32, rem = lanes % 32;
      const int w = (along_y ? 1 : 0) | ((int)(pl.recs + 1) << 12);
      const int dxy = (dx & 0xffff) | (dy << 16);
      for (int sb = 0; sb < nfb; ++sb)
        for (int lb = 0; lb < full; ++lb)
          units.push_back({make_int4(off, dxy, lb | ((R * sb) << 16), w), pl.cost});
      if (rem > 0) {
        // the ragged last lane block: 2 or 4 blocks share a warp when it
        // is at most 16 or 8 lanes wide (blocks sb, sb + s, ...; s =
        // group_stride, as the kernel reads it)
        const int lg = rem <= 8 ? 2 : rem <= 16 ? 1 : 0, G = 1 << lg;
        const int sstride = group_stride(R, lg);
        const int span = lg == 0 ? 1 : G * sstride;
        for (int base = 0; base < nfb; base += span)
          for (int j = 0; j < (lg == 0 ? 1 : sstride) && base + j < nfb; ++j)
            units.push_back({make_int4(off, dxy, full | ((R * (base + j)) << 16), w | (lg << 1)), pl.cost});
      }
    }
  };
  {
    const int nt = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t)
      pool.emplace_back([&, t]() {
        for (int dy = t; dy < n; dy += nt) build_row(dy, rows[dy]);
      });
    for (std::thread &th : pool) th.join();
  }
  std::vector<U> units;
  std::vector<float> rec;
  double taps = 0.0;
  for (int dy = 0; dy < n; ++dy) {
    Row &o = rows[dy];
    if (o.s != VIE_OK) {
      set_error("displacement kernel: stencil longer than the unit encoding allows");
      return o.s;
    }
    const int base = (int)(rec.size() / 4);
    for (U u : o.units) {
      u.u.x += base;
      units.push_back(u);
    }
    rec.insert(rec.end(), o.rec.begin(), o.rec.end());
    taps += o.taps;
    std::vector<U>().swap(o.units);
    std::vector<float>().swap(o.rec);
  }
  for (int i = 0; i < 32; ++i) rec.push_back(0.f);  // the L1 prefetch may reach 127 bytes past a stencil
  std::stable_sort(units.begin(), units.end(), [](const U &p, const U &q) { return p.cost > q.cost; });
  std::vector<int4> uv(units.size());
  for (size_t i = 0; i < units.size(); ++i) uv[i] = units[i].u;
  VIE_CUDA(vie_malloc((void **)&geo->units, sizeof(int4) * uv.size()));
  VIE_CUDA(cudaMemcpy(geo->units, uv.data(), sizeof(int4) * uv.size(), cudaMemcpyHostToDevice));
  VIE_CUDA(vie_malloc((void **)&geo->stencil, sizeof(float) * rec.size()));
  VIE_CUDA(cudaMemcpy(geo->stencil, rec.data(), sizeof(float) * rec.size(), cudaMemcpyHostToDevice));
  VIE_CUDA(vie_malloc((void **)&geo->doff, sizeof(long long) * doff.size()));
  VIE_CUDA(cudaMemcpy(geo->doff, doff.data(), sizeof(long long) * doff.size(), cudaMemcpyHostToDevice));
  geo->n_units = (long)uv.size();
  double rb = 0.0;
  for (int dy = -(n - 1); dy < n; ++dy)
    for (int dx = -(n - 1); dx < n; ++dx)
      if (dx || dy) rb += 1.0 / sqrt((double)dx * dx + (double)dy * dy);
  geo->inv_r_sum = rb;
  geo->stencil_bytes = sizeof(float) * rec.size();
  geo->taps = taps;
  return VIE_OK;
}

vie_status geometry_acquire(int device, int n, int ldp, bool global, int R, Geometry **out) {
  std::lock_guard<std::mutex> lock(g_geo_mu);
  for (Geometry *g : g_geo)
    if (g->device == device && g->n == n && g->ldp == ldp && g->global == (int)global && g->depth == R) {
      ++g->refs;
      *out = g;
      return VIE_OK;
    }
  Geometry *g = new Geometry;
  g->device = device;
  g->n = n;
  g->ldp = ldp;
  g->global = global;
  g->depth = R;
  const vie_status s = geometry_build(n, ldp, global, R, g);
  if (s != VIE_OK) {
    geometry_free(g);
    return s;
  }
  g->refs = 1;
  g_geo.push_back(g);
  geometry_trim();
  *out = g;
  return VIE_OK;
}

void geometry_release(Geometry *g) {
  std::lock_guard<std::mutex> lock(g_geo_mu);
  --g->refs;
  geometry_trim();
}

}  // namespace

// Integral of 1/|z| over the unit square centred at (t1, t2).  The function
// P(u, v) = u asinh(v / |u|) + v asinh(u / |v|) (0 where u or v is 0) has
// d2P/dudv = 1 / sqrt(u^2 + v^2) and is odd in u and in v, so the integral is
// the signed sum of P over the square's corners: the closed form of Remark
// REM: NEW KERNEL (its F written with asinh), in FP64.
double unit_cell_integral(double t1, double t2) {
  auto P = [](double u, double v) {
    if (u == 0.0 || v == 0.0) return 0.0;
    return u * asinh(v / fabs(u)) + v * asinh(u / fabs(v));
  };
  double acc = 0.0;
  for (int a = -1; a <= 1; a += 2)
    for (int b = -1; b <= 1; b += 2) acc += a * b * P(t1 + 0.5 * a, t2 + 0.5 * b);
  return acc;
}

vie_status disp_mii_prepare(DispPlan *dp, int n, double *diag_value, cudaStream_t st) {
  // per D of the half plane in disp_index order: dy = 0, dx = 1 .. n - 1;
  // then dy = 1 .. n - 1, dx = -(n - 1) .. n - 1.  A_jk = e^{-tau} times
  // (h / 2 pi) G(D), G the unit-cell integral (it scales with h).
  const double hh = 1.0 / n, c = hh / (2.0 * kPi);
  std::vector<float> tab;
  tab.reserve((size_t)(n - 1) + (size_t)(n - 1) * (2 * n - 1));
  double rb = 0.0;  // bound on every row sum: all nonzero D of the full plane
  for (int dx = 1; dx < n; ++dx) tab.push_back((float)(c * unit_cell_integral(dx, 0)));
  for (int dy = 1; dy < n; ++dy)
    for (int dx = -(n - 1); dx < n; ++dx) tab.push_back((float)(c * unit_cell_integral(dx, dy)));
  for (int dy = -(n - 1); dy < n; ++dy)
    for (int dx = -(n - 1); dx < n; ++dx)
      if (dx || dy) rb += c * unit_cell_integral(dx, dy);
  *diag_value = c * unit_cell_integral(0.0, 0.0);
  if (dp->wtab) vie_free((void *)dp->wtab);
  dp->wtab = nullptr;
  float *d = nullptr;
  VIE_CUDA(vie_malloc((void **)&d, sizeof(float) * tab.size()));
  dp->wtab = d;
  VIE_CUDA(cudaMemcpyAsync(d, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice, st));
  VIE_CUDA(cudaStreamSynchronize(st));
  dp->rbound = std::max(dp->rbound, rb);
  return VIE_OK;
}

vie_status disp_prepare(DispPlan *dp, int n, const float *sig_padded, int device, cudaStream_t st) {
  dp->usable = 0;
  if (n < 2 || n > 4096) return VIE_OK;
  DevProps prop;
  VIE_TRY(get_dev_props(device, &prop));
  // the lattice in shared memory where it fits (with the smaller stack
  // depth's padding, if only that fits), else (n <= kGlobalMaxN) in global
  // memory, read through L1
  const size_t optin = (size_t)prop.sharedMemPerBlockOptin;
  int R = disp_depth(n);
  if (disp_smem_bytes(n, R) > optin && disp_smem_bytes(n, 8) <= optin) R = 8;
  const bool global = disp_smem_bytes(n, R) > optin;
  if (global && n > kGlobalMaxN) return VIE_OK;
  const int ldp = disp_pitch(global ? kGlobalMaxN : n, R), rows = global ? ldp : n + R;
  const size_t smem = global ? 16 : disp_smem_bytes(n, R);
  DispKernel k = global ? (R == 8 ? k_pairs_disp_global<8> : k_pairs_disp_global<12>) : pick_disp(ldp, R, false);
  DispKernel ks = global ? (R == 8 ? k_store_disp_global<8> : k_store_disp_global<12>) : pick_disp(ldp, R, true);
  DispKernel kst = R == 8 ? k_stream_disp<8> : k_stream_disp<12>;
  VIE_TRY(raise_smem_limit((const void *)k, (size_t)((int)smem)));
  if (global) {
    // all of the SM's unified memory it can get as L1 (a per-kernel preference)
    VIE_CUDA(cudaFuncSetAttribute((const void *)k, cudaFuncAttributePreferredSharedMemoryCarveout, 0));
    VIE_CUDA(cudaFuncSetAttribute((const void *)ks, cudaFuncAttributePreferredSharedMemoryCarveout, 0));
  }
  int bps = 0;
  VIE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, kThreads, smem));
  if (bps < 1) return VIE_OK;
  // the store and stream kernels of the displacement-major operator
  const long N = (long)n * n;
  const size_t smem_store = global ? 16 : sizeof(float) * (size_t)rows * ldp + 16;
  const size_t smem_stream = 16;
  VIE_TRY(raise_smem_limit((const void *)ks, (size_t)((int)smem_store)));
  VIE_TRY(raise_smem_limit((const void *)kst, (size_t)((int)smem_stream)));
  int bps_store = 0, bps_stream = 0;
  VIE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps_store, ks, kThreads, smem_store));
  VIE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps_stream, kst, kThreads, smem_stream));
  if (bps_store < 1 || bps_stream < 1) return VIE_OK;
  Geometry *geo = nullptr;
  vie_status s = geometry_acquire(device, n, ldp, global, R, &geo);
  if (s != VIE_OK) return s;
  dp->geometry = geo;
  dp->doff = geo->doff;
  dp->units = geo->units;
  dp->stencil = geo->stencil;
  dp->n_units = geo->n_units;
  dp->taps = geo->taps;
  dp->stencil_bytes = geo->stencil_bytes;
  VIE_CUDA(vie_malloc((void **)&dp->counter, 2 * sizeof(int)));
  VIE_CUDA(cudaMemset(dp->counter, 0, 2 * sizeof(int)));
  const long lat_elems = (long)rows * ldp;
  VIE_CUDA(vie_malloc((void **)&dp->lattice, sizeof(float) * lat_elems));
  k_make_lattice<<<(int)std::min((lat_elems + 255) / 256, 4096L), 256, 0, st>>>(n, sig_padded, rows, ldp, 0,
                                                                                (float *)dp->lattice);
  VIE_CHECK_LAUNCH("k_make_lattice");
  if (global) {
    VIE_CUDA(vie_malloc((void **)&dp->lattice_t, sizeof(float) * lat_elems));
    k_make_lattice<<<(int)std::min((lat_elems + 255) / 256, 4096L), 256, 0, st>>>(n, sig_padded, rows, ldp, 1,
                                                                                  (float *)dp->lattice_t);
    VIE_CHECK_LAUNCH("k_make_lattice");
  }
  dp->global = global;
  VIE_CUDA(vie_malloc((void **)&dp->smax, sizeof(unsigned)));
  VIE_CUDA(cudaMemset(dp->smax, 0, sizeof(unsigned)));
  VIE_CUDA(vie_malloc((void **)&dp->scale, sizeof(double)));
  VIE_CUDA(vie_malloc((void **)&dp->src_t, sizeof(float) * (size_t)n * n));
  VIE_CUDA(vie_malloc((void **)&dp->ss32, sizeof(float) * (size_t)n * n));
  VIE_CUDA(vie_malloc((void **)&dp->yacc, sizeof(unsigned long long) * 2 * (size_t)n * n));
  VIE_CUDA(cudaMemset(dp->yacc, 0, sizeof(unsigned long long) * 2 * (size_t)n * n));
  // every row sum of A is below sum over all nonzero displacements of
  // h / (2 pi r) (the sum of 1 / |D| is kept with the geometry)
  dp->rbound = geo->inv_r_sum / (2.0 * kPi * n);
  dp->n = n;
  dp->lat_elems = lat_elems;
  dp->ldp = ldp;
  dp->smem = smem;
  dp->grid = bps * prop.multiProcessorCount;
  dp->kernel = (const void *)k;
  dp->kernel_store = (const void *)ks;
  dp->smem_store = smem_store;
  dp->grid_store = bps_store * prop.multiProcessorCount;
  dp->kernel_stream = (const void *)kst;
  dp->smem_stream = smem_stream;
  dp->grid_stream = std::min(bps_stream * prop.multiProcessorCount, dp->grid);
  dp->stored = N * (N - 1) / 2;
  dp->usable = 1;
  return VIE_OK;
}

void disp_release(DispPlan *dp) {
  if (dp->geometry) geometry_release((Geometry *)dp->geometry);
  if (dp->counter) vie_free(dp->counter);
  if (dp->lattice) vie_free(dp->lattice);
  if (dp->lattice_t) vie_free(dp->lattice_t);
  if (dp->smax) vie_free(dp->smax);
  if (dp->scale) vie_free(dp->scale);
  if (dp->src_t) vie_free(dp->src_t);
  if (dp->ss32) vie_free(dp->ss32);
  if (dp->yacc) vie_free(dp->yacc);
  if (dp->wtab) vie_free((void *)dp->wtab);
  dp->wtab = nullptr;
  dp->yacc = nullptr;
  dp->ss32 = nullptr;
  dp->geometry = nullptr;
  dp->src_t = nullptr;
  dp->smax = nullptr;
  dp->scale = nullptr;
  dp->units = nullptr;
  dp->stencil = nullptr;
  dp->doff = nullptr;
  dp->counter = nullptr;
  dp->lattice = nullptr;
  dp->lattice_t = nullptr;
  dp->global = 0;
  dp->usable = 0;
}

vie_status disp_source(const DispPlan &dp, long N, int op, const double *sigma_s, const double *g,
                       float *src, cudaStream_t st) {
  const int blocks = (int)std::min((N + 255) / 256, 1024L);
  k_disp_source<<<blocks, 256, 0, st>>>(N, dp.n, op, sigma_s, g, src, dp.src_t, dp.smax);
  VIE_CHECK_LAUNCH("k_disp_source");
  return VIE_OK;
}

vie_status disp_expand(const DispPlan &dp, int n, const float *wbuf, const double *sigma_s, const double *diag,
                       long ldk, float *k32, void *khi, void *klo, int device, cudaStream_t st) {
  const long N = (long)n * n;
  const size_t esz = k32 ? sizeof(float) : sizeof(__nv_bfloat16);
  if (ldk > N) {  // dense K (ldk = 0: symmetric blocks)
    // zero the padding columns [N, ldk) of every row
    if (k32) VIE_CUDA(cudaMemset2DAsync(k32 + N, ldk * esz, 0, (ldk - N) * esz, N, st));
    if (khi) {
      VIE_CUDA(cudaMemset2DAsync((__nv_bfloat16 *)khi + N, ldk * esz, 0, (ldk - N) * esz, N, st));
      VIE_CUDA(cudaMemset2DAsync((__nv_bfloat16 *)klo + N, ldk * esz, 0, (ldk - N) * esz, N, st));
    }
  }
  DevProps prop;
  VIE_TRY(get_dev_props(device, &prop));
  const size_t smem = expand_smem_bytes(n);
  if (smem > (size_t)prop.sharedMemPerBlockOptin) {
    set_error("vie_assemble: grid too large for the pair-weight expansion");
    return VIE_ERR_UNSUPPORTED;
  }
  const int out = ldk == 0 ? kSymBlocks : k32 ? kDenseF32 : kDenseBF16;
  const void *kx = out == kSymBlocks  ? (const void *)k_expand_pairs<kSymBlocks>
                   : out == kDenseF32 ? (const void *)k_expand_pairs<kDenseF32>
                                      : (const void *)k_expand_pairs<kDenseBF16>;
  VIE_TRY(raise_smem_limit(kx, (size_t)((int)smem)));
  k_to_f32<<<(int)std::min((N + 255) / 256, 1024L), 256, 0, st>>>(N, sigma_s, dp.ss32);
  VIE_CHECK_LAUNCH("k_to_f32");
  const int grid = prop.multiProcessorCount;
  if (out == kSymBlocks)
    k_expand_pairs<kSymBlocks><<<grid, 1024, smem, st>>>(n, wbuf, dp.doff, dp.ss32, diag, sigma_s, 0, k32, nullptr,
                                                         nullptr);
  else if (out == kDenseF32)
    k_expand_pairs<kDenseF32><<<grid, 1024, smem, st>>>(n, wbuf, dp.doff, dp.ss32, diag, sigma_s, ldk, k32,
                                                        nullptr, nullptr);
  else
    k_expand_pairs<kDenseBF16><<<grid, 1024, smem, st>>>(n, wbuf, dp.doff, dp.ss32, diag, sigma_s, ldk, nullptr,
                                                         (unsigned short *)khi, (unsigned short *)klo);
  VIE_CHECK_LAUNCH("k_expand_pairs");
  return VIE_OK;
}

int symv_max_n() { return 32 * kSymvCols; }
size_t symv_block_floats(int n) { return (size_t)n * (n + 1) / 2 * n * n; }
size_t symv_partial_floats(int n) { return (size_t)n * (n + 1) / 2 * 2 * n; }

vie_status symv_apply(int n, int op, const double *sigma_s, const double *g, const float *blocks, float *s,
                      float *partial, double *y, int device, cudaStream_t st) {
  if (n > 32 * kSymvCols) {
    set_error("symmetric blocks: n too large");
    return VIE_ERR_UNSUPPORTED;
  }
  const long N = (long)n * n;
  DevProps prop;
  VIE_TRY(get_dev_props(device, &prop));
  k_symv_source<<<(int)std::min((N + 255) / 256, 1024L), 256, 0, st>>>(N, op, sigma_s, g, s);
  VIE_CHECK_LAUNCH("k_symv_source");
  const int items = n * (n + 1) / 2;
  k_symv_blocks<<<std::min(items, 8 * prop.multiProcessorCount), 256, 0, st>>>(n, blocks, s, partial);
  VIE_CHECK_LAUNCH("k_symv_blocks");
  k_symv_reduce<<<(int)std::min((N + 63) / 64, 4096L), 256, 0, st>>>(n, op, partial, g, y);
  VIE_CHECK_LAUNCH("k_symv_reduce");
  return VIE_OK;
}

vie_status disp_reduce(const DispPlan &dp, long N, int op, const double *diag, const double *sigma_s,
                       const double *g, double *y, cudaStream_t st) {
  const int blocks = (int)std::min((N + 255) / 256, 4096L);
  k_disp_reduce<<<blocks, 256, 0, st>>>(N, dp.n, op, (unsigned long long *)dp.yacc, dp.scale, diag, sigma_s,
                                        g, y);
  VIE_CHECK_LAUNCH("k_disp_reduce");
  return VIE_OK;
}

namespace {

DispArgs disp_args(const DispPlan &dp, int n, float tau_scale2, float wcoef, const float *src, float *wbuf) {
  DispArgs a;
  a.lat = (const float *)dp.lattice;
  a.lat_t = (const float *)dp.lattice_t;
  a.stencil = (const float4 *)dp.stencil;
  a.src = src;
  a.src_t = dp.src_t;
  a.smax = dp.smax;
  a.scale_out = dp.scale;
  a.rbound = dp.rbound;
  a.yacc = (unsigned long long *)dp.yacc;
  a.units = (const int4 *)dp.units;
  a.counter = dp.counter;
  a.wbuf = wbuf;
  a.doff = dp.doff;
  a.wtab = dp.wtab;
  a.n_units = dp.n_units;
  a.n = n;
  a.ldp = dp.ldp;
  a.lat_elems = dp.lat_elems;
  a.tau_scale2 = tau_scale2;
  a.wcoef = wcoef;
  return a;
}

}  // namespace

vie_status disp_launch(const DispPlan &dp, int n, float tau_scale2, float wcoef, const float *src,
                       cudaStream_t st) {
  DispArgs a = disp_args(dp, n, tau_scale2, wcoef, src, nullptr);
  void *args[] = {&a};
  VIE_CUDA(cudaLaunchKernel(dp.kernel, dim3(dp.grid), dim3(kThreads), args, dp.smem, st));
  count_launch();
  return VIE_OK;
}

vie_status disp_store(const DispPlan &dp, int n, float tau_scale2, float wcoef, float *wbuf, cudaStream_t st) {
  DispArgs a = disp_args(dp, n, tau_scale2, wcoef, nullptr, wbuf);
  void *args[] = {&a};
  VIE_CUDA(cudaLaunchKernel(dp.kernel_store, dim3(dp.grid_store), dim3(kThreads), args, dp.smem_store, st));
  count_launch();
  return VIE_OK;
}

vie_status disp_stream(const DispPlan &dp, int n, const float *wbuf, const float *src, cudaStream_t st) {
  DispArgs a = disp_args(dp, n, 0.f, 0.f, src, const_cast<float *>(wbuf));
  void *args[] = {&a};
  VIE_CUDA(cudaLaunchKernel(dp.kernel_stream, dim3(dp.grid_stream), dim3(kThreads), args, dp.smem_stream, st));
  count_launch();
  return VIE_OK;
}

}  // namespace vie
