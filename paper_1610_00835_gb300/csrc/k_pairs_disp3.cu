// Displacement-major pair kernel in 3D (n <= 32, FP32 tiles, S = 64).
//
// The 3D form of k_pairs_disp.cu (Section 2, Eq. EQ:Kernel; Section 3.2,
// M-iii): y_j = sum_{k != j} A_jk s_k with A_jk = h^3 e^{-tau} / (4 pi r^2)
// and tau the S-step midpoint march of the trilinear interpolant of sigma_t.
// The S samples of the segment from j to j + D sit at (i + 1/2) D / S from j,
// so their trilinear weights, summed per lattice cell, give a stencil W_D with
// sum_i sigma(u_j + (i + 1/2) D / S) = sum_c W_D(c) sigma[j + c] for every j.
//
// W_D is stored as runs along one axis, each cut into the fewest chunks of at
// most 8 cells, of equal length, grouped by length behind a per-D header (the
// same records and packed-pair march as in 2D, disp_march.cuh).  Three orientations,
// chosen per D by estimated cost: runs along z with lanes on x (units fix a y),
// runs along y with lanes on x (units fix a z), runs along x with lanes on y
// (units fix a z).  A thread stacks kR targets along the run axis.  When the
// lane extent of D is below 32, a warp holds 32 / gw lane groups of width gw
// (gw the power of two at or above it) at third-axis coordinates gw apart:
// with the odd pitches n + 1 and (n + 1)^2 the groups fall in distinct banks.
//
// The lattice is the padded (n + 1)^3 sigma_t array, linear (x fastest), with
// kPad3 zero planes appended: reads of discarded stacked targets only run
// forward along the run axis, by at most kPad3 strides, so every read stays in
// shared memory.  The weights of valid
// targets only touch the (n + 1)^3 part.
//
// Only D in a half space is marched (A_jk = A_kj); each pair adds w s_k to y_j
// and w s_j to y_k in 64-bit fixed point (the scale of the 2D kernel) with
// integer atomics on global memory: exact, so applies are bitwise
// reproducible.  Runs along x put their sums in a second array with y fastest,
// so a warp's atomics always cover contiguous words.  k_disp3_reduce adds the
// two sums of each target, converts once, adds the self cell and clears both.
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

using dmarch::kMaxChunk;
using dmarch::kR;
using dmarch::march_runs;
using dmarch::red_add;
using march::kS;

constexpr int kThreads3 = 1024;
constexpr int kPad3 = kR - 1;  // zero planes after the lattice
constexpr int kMaxN3 = 32;                     // one lane block per unit

struct Disp3Args {
  const float *lat;          // [(n + 1 + kPad3) (n + 1)^2] sigma_t, x fastest
  const float4 *stencil;     // chunk records of every W_D
  const float *src;          // s, FP32 [N], x fastest
  const float *src_t;        // s with y fastest: s(x, y, z) = src_t[(z n + x) n + y]
  unsigned *smax;            // bits of max |s| (set by the source kernel)
  double *scale_out;         // fixed-point scale of this apply
  double rbound;             // bound on every row sum of A
  unsigned long long *yacc;  // [2 N] int64 sums (x fastest, then y fastest), zero between applies
  float *pairs;              // store mode: the weight of every unordered pair (displacement-major)
  const long long *doff;     // store mode: first stored weight of each D of the half space
  const int4 *units;         // see geometry3_build
  int *counter;              // [2]
  long n_units;
  int n, ldp, plane;
  long lat_elems;
  float tau_scale2, wcoef;
};

// STORE: instead of the apply's sums, write w = h^3 e^{-tau} / (4 pi r^2) of
// every pair (j, j + D) to pairs: per D of the half space its box of targets,
// x fastest, then y, then z.  A warp's stores are contiguous when its lanes
// run along x; for runs along x (lanes on y) they are strided, but the units
// of one D run back to back and L2 gathers its box before writing it out.
template <int LDP, int PLANE, bool STORE>
__global__ void __launch_bounds__(kThreads3, 1) k_pairs_disp3(Disp3Args a) {
  extern __shared__ float4 smem4[];
  float *lat = reinterpret_cast<float *>(smem4);
  const int tid = threadIdx.x, lane = tid & 31;
  {
    const float4 *g4 = reinterpret_cast<const float4 *>(a.lat);
    const long n4 = a.lat_elems / 4;
    for (long i = tid; i < n4; i += kThreads3) smem4[i] = g4[i];
    for (long i = n4 * 4 + tid; i < a.lat_elems; i += kThreads3) lat[i] = a.lat[i];
  }
  __syncthreads();
  double scale_d = 1.0;
  if constexpr (!STORE) {
    const float smax = __uint_as_float(*a.smax);
    if (smax > 0.f) scale_d = ldexp(1.0, ilogb(4.611686018427387904e18 / ((double)smax * a.rbound)));
  }
  const float scale = (float)scale_d;
  const int n = a.n;
  const int ldp = LDP > 0 ? LDP : a.ldp, plane = PLANE > 0 ? PLANE : a.plane;
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
    const int dx = (signed char)(un.y & 0xff), dy = (signed char)((un.y >> 8) & 0xff);
    const int dz = (signed char)((un.y >> 16) & 0xff);
    const int orient = (un.y >> 24) & 3, lg = (un.y >> 26) & 7;
    const int sb = un.z & 0xff, c3 = (un.z >> 8) & 0xff;
    const int nrec = un.w;
    const int xlo = max(0, -dx), xhi = n - max(0, dx);
    const int ylo = max(0, -dy), yhi = n - max(0, dy);
    const int zlo = max(0, -dz), zhi = n - max(0, dz);
    // lane, stack (run) and third axes of this orientation
    const int llo = orient == 2 ? ylo : xlo, lhi = orient == 2 ? yhi : xhi;
    const int slo = orient == 0 ? zlo : orient == 1 ? ylo : xlo;
    const int shi = orient == 0 ? zhi : orient == 1 ? yhi : xhi;
    const int thi = orient == 0 ? yhi : zhi;
    const int gw = 32 >> lg, g = lane >> (5 - lg), lig = lane & (gw - 1);
    int c = c3 + gw * g;
    bool lvalid = c < thi;
    if (!lvalid) c = c3;
    int la = llo + lig;
    lvalid = lvalid && la < lhi;
    la = min(la, lhi - 1);
    const int b0 = slo + kR * sb;
    int x, y, z;
    if (orient == 0) {
      x = la; z = b0; y = c;
    } else if (orient == 1) {
      x = la; y = b0; z = c;
    } else {
      y = la; x = b0; z = c;
    }
    const unsigned base = lat_base + 4u * (unsigned)(x + ldp * y + plane * z);
    {
      // bring this D's chunk records into L1 (one 128-byte line per lane)
      const char *r0 = reinterpret_cast<const char *>(a.stencil + un.x);
      const int lines = (int)(((reinterpret_cast<size_t>(r0) & 127) + 16L * nrec + 127) >> 7);
      for (int l = lane; l < lines; l += 32) asm volatile("prefetch.global.L1 [%0];" ::"l"(r0 + 128L * l));
    }
    float acc[kR];
#pragma unroll
    for (int q = 0; q < kR; ++q) acc[q] = 0.f;
    if (orient == 0)
      march_runs<PLANE, kR>(a.stencil + un.x, base, plane, acc);
    else if (orient == 1)
      march_runs<LDP, kR>(a.stencil + un.x, base, ldp, acc);
    else
      march_runs<1, kR>(a.stencil + un.x, base, 1, acc);
    const float r2 = (float)(dx * dx + dy * dy + dz * dz);
    const float inv_r = rsqrtf(r2);
    const float tscale = -a.tau_scale2 * r2 * inv_r;  // -(h/S) log2(e) r
    const float wk = a.wcoef * inv_r * inv_r;
    if constexpr (STORE) {
      const int m2 = 2 * n - 1;
      const long base = __ldg(a.doff + ((long)(dz + n - 1) * m2 + (dy + n - 1)) * m2 + (dx + n - 1));
      const long wx = xhi - xlo, wy = yhi - ylo;
      // the unit's first target in the box, and the stride of its stacked targets
      const long o0 = base + ((long)(z - zlo) * wy + (y - ylo)) * wx + (x - xlo);
      const long ostep = orient == 0 ? wx * wy : orient == 1 ? wx : 1;
#pragma unroll
      for (int q = 0; q < kR; ++q)
        if (lvalid && b0 + q < shi) __stcs(a.pairs + o0 + q * ostep, wk * exp2f(tscale * acc[q]));
      continue;
    }
    // targets and partners in the layout whose fastest axis carries the lanes:
    // x fastest (s, the first half of yacc) or, for runs along x, y fastest
    // (s_t, the second half), so the atomics of a warp hit contiguous words
    const long nn = (long)n * n;
    const bool ty = orient == 2;
    const float *sv = ty ? a.src_t : a.src;
    unsigned long long *ya = ty ? a.yacc + nn * n : a.yacc;
    const long j0 = ty ? ((long)z * n + x) * n + y : x + (long)n * (y + (long)n * z);
    const long jstep = orient == 0 ? nn : n;
    const long dk = ty ? dy + (long)n * (dx + (long)n * dz) : dx + (long)n * (dy + (long)n * dz);
#pragma unroll
    for (int q = 0; q < kR; ++q) {
      if (lvalid && b0 + q < shi) {
        const long j = j0 + q * jstep, k = j + dk;
        const float sj = __ldg(sv + j), sk = __ldg(sv + k);
        const float w = wk * exp2f(tscale * acc[q]) * scale;
        red_add(ya + j, (unsigned long long)__float2ll_rn(w * sk));
        red_add(ya + k, (unsigned long long)__float2ll_rn(w * sj));
      }
    }
  }
  __syncthreads();
  if (!STORE && blockIdx.x == 0 && tid == 0) *a.scale_out = scale_d;
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(a.counter + 1, 1) == (int)gridDim.x - 1) {
      a.counter[0] = 0;
      a.counter[1] = 0;
      if constexpr (!STORE) *a.smax = 0u;  // every CTA read it before this, the next source kernel sets it
      __threadfence();
    }
  }
}

// the padded lattice (pitch n + 1, x fastest) followed by kPad3 zero planes
__global__ void k_make_lattice3(long lat, long total, const float *__restrict__ pad, float *__restrict__ out) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x)
    out[i] = i < lat ? pad[i] : 0.f;
}

// s = sigma_s g (or g) in FP32, its copy with y fastest, and max |s|
__global__ void k_disp3_source(long N, int n, int op, const double *__restrict__ ss, const double *__restrict__ g,
                               float *__restrict__ s, float *__restrict__ s_t, unsigned *__restrict__ smax) {
  unsigned m = 0u;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    const float v = (float)(op == VIE_OP_A_RAW ? g[i] : ss[i] * g[i]);
    s[i] = v;
    const long x = i % n, y = (i / n) % n, z = i / ((long)n * n);
    s_t[(z * n + x) * n + y] = v;
    m = max(m, __float_as_uint(fabsf(v)));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(smax, m);
}

// y_j = (both sums of j) / scale + d_j s_j, and yacc back to zero.  yacc holds
// N sums with x fastest, then N with y fastest (the runs along x).
__global__ void k_disp3_reduce(long N, int n, int op, unsigned long long *__restrict__ yacc,
                               const double *__restrict__ scale, const double *__restrict__ diag,
                               const double *__restrict__ ss, const double *__restrict__ g,
                               double *__restrict__ y) {
  const double inv = 1.0 / *scale;
  for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < N; j += (long)gridDim.x * blockDim.x) {
    const long x = j % n, yy = (j / n) % n, z = j / ((long)n * n);
    const long jt = N + (z * n + x) * n + yy;
    const unsigned long long acc = yacc[j] + yacc[jt];
    yacc[j] = 0ull;
    yacc[jt] = 0ull;
    const double sj = op == VIE_OP_A_RAW ? g[j] : ss[j] * g[j];
    const double v = (double)(long long)acc * inv + diag[j] * sj;
    y[j] = op == VIE_OP_I_MINUS_K ? g[j] - v : v;
  }
}

// ---- the dense operator from the stored pair weights (the 3D form of
// k_expand_pairs): K_jk = A_jk sigma_s,k (j != k) and K_jj = d_j sigma_s,j,
// row-major N x ldk, FP32 or BF16 hi + lo (lo = bf16(v - hi)), each stored
// weight read once.  Grid lines (y, z) play the part of the 2D grid rows: an
// item is a line displacement (dy, dz) (dz > 0, or dz = 0 and dy >= 0) and a
// target line (yj, zj); the stored rows "D = (dx, dy, dz), targets (., yj,
// zj)" of every dx go to shared memory (T[dx + n - 1][xj]), then
//   K[j][k] = T sigma_s,k  for j = (xj, yj, zj), k = (xk, yj + dy, zj + dz),
//   K[k][j] = T sigma_s,j  for the same pairs seen from k,
// each written as whole row segments of n columns.  Every ordered pair is
// written once: from its own line displacement when that is in the half
// plane, else from the opposite one.  For (dy, dz) = (0, 0) the line of j
// gets its columns k > j from the first part and k < j from the second, and
// the diagonal.
constexpr int kExpF32 = 0, kExpBF16 = 1, kExpSym = 2;  // kExpSym: A in the n x n blocks of the items
// small CTAs, several per SM: an item is small (2 n^2 entries), and one CTA's
// barriers then leave the SM to the others
constexpr int kExpThreads = 256, kExpWarps = kExpThreads / 32;
constexpr int kExpRows = (2 * kMaxN3 - 1 + kExpWarps - 1) / kExpWarps;  // T rows per warp

template <int OUT>
__device__ __forceinline__ void put_k(long idx, float v, float *k32, unsigned short *khi, unsigned short *klo) {
  if constexpr (OUT == kExpBF16) {
    const unsigned short hi = bf16_bits_rn(v);
    khi[idx] = hi;
    klo[idx] = bf16_bits_rn(v - __uint_as_float((unsigned)hi << 16));
  } else {
    k32[idx] = v;
  }
}

// items: ioff[q] = first item of line displacement q (q < nq; ioff[nq] = the
// total), iqd[q] = dy | dz << 16 (dy as a signed 16-bit value)
struct ExpItem {
  int dy, dz, yj, zj, ylo, wyl;
  bool same;  // (dy, dz) = (0, 0): one grid line
  long jrow, krow;
};

__device__ __forceinline__ ExpItem exp_decode(int t, int n, const int *__restrict__ ioff,
                                              const int *__restrict__ iqd, int nq) {
  int lo = 0, hi = nq - 1;  // the last q with ioff[q] <= t
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ioff[mid] <= t) lo = mid; else hi = mid - 1;
  }
  const int qd = iqd[lo];
  ExpItem it;
  it.dy = (short)(qd & 0xffff);
  it.dz = qd >> 16;
  it.ylo = it.dy < 0 ? -it.dy : 0;
  it.wyl = n - (it.dy < 0 ? -it.dy : it.dy);
  const int local = t - ioff[lo];
  it.yj = it.ylo + local % it.wyl;
  it.zj = local / it.wyl;
  it.same = it.dy == 0 && it.dz == 0;
  it.jrow = (long)n * (it.yj + (long)n * it.zj);
  it.krow = (long)n * (it.yj + it.dy + (long)n * (it.zj + it.dz));
  return it;
}

// row i of this warp holds dx = -(n - 1) + warp + i kExpWarps (lane = xj - xlo)
__device__ __forceinline__ bool exp_row(const ExpItem &it, int n, int warp, int i, int lane, int &dx, int &xlo,
                                        int &wx) {
  dx = -(n - 1) + warp + i * kExpWarps;
  xlo = dx < 0 ? -dx : 0;
  wx = n - (dx < 0 ? -dx : dx);
  return dx < n && !(it.same && dx <= 0) && lane < wx;
}

// this warp's stored rows of item it into v, and the lane's sigma_s on both lines
__device__ __forceinline__ void exp_load(const ExpItem &it, int n, int warp, int lane, const float *__restrict__ w,
                                         const long long *__restrict__ doff, const float *__restrict__ ss,
                                         float (&v)[kExpRows], float &ssj, float &ssk) {
  const int m2 = 2 * n - 1;
#pragma unroll
  for (int i = 0; i < kExpRows; ++i) {
    int dx, xlo, wx;
    v[i] = 0.f;
    if (exp_row(it, n, warp, i, lane, dx, xlo, wx))
      v[i] = __ldcs(w + doff[((long)(it.dz + n - 1) * m2 + (it.dy + n - 1)) * m2 + (dx + n - 1)] +
                    ((long)it.zj * it.wyl + (it.yj - it.ylo)) * wx + lane);
  }
  ssj = lane < n ? __ldg(ss + it.jrow + lane) : 0.f;  // n <= 32: one column per lane
  ssk = lane < n ? __ldg(ss + it.krow + lane) : 0.f;
}

// Software-pipelined: while a CTA writes the K entries of one item, the row
// loads of its next item are in flight.
template <int OUT>
__global__ void __launch_bounds__(kExpThreads, 4) k_expand_pairs3(int n, const float *__restrict__ w,
                                                           const long long *__restrict__ doff,
                                                           const int *__restrict__ ioff, const int *__restrict__ iqd,
                                                           int nq, const float *__restrict__ ss,
                                                           const double *__restrict__ diag,
                                                           const double *__restrict__ ss64, long ldk, float *k32,
                                                           unsigned short *khi, unsigned short *klo) {
  extern __shared__ float T[];  // [2n - 1][p]
  const int p = n + 2;           // strides p and 1 - p: at most one is even (2-way conflicts)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;  // blockDim.x = kExpThreads
  const int items = ioff[nq];
  int t = blockIdx.x;
  if (t >= items) return;
  ExpItem cur = exp_decode(t, n, ioff, iqd, nq);
  float v[kExpRows], ssj_n, ssk_n;
  exp_load(cur, n, warp, lane, w, doff, ss, v, ssj_n, ssk_n);
  for (; t < items; t += gridDim.x) {
#pragma unroll
    for (int i = 0; i < kExpRows; ++i) {
      int dx, xlo, wx;
      if (exp_row(cur, n, warp, i, lane, dx, xlo, wx)) T[(dx + n - 1) * p + xlo + lane] = v[i];
    }
    const float ssj_l = ssj_n, ssk_l = ssk_n;
    __syncthreads();
    ExpItem nxt = cur;
    const int tn = t + gridDim.x;
    if (tn < items) {
      nxt = exp_decode(tn, n, ioff, iqd, nq);
      exp_load(nxt, n, warp, lane, w, doff, ss, v, ssj_n, ssk_n);
    }
    const long jrow = cur.jrow, krow = cur.krow;
    if constexpr (OUT == kExpSym) {
      // block t: A_jk for j on line (yj, zj) (row xj), k on line (yk, zk)
      // (column xk); no sigma_s; the one-line blocks whole, with d_j
      float *blk = k32 + (long)t * n * n;
      for (int xj = warp; xj < n; xj += kExpWarps) {
        const int xk = lane;
        if (xk < n) {
          const int dx = xk - xj;
          float tv;
          if (!cur.same || dx > 0)
            tv = T[(dx + n - 1) * p + xj];
          else if (dx < 0)
            tv = T[(-dx + n - 1) * p + xk];  // A_jk = A_kj, stored under (-dx, 0, 0) for target xk
          else
            tv = (float)diag[jrow + xj];
          blk[(long)xj * n + xk] = tv;
        }
      }
    } else if (!cur.same) {
      for (int xj = warp; xj < n; xj += kExpWarps) {
        const float *tb = T + (n - 1 - xj) * p + xj;  // T[(xk - xj + n - 1) p + xj]
        const long rb = (jrow + xj) * ldk + krow;
        if (lane < n) put_k<OUT>(rb + lane, tb[lane * p] * ssk_l, k32, khi, klo);
      }
      for (int xk = warp; xk < n; xk += kExpWarps) {
        const float *tb = T + (xk + n - 1) * p;  // T[(xk - xj + n - 1) p + xj]
        const long rb = (krow + xk) * ldk + jrow;
        if (lane < n) put_k<OUT>(rb + lane, tb[lane * (1 - p)] * ssj_l, k32, khi, klo);
      }
    } else {
      for (int r = warp; r < n; r += kExpWarps) {
        const long rb = (jrow + r) * ldk + jrow;
        const int x = lane;
        if (x < n && x != r) {
          const float tv = x > r ? T[(x - r + n - 1) * p + r] : T[(r - x + n - 1) * p + x];
          put_k<OUT>(rb + x, tv * ssj_l, k32, khi, klo);
        }
      }
      for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const long j = jrow + r;
        put_k<OUT>(j * ldk + j, (float)(diag[j] * ss64[j]), k32, khi, klo);
      }
    }
    __syncthreads();
    cur = nxt;
  }
}

// ---- applies of A stored in the expansion's blocks (kExpSym)
//
// y = A s with s = sigma_s g (or g).  k_symv3_blocks: one warp per block t
// (item (dy, dz) and target line Lj; Lk = Lj + (dy, dz)) stages the block in
// shared memory and writes P[t][0, n) = its row sums against s on Lk and, for
// (dy, dz) != 0, P[t][n, 2n) = its column sums against s on Lj (A_kj = A_jk);
// all sums in a fixed order.  k_symv3_reduce: one CTA per grid line adds, for
// each target, the partials of every block that touches its line.
constexpr int kSymvWarps3 = 8;

__global__ void __launch_bounds__(32 * kSymvWarps3, 4) k_symv3_blocks(int n, const float *__restrict__ A,
                                                                   const float *__restrict__ s,
                                                                   const int *__restrict__ ioff,
                                                                   const int *__restrict__ iqd, int nq,
                                                                   float *__restrict__ P) {
  __shared__ float tile[kSymvWarps3][32][33];
  __shared__ float sjs[kSymvWarps3][32], sks[kSymvWarps3][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int items = ioff[nq];
  float(*tl)[33] = tile[warp];
  for (int t = blockIdx.x * kSymvWarps3 + warp; t < items; t += gridDim.x * kSymvWarps3) {
    const ExpItem it = exp_decode(t, n, ioff, iqd, nq);
    const float *blk = A + (long)t * n * n;
    float v[32];
#pragma unroll
    for (int xj = 0; xj < 32; ++xj) v[xj] = (xj < n && lane < n) ? __ldcs(blk + (long)xj * n + lane) : 0.f;
    const float sj = lane < n ? s[it.jrow + lane] : 0.f, sk = lane < n ? s[it.krow + lane] : 0.f;
    // every load of the block issued before the first shared store
    asm volatile("" ::: "memory");
    sjs[warp][lane] = sj;
    sks[warp][lane] = sk;
#pragma unroll
    for (int xj = 0; xj < 32; ++xj) tl[xj][lane] = v[xj];
    __syncwarp();
    float r = 0.f, c = 0.f;
    for (int x = 0; x < n; ++x) {
      r = fmaf(tl[lane][x], sks[warp][x], r);  // row lane, column x
      c = fmaf(tl[x][lane], sjs[warp][x], c);  // row x, column lane
    }
    float *pt = P + (long)t * 2 * n;
    if (lane < n) {
      pt[lane] = r;
      if (!it.same) pt[n + lane] = c;
    }
    __syncwarp();
  }
}

// hi + lo += v: Knuth's error-free TwoSum on hi, the rounding error into lo
__device__ __forceinline__ void pair_add(float &hi, float &lo, float v) {
  const float s1 = __fadd_rn(hi, v);
  const float bv = __fsub_rn(s1, hi);
  lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s1, bv)), __fsub_rn(v, bv)));
  hi = s1;
}

// Per grid line L = blockIdx.x (y = L % n, z = L / n): warp w adds, for
// target x = lane, the partials of the line displacements q = w, w + 8, ...:
// the row sums of block (q, L) and then the column sums of block (q, L - q),
// as an FP32 hi + lo pair; the eight warps' pairs are then added in warp order.
__global__ void __launch_bounds__(32 * kSymvWarps3, 4) k_symv3_reduce(int n, int op, const float *__restrict__ P,
                                                                   const int *__restrict__ ioff,
                                                                   const int *__restrict__ iqd, int nq,
                                                                   const double *__restrict__ g,
                                                                   double *__restrict__ y) {
  __shared__ float hs[kSymvWarps3][32], ls[kSymvWarps3][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int L = blockIdx.x, yl = L % n, zl = L / n;
  float hi = 0.f, lo = 0.f;
  if (lane < n) {
    // kBatch displacements per step, their loads issued before the first add
    constexpr int kBatch = 8;
    for (int q0 = warp; q0 < nq; q0 += kBatch * kSymvWarps3) {
      float va[kBatch], vb[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int q = q0 + u * kSymvWarps3;
        va[u] = vb[u] = 0.f;
        if (q < nq) {
          const int qd = iqd[q];
          const int dy = (short)(qd & 0xffff), dz = qd >> 16;
          const int ylo = dy < 0 ? -dy : 0, wyl = n - (dy < 0 ? -dy : dy);
          // L as the target line of block q: L + (dy, dz) inside the grid
          const int yk = yl + dy, zk = zl + dz;
          if (yk >= 0 && yk < n && zk < n) va[u] = __ldcs(P + (ioff[q] + (long)zl * wyl + (yl - ylo)) * 2 * n + lane);
          // L as the source line: L - (dy, dz) inside the grid, (dy, dz) != 0
          const int yj = yl - dy, zj = zl - dz;
          if ((dy != 0 || dz != 0) && yj >= 0 && yj < n && zj >= 0)
            vb[u] = __ldcs(P + (ioff[q] + (long)zj * wyl + (yj - ylo)) * 2 * n + n + lane);
        }
      }
      asm volatile("" ::: "memory");  // the batch's loads issued before its first add
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        pair_add(hi, lo, va[u]);  // a missing block adds an exact zero
        pair_add(hi, lo, vb[u]);
      }
    }
  }
  hs[warp][lane] = hi;
  ls[warp][lane] = lo;
  __syncthreads();
  if (warp == 0 && lane < n) {
    hi = hs[0][lane];
    lo = ls[0][lane];
    for (int w = 1; w < kSymvWarps3; ++w) {
      pair_add(hi, lo, hs[w][lane]);
      lo = __fadd_rn(lo, ls[w][lane]);
    }
    const long j = (long)L * n + lane;
    const double v = (double)hi + (double)lo;
    y[j] = op == VIE_OP_I_MINUS_K ? g[j] - v : v;
  }
}

__global__ void k_symv3_source(long N, int op, const double *__restrict__ ss, const double *__restrict__ g,
                               float *__restrict__ s) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x)
    s[i] = (float)(op == VIE_OP_A_RAW ? g[i] : ss[i] * g[i]);
}

__global__ void k_to_f32_3(long N, const double *__restrict__ x, float *__restrict__ y) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

typedef void (*Disp3Kernel)(Disp3Args);

Disp3Kernel pick_disp3(int n, bool store = false) {
  if (store) return n == 32 ? k_pairs_disp3<33, 1089, true> : k_pairs_disp3<0, 0, true>;
  return n == 32 ? k_pairs_disp3<33, 1089, false> : k_pairs_disp3<0, 0, false>;
}

// ---- geometry (host): stencils, chunk records and work units, per (device, n)

struct Run3 {
  int cx, cy, cz, len, woff;  // first cell, cells, first weight in the shared weight list
};

// W_D on its box of cells [min(0, d), max(0, d)] per axis: the trilinear
// weights of the S midpoint samples (i + 1/2) D / S summed per cell (Section
// 3.2, M-iii), cells of zero weight excluded from the runs
void stencil3(int dx, int dy, int dz, std::vector<double> &box, int &ox, int &oy, int &oz, int &bx, int &by,
              int &bz) {
  ox = std::min(0, dx), oy = std::min(0, dy), oz = std::min(0, dz);
  bx = std::abs(dx) + 1, by = std::abs(dy) + 1, bz = std::abs(dz) + 1;
  box.assign((size_t)bx * by * bz, 0.0);
  for (int i = 0; i < kS; ++i) {
    const double px = (i + 0.5) * dx / kS, py = (i + 0.5) * dy / kS, pz = (i + 0.5) * dz / kS;
    const double fx = floor(px), fy = floor(py), fz = floor(pz);
    const double ax = px - fx, ay = py - fy, az = pz - fz;
    for (int c = 0; c < 8; ++c) {
      const double w = (c & 1 ? ax : 1.0 - ax) * (c & 2 ? ay : 1.0 - ay) * (c & 4 ? az : 1.0 - az);
      if (w == 0.0) continue;
      const int cx = (int)fx + (c & 1) - ox, cy = (int)fy + ((c >> 1) & 1) - oy, cz = (int)fz + (c >> 2) - oz;
      box[((size_t)cz * by + cy) * bx + cx] += w;
    }
  }
}

// runs of nonzero cells along axis ax (0 x, 1 y, 2 z) of the box
void box_runs(const std::vector<double> &box, int ox, int oy, int oz, int bx, int by, int bz, int ax,
              std::vector<Run3> &runs, std::vector<double> &wts) {
  runs.clear();
  wts.clear();
  const int ext[3] = {bx, by, bz};
  const int a1 = ax == 0 ? 1 : 0, a2 = ax == 2 ? 1 : 2;  // the two other axes
  int p[3];
  for (p[a2] = 0; p[a2] < ext[a2]; ++p[a2])
    for (p[a1] = 0; p[a1] < ext[a1]; ++p[a1]) {
      bool open = false;
      for (p[ax] = 0; p[ax] < ext[ax]; ++p[ax]) {
        const double w = box[((size_t)p[2] * by + p[1]) * bx + p[0]];
        if (w != 0.0) {
          if (!open) {
            runs.push_back({p[0] + ox, p[1] + oy, p[2] + oz, 0, (int)wts.size()});
            open = true;
          }
          wts.push_back(w);
          runs.back().len++;
        } else {
          open = false;
        }
      }
    }
}

// A run of L cells is cut into ceil(L / kMaxChunk) chunks of equal length
// (lengths differ by at most one); f(first cell, length) per chunk.
template <typename F>
void for_each_chunk3(const std::vector<Run3> &runs, F f) {
  for (size_t r = 0; r < runs.size(); ++r) {
    const int L = runs[r].len, nch = (L + kMaxChunk - 1) / kMaxChunk;
    int c0 = 0;
    for (int c = 0; c < nch; ++c) {
      const int lc = L / nch + (c < L % nch ? 1 : 0);
      f(r, c0, lc);
      c0 += lc;
    }
  }
}

// Estimated instructions per thread of one unit (as in 2D): per chunk its
// record loads and loop, Lc + kR - 1 lattice loads, the packed multiply-adds
// and a weight broadcast per tap; per unit the epilogue.
struct Plan3 {
  long chunks, recs, cost;
};

Plan3 chunk_plan3(const std::vector<Run3> &runs) {
  Plan3 p{0, 1, 12L * kR + 40};
  for_each_chunk3(runs, [&](size_t, int, int lc) {
    ++p.chunks;
    p.recs += (lc + 4) / 4;
    p.cost += 4 + (lc + 4) / 4 + (lc + kR - 1) + ((lc + 1) / 2) * (kR / 2) + (lc / 2) * (kR / 2 + 1) + lc;
  });
  return p;
}

int pow2ceil(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

struct Geometry3 {
  int device = -1, n = 0, refs = 0;
  int4 *units = nullptr;
  float *stencil = nullptr;
  long n_units = 0;
  double taps = 0.0;
};
std::mutex g_geo3_mu;
std::vector<Geometry3 *> g_geo3;
constexpr int kGeo3Keep = 2;

void geometry3_free(Geometry3 *g) {
  if (g->units) vie_free(g->units);
  if (g->stencil) vie_free(g->stencil);
  delete g;
}

void geometry3_trim() {
  int unused = 0;
  for (Geometry3 *g : g_geo3) unused += g->refs == 0;
  for (size_t i = 0; i < g_geo3.size() && unused > kGeo3Keep;) {
    if (g_geo3[i]->refs == 0) {
      geometry3_free(g_geo3[i]);
      g_geo3.erase(g_geo3.begin() + i);
      --unused;
    } else {
      ++i;
    }
  }
}

struct Unit3 {
  int4 u;
  long cost;
};

// the records and units of the displacements with one dz (record offsets local
// to this plane's record list)
struct Plane3 {
  std::vector<Unit3> units;
  std::vector<float> rec;
  double taps = 0.0;
};

void build_plane3(int n, int dz, Plane3 &out) {
  const int ldp = n + 1, plane = ldp * ldp;
  std::vector<double> box;
  std::vector<Run3> runs[3];
  std::vector<double> wts[3];
  std::vector<Unit3> &units = out.units;
  std::vector<float> &rec = out.rec;
  for (int dy = -(n - 1); dy < n; ++dy)
    for (int dx = -(n - 1); dx < n; ++dx) {
      if (dz == 0 && (dy < 0 || (dy == 0 && dx <= 0))) continue;
      const int wx = n - std::abs(dx), wy = n - std::abs(dy), wz = n - dz;
      int ox, oy, oz, bx, by, bz;
      stencil3(dx, dy, dz, box, ox, oy, oz, bx, by, bz);
      long nnz = 0;
      for (double v : box) nnz += v != 0.0;
      out.taps += (double)nnz * wx * wy * wz;
      // orientations: 0 runs z / lanes x / third y; 1 runs y / lanes x / third z; 2 runs x / lanes y / third z
      const int run_axis[3] = {2, 1, 0};
      const int lanes_of[3] = {wx, wx, wy}, stack_of[3] = {wz, wy, wx}, third_of[3] = {wy, wz, wz};
      int best = -1;
      long best_cost = 0;
      Plan3 plans[3];
      for (int o = 0; o < 3; ++o) {
        box_runs(box, ox, oy, oz, bx, by, bz, run_axis[o], runs[o], wts[o]);
        plans[o] = chunk_plan3(runs[o]);
        const long nunits = (long)((stack_of[o] + kR - 1) / kR) * std::min(pow2ceil(lanes_of[o]), third_of[o]);
        const long cost = nunits * plans[o].cost;
        if (best < 0 || cost < best_cost) {
          best = o;
          best_cost = cost;
        }
      }
      const Plan3 &pl = plans[best];
      const int off = (int)(rec.size() / 4);
      // header: chunks per length (16 bits per length 1..8), then the chunks
      // grouped by length, each group in run order
      unsigned counts[4] = {0u, 0u, 0u, 0u};
      for_each_chunk3(runs[best], [&](size_t, int, int lc) { counts[(lc - 1) >> 1] += 1u << (16 * ((lc - 1) & 1)); });
      float hbits[4];
      memcpy(hbits, counts, sizeof hbits);
      for (float f : hbits) rec.push_back(f);
      for (int len = 1; len <= kMaxChunk; ++len)
        for_each_chunk3(runs[best], [&](size_t ri, int c0, int lc) {
          if (lc != len) return;
          const Run3 &r = runs[best][ri];
          int cx = r.cx, cy = r.cy, cz = r.cz;
          if (run_axis[best] == 0) cx += c0;
          if (run_axis[best] == 1) cy += c0;
          if (run_axis[best] == 2) cz += c0;
          const int eoff = cx + ldp * cy + plane * cz;
          float obits;
          memcpy(&obits, &eoff, sizeof obits);
          rec.push_back(obits);
          for (int i = 0; i < lc; ++i) rec.push_back((float)wts[best][r.woff + c0 + i]);
          for (int i = lc + 1; i < 4 * ((lc + 4) / 4); ++i) rec.push_back(0.f);
        });
      const int lanes = lanes_of[best], third = third_of[best];
      const int gw = pow2ceil(lanes), lg = 5 - __builtin_ctz(gw);  // 32 / gw lane groups
      const int tlo = best == 0 ? std::max(0, -dy) : 0;           // third axis y (orientation 0) or z
      const int nsb = (stack_of[best] + kR - 1) / kR;
      const int dxyz = (dx & 0xff) | ((dy & 0xff) << 8) | ((dz & 0xff) << 16) | (best << 24) | (lg << 26);
      const int w = (int)pl.recs;  // the D's record float4s (header included)
      for (int sb = 0; sb < nsb; ++sb)
        for (int j = 0; j < gw && j < third; ++j)
          units.push_back({make_int4(off, dxyz, sb | ((tlo + j) << 8), w), pl.cost});
    }
}

// Units (int4): x = the D's record header (float4 index); y = dx | dy << 8 |
// dz << 16 (8-bit two's complement) | orientation << 24 | log2(lane groups)
// << 26; z = stack block | first third-axis coordinate << 8; w = the D's
// record float4s.
// The planes dz are built on host threads and joined in dz order.
vie_status geometry3_build(int n, Geometry3 *geo) {
  std::vector<Plane3> planes(n);
  const int nt = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  for (int t = 0; t < nt; ++t)
    pool.emplace_back([&, t]() {
      for (int dz = t; dz < n; dz += nt) build_plane3(n, dz, planes[dz]);
    });
  for (std::thread &th : pool) th.join();
  std::vector<Unit3> units;
  std::vector<float> rec;
  double taps = 0.0;
  for (int dz = 0; dz < n; ++dz) {
    const int base = (int)(rec.size() / 4);
    for (Unit3 u : planes[dz].units) {
      u.u.x += base;
      units.push_back(u);
    }
    rec.insert(rec.end(), planes[dz].rec.begin(), planes[dz].rec.end());
    taps += planes[dz].taps;
    std::vector<Unit3>().swap(planes[dz].units);
    std::vector<float>().swap(planes[dz].rec);
  }
  for (int i = 0; i < 32; ++i) rec.push_back(0.f);  // the L1 prefetch may reach 127 bytes past a stencil
  std::stable_sort(units.begin(), units.end(), [](const Unit3 &p, const Unit3 &q) { return p.cost > q.cost; });
  std::vector<int4> uv(units.size());
  for (size_t i = 0; i < units.size(); ++i) uv[i] = units[i].u;
  VIE_CUDA(vie_malloc((void **)&geo->units, sizeof(int4) * uv.size()));
  VIE_CUDA(cudaMemcpy(geo->units, uv.data(), sizeof(int4) * uv.size(), cudaMemcpyHostToDevice));
  VIE_CUDA(vie_malloc((void **)&geo->stencil, sizeof(float) * rec.size()));
  VIE_CUDA(cudaMemcpy(geo->stencil, rec.data(), sizeof(float) * rec.size(), cudaMemcpyHostToDevice));
  geo->n_units = (long)uv.size();
  geo->taps = taps;
  return VIE_OK;
}

vie_status geometry3_acquire(int device, int n, Geometry3 **out) {
  std::lock_guard<std::mutex> lock(g_geo3_mu);
  for (Geometry3 *g : g_geo3)
    if (g->device == device && g->n == n) {
      ++g->refs;
      *out = g;
      return VIE_OK;
    }
  Geometry3 *g = new Geometry3;
  g->device = device;
  g->n = n;
  const vie_status s = geometry3_build(n, g);
  if (s != VIE_OK) {
    geometry3_free(g);
    return s;
  }
  g->refs = 1;
  g_geo3.push_back(g);
  geometry3_trim();
  *out = g;
  return VIE_OK;
}

void geometry3_release(Geometry3 *g) {
  std::lock_guard<std::mutex> lock(g_geo3_mu);
  --g->refs;
  geometry3_trim();
}

}  // namespace

size_t disp3_smem_bytes(int n) {
  const long p = n + 1;
  return sizeof(float) * (size_t)(p * p * (p + kPad3));
}

vie_status disp3_prepare(DispPlan3 *dp, int n, const float *sig_padded, int device, cudaStream_t st) {
  dp->usable = 0;
  if (n < 2 || n > kMaxN3) return VIE_OK;
  DevProps prop;
  VIE_TRY(get_dev_props(device, &prop));
  const size_t smem = disp3_smem_bytes(n);
  if (smem > (size_t)prop.sharedMemPerBlockOptin) return VIE_OK;
  Disp3Kernel k = pick_disp3(n);
  VIE_TRY(raise_smem_limit((const void *)k, (size_t)((int)smem)));
  int bps = 0;
  VIE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, kThreads3, smem));
  if (bps < 1) return VIE_OK;
  Geometry3 *geo = nullptr;
  vie_status s = geometry3_acquire(device, n, &geo);
  if (s != VIE_OK) return s;
  dp->geometry = geo;
  dp->units = geo->units;
  dp->stencil = geo->stencil;
  dp->n_units = geo->n_units;
  dp->taps = geo->taps;
  const long N = (long)n * n * n, p = n + 1;
  const long lat = p * p * p, lat_elems = p * p * (p + kPad3);
  VIE_CUDA(vie_malloc((void **)&dp->counter, 2 * sizeof(int)));
  VIE_CUDA(cudaMemset(dp->counter, 0, 2 * sizeof(int)));
  VIE_CUDA(vie_malloc((void **)&dp->lattice, sizeof(float) * lat_elems));
  k_make_lattice3<<<(int)std::min((lat_elems + 255) / 256, 4096L), 256, 0, st>>>(lat, lat_elems, sig_padded,
                                                                                 (float *)dp->lattice);
  VIE_CHECK_LAUNCH("k_make_lattice3");
  VIE_CUDA(vie_malloc((void **)&dp->smax, sizeof(unsigned)));
  VIE_CUDA(cudaMemset(dp->smax, 0, sizeof(unsigned)));
  VIE_CUDA(vie_malloc((void **)&dp->scale, sizeof(double)));
  VIE_CUDA(vie_malloc((void **)&dp->src_t, sizeof(float) * (size_t)N));
  VIE_CUDA(vie_malloc((void **)&dp->yacc, sizeof(unsigned long long) * 2 * (size_t)N));
  VIE_CUDA(cudaMemset(dp->yacc, 0, sizeof(unsigned long long) * 2 * (size_t)N));
  // every row sum of A is below sum over all nonzero displacements of h / (4 pi |D|^2)
  double rb = 0.0;
  for (int dz = -(n - 1); dz < n; ++dz)
    for (int dy = -(n - 1); dy < n; ++dy)
      for (int dx = -(n - 1); dx < n; ++dx)
        if (dx || dy || dz) rb += 1.0 / ((double)dx * dx + (double)dy * dy + (double)dz * dz);
  dp->rbound = rb / (4.0 * kPi * n);
  dp->n = n;
  dp->lat_elems = lat_elems;
  dp->smem = smem;
  dp->grid = bps * prop.multiProcessorCount;
  dp->kernel = (const void *)k;
  dp->usable = 1;
  return VIE_OK;
}

void disp3_release(DispPlan3 *dp) {
  if (dp->geometry) geometry3_release((Geometry3 *)dp->geometry);
  if (dp->doff) vie_free(dp->doff);
  if (dp->ioff) vie_free(dp->ioff);
  if (dp->iqd) vie_free(dp->iqd);
  if (dp->counter) vie_free(dp->counter);
  if (dp->lattice) vie_free(dp->lattice);
  if (dp->smax) vie_free(dp->smax);
  if (dp->scale) vie_free(dp->scale);
  if (dp->src_t) vie_free(dp->src_t);
  if (dp->yacc) vie_free(dp->yacc);
  *dp = DispPlan3{};
}

vie_status disp3_apply(const DispPlan3 &dp, int op, const double *sigma_s, const double *g, const double *diag,
                       float *src, float tau_scale2, float wcoef, double *y, cudaEvent_t mid0, cudaEvent_t mid1,
                       cudaStream_t st) {
  const int n = dp.n;
  const long N = (long)n * n * n;
  const int blocks = (int)std::min((N + 255) / 256, 1024L);
  k_disp3_source<<<blocks, 256, 0, st>>>(N, n, op, sigma_s, g, src, dp.src_t, dp.smax);
  VIE_CHECK_LAUNCH("k_disp3_source");
  if (mid0) VIE_CUDA(cudaEventRecord(mid0, st));
  Disp3Args a;
  a.lat = (const float *)dp.lattice;
  a.stencil = (const float4 *)dp.stencil;
  a.src = src;
  a.src_t = dp.src_t;
  a.smax = dp.smax;
  a.scale_out = dp.scale;
  a.rbound = dp.rbound;
  a.yacc = dp.yacc;
  a.units = (const int4 *)dp.units;
  a.counter = dp.counter;
  a.n_units = dp.n_units;
  a.n = n;
  a.ldp = n + 1;
  a.plane = (n + 1) * (n + 1);
  a.lat_elems = dp.lat_elems;
  a.tau_scale2 = tau_scale2;
  a.wcoef = wcoef;
  void *args[] = {&a};
  VIE_CUDA(cudaLaunchKernel(dp.kernel, dim3(dp.grid), dim3(kThreads3), args, dp.smem, st));
  count_launch();
  if (mid1) VIE_CUDA(cudaEventRecord(mid1, st));
  k_disp3_reduce<<<(int)std::min((N + 255) / 256, 4096L), 256, 0, st>>>(N, n, op, dp.yacc, dp.scale, diag,
                                                                        sigma_s, g, y);
  VIE_CHECK_LAUNCH("k_disp3_reduce");
  return VIE_OK;
}

static size_t expand3_smem_bytes(int n) { return sizeof(float) * (size_t)(2 * n - 1) * (n + 2); }

// the store kernel's launch shape, the offsets of the stored weights per D
// and the expansion's items (once per plan)
static vie_status disp3_store_setup(DispPlan3 *dp, int device) {
  if (dp->kernel_store) return VIE_OK;
  const int n = dp->n;
  DevProps prop;
  VIE_TRY(get_dev_props(device, &prop));
  Disp3Kernel k = pick_disp3(n, true);
  VIE_TRY(raise_smem_limit((const void *)k, (size_t)((int)dp->smem)));
  int bps = 0;
  VIE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, kThreads3, dp->smem));
  if (bps < 1) {
    set_error("vie_assemble: the 3D store kernel does not fit an SM");
    return VIE_ERR_UNSUPPORTED;
  }
  const long m2 = 2 * n - 1;
  std::vector<long long> doff((size_t)(m2 * m2 * m2), 0);
  long off = 0;
  for (int dz = 0; dz < n; ++dz)
    for (int dy = -(n - 1); dy < n; ++dy)
      for (int dx = -(n - 1); dx < n; ++dx) {
        if (dz == 0 && (dy < 0 || (dy == 0 && dx <= 0))) continue;
        const long idx = ((long)(dz + n - 1) * m2 + (dy + n - 1)) * m2 + (dx + n - 1);
        doff[idx] = off;
        off += (long)(n - std::abs(dx)) * (n - std::abs(dy)) * (n - dz);
      }
  std::vector<int> ioff, iqd;
  int items = 0;
  for (int dz = 0; dz < n; ++dz)
    for (int dy = dz == 0 ? 0 : -(n - 1); dy < n; ++dy) {
      ioff.push_back(items);
      iqd.push_back((dy & 0xffff) | (dz << 16));
      items += (n - std::abs(dy)) * (n - dz);
    }
  ioff.push_back(items);
  VIE_CUDA(vie_malloc(&dp->doff, sizeof(long long) * doff.size()));
  VIE_CUDA(cudaMemcpy(dp->doff, doff.data(), sizeof(long long) * doff.size(), cudaMemcpyHostToDevice));
  VIE_CUDA(vie_malloc(&dp->ioff, sizeof(int) * ioff.size()));
  VIE_CUDA(cudaMemcpy(dp->ioff, ioff.data(), sizeof(int) * ioff.size(), cudaMemcpyHostToDevice));
  VIE_CUDA(vie_malloc(&dp->iqd, sizeof(int) * iqd.size()));
  VIE_CUDA(cudaMemcpy(dp->iqd, iqd.data(), sizeof(int) * iqd.size(), cudaMemcpyHostToDevice));
  dp->nq = (int)iqd.size();
  dp->items = items;
  dp->stored = off;
  dp->grid_store = bps * prop.multiProcessorCount;
  dp->kernel_store = (const void *)k;
  return VIE_OK;
}

vie_status disp3_assemble(DispPlan3 *dp, float tau_scale2, float wcoef, const double *sigma_s, const double *diag,
                          long ldk, float *k32, void *khi, void *klo, int device, cudaStream_t st) {
  if (!dp->usable) {
    set_error("vie_assemble: no 3D displacement plan");
    return VIE_ERR_UNSUPPORTED;
  }
  VIE_TRY(disp3_store_setup(dp, device));
  const int n = dp->n;
  const long N = (long)n * n * n;
  float *pairs = nullptr, *ss32 = nullptr;
  VIE_CUDA(vie_malloc(&pairs, sizeof(float) * (size_t)dp->stored));
  cudaError_t ce = vie_malloc(&ss32, sizeof(float) * (size_t)N);
  if (ce != cudaSuccess) {
    vie_free(pairs);
    return cuda_fail(ce, "cudaMalloc");
  }
  vie_status s = VIE_OK;
  {
    Disp3Args a{};
    a.lat = (const float *)dp->lattice;
    a.stencil = (const float4 *)dp->stencil;
    a.pairs = pairs;
    a.doff = dp->doff;
    a.units = (const int4 *)dp->units;
    a.counter = dp->counter;
    a.n_units = dp->n_units;
    a.n = n;
    a.ldp = n + 1;
    a.plane = (n + 1) * (n + 1);
    a.lat_elems = dp->lat_elems;
    a.tau_scale2 = tau_scale2;
    a.wcoef = wcoef;
    void *args[] = {&a};
    ce = cudaLaunchKernel(dp->kernel_store, dim3(dp->grid_store), dim3(kThreads3), args, dp->smem, st);
    if (ce != cudaSuccess) s = cuda_fail(ce, "k_pairs_disp3 (store)");
    else count_launch();
  }
  const size_t esz = k32 ? sizeof(float) : sizeof(unsigned short);
  if (s == VIE_OK && ldk > N) {  // dense K: zero the padding columns [N, ldk) of every row
    if (k32) ce = cudaMemset2DAsync(k32 + N, ldk * esz, 0, (ldk - N) * esz, N, st);
    else {
      ce = cudaMemset2DAsync((unsigned short *)khi + N, ldk * esz, 0, (ldk - N) * esz, N, st);
      if (ce == cudaSuccess) ce = cudaMemset2DAsync((unsigned short *)klo + N, ldk * esz, 0, (ldk - N) * esz, N, st);
    }
    if (ce != cudaSuccess) s = cuda_fail(ce, "cudaMemset2DAsync");
  }
  if (s == VIE_OK) {
    k_to_f32_3<<<(int)std::min((N + 255) / 256, 1024L), 256, 0, st>>>(N, sigma_s, ss32);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) s = cuda_fail(ce, "k_to_f32_3");
  }
  if (s == VIE_OK) {
    const size_t smem = expand3_smem_bytes(n);
    DevProps prop;
    s = get_dev_props(device, &prop);
    if (s == VIE_OK) {
      const int grid = 4 * prop.multiProcessorCount;
      if (ldk == 0)
        k_expand_pairs3<kExpSym><<<grid, kExpThreads, smem, st>>>(n, pairs, dp->doff, dp->ioff, dp->iqd, dp->nq, ss32,
                                                                 diag, sigma_s, 0, k32, nullptr, nullptr);
      else if (k32)
        k_expand_pairs3<kExpF32><<<grid, kExpThreads, smem, st>>>(n, pairs, dp->doff, dp->ioff, dp->iqd, dp->nq, ss32, diag,
                                                          sigma_s, ldk, k32, nullptr, nullptr);
      else
        k_expand_pairs3<kExpBF16><<<grid, kExpThreads, smem, st>>>(n, pairs, dp->doff, dp->ioff, dp->iqd, dp->nq, ss32,
                                                           diag, sigma_s, ldk, nullptr, (unsigned short *)khi,
                                                           (unsigned short *)klo);
      ce = cudaGetLastError();
      if (ce != cudaSuccess) s = cuda_fail(ce, "k_expand_pairs3");
      else count_launch();
    }
  }
  // the frees wait for the device (the expansion reads both buffers)
  vie_free(pairs);
  vie_free(ss32);
  return s;
}

vie_status disp3_sym_sizes(DispPlan3 *dp, int device, long *block_floats, long *partial_floats) {
  if (!dp->usable) {
    set_error("vie_assemble: no 3D displacement plan");
    return VIE_ERR_UNSUPPORTED;
  }
  VIE_TRY(disp3_store_setup(dp, device));
  *block_floats = dp->items * (long)dp->n * dp->n;
  *partial_floats = dp->items * 2L * dp->n;
  return VIE_OK;
}

vie_status symv3_apply(const DispPlan3 &dp, int op, const double *sigma_s, const double *g, const float *blocks,
                       float *s, float *partial, double *y, int device, cudaStream_t st) {
  const int n = dp.n;
  const long N = (long)n * n * n;
  DevProps prop;
  VIE_TRY(get_dev_props(device, &prop));
  k_symv3_source<<<(int)std::min((N + 255) / 256, 1024L), 256, 0, st>>>(N, op, sigma_s, g, s);
  VIE_CHECK_LAUNCH("k_symv3_source");
  const long ctas = std::min((dp.items + kSymvWarps3 - 1) / kSymvWarps3, 8L * prop.multiProcessorCount);
  k_symv3_blocks<<<(int)ctas, 32 * kSymvWarps3, 0, st>>>(n, blocks, s, dp.ioff, dp.iqd, dp.nq, partial);
  VIE_CHECK_LAUNCH("k_symv3_blocks");
  k_symv3_reduce<<<n * n, 32 * kSymvWarps3, 0, st>>>(n, op, partial, dp.ioff, dp.iqd, dp.nq, g, y);
  VIE_CHECK_LAUNCH("k_symv3_reduce");
  return VIE_OK;
}

}  // namespace vie
