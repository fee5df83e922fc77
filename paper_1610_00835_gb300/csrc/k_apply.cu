// Operator apply: kernel tiles generated on the fly (Section 3.2, approach
// M-iii; Section 3.3, "the main computational cost ... evaluations of K U").
//
// For a target cell j and a source cell k != j on the uniform grid, with
// lattice coordinates u = x/h - 1/2 (cell centres on the integers):
//   tau_jk = (r_jk / S) sum_{i=0}^{S-1} sigma_t~(u_j + (i+1/2)/S (u_k - u_j))
//   A_jk   = h^d exp(-tau_jk) / (|S^{d-1}| r_jk^{d-1})
// (Section 2, definitions of E(x,y) and of the kernel, Eq. EQ:Kernel), and
//   y_j = sum_{k != j} A_jk s_k + d_j s_j
// with s = sigma_s g (op K) or s = g (op A), d_j the self-cell integral.
//
// FP32 path: one CTA of 256 threads owns 256 consecutive targets and one
// contiguous range of sources (a "split"); sigma_t sits in shared memory as
// an (n+1)^d lattice padded by one edge copy, so the bilinear/trilinear
// corner loads need no clamping.  In cell units the sample positions
// u_j + (i+1/2)/S (u_k - u_j) are exact in FP32 for S a power of two (all
// operands are multiples of 1/(2S) below 2^12), so only the interpolated
// values and the sums round.  Floors use the round-to-nearest of
// (u - 1/2) + 1.5*2^23, an FP32 add instead of a conversion; at exact
// integers it may pick the lower cell with weight 1, which gives the same
// value because the interpolant is continuous.  Partial sums are FP32 over
// at most 64 sources, FP64 across them, and written per split; a second
// kernel adds the splits in a fixed order (deterministic) with the diagonal.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "vie_internal.cuh"

namespace vie {

namespace {

constexpr float kMagic = 12582912.0f;       // 1.5 * 2^23
constexpr int kMagicBits = 0x4B400000;      // bit pattern of kMagic
constexpr float kLog2e = 1.4426950408889634f;

struct PairArgs {
  const float *sig;     // padded sigma_t lattice (global); copied to smem if staged
  const float *src;     // s_k, FP32 [N]
  double *partial;      // [splits][N]
  long N;
  int n, P, tiles, splits, chunk, S;
  long lattice;         // P^dim
  float tau_scale2;     // (h / S) * log2(e)   (march) or h * sigma_c * log2(e) (closed)
  float wcoef;          // h / (2 pi) in 2D, h / (4 pi) in 3D
};

// Floor of a non-negative lattice coordinate p (|p| < 2^22) with its weight:
// returns the integer cell index and writes a = p - cell in [0, 1].
__device__ __forceinline__ int floor_frac(float p, float &a) {
  float y = (p - 0.5f) + kMagic;
  float fl = y - kMagic;
  a = p - fl;
  return __float_as_int(y) - kMagicBits;
}

template <int DIM>
__device__ __forceinline__ float sample(const float *__restrict__ s, int P, float px, float py,
                                        float pz) {
  float ax, ay;
  int ix = floor_frac(px, ax);
  int iy = floor_frac(py, ay);
  if (DIM == 2) {
    const float *r0 = s + iy * P + ix;
    float v00 = r0[0], v10 = r0[1], v01 = r0[P], v11 = r0[P + 1];
    float lo = fmaf(ax, v10 - v00, v00);
    float hi = fmaf(ax, v11 - v01, v01);
    return fmaf(ay, hi - lo, lo);
  } else {
    float az;
    int iz = floor_frac(pz, az);
    const float *r0 = s + (iz * P + iy) * P + ix;
    const float *r1 = r0 + P * P;
    float a0 = fmaf(ax, r0[1] - r0[0], r0[0]);
    float a1 = fmaf(ax, r0[P + 1] - r0[P], r0[P]);
    float b0 = fmaf(ax, r1[1] - r1[0], r1[0]);
    float b1 = fmaf(ax, r1[P + 1] - r1[P], r1[P]);
    float c0 = fmaf(ay, a1 - a0, a0);
    float c1 = fmaf(ay, b1 - b0, b0);
    return fmaf(az, c1 - c0, c0);
  }
}

// Sum over the S midpoint samples of sigma_t~ on the segment u_j -> u_k.
// Four independent accumulators bound the FP32 rounding of the 64-term sum.
template <int DIM, int S_CT>
__device__ __forceinline__ float march(const float *__restrict__ s, int P, int S, float jx,
                                       float jy, float jz, float dx, float dy, float dz) {
  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
  if (S_CT > 0) {
#pragma unroll
    for (int i = 0; i < S_CT; i += 4) {
      const float t0 = (i + 0.5f) / S_CT, t1 = (i + 1.5f) / S_CT;
      const float t2 = (i + 2.5f) / S_CT, t3 = (i + 3.5f) / S_CT;
      acc0 += sample<DIM>(s, P, fmaf(t0, dx, jx), fmaf(t0, dy, jy), fmaf(t0, dz, jz));
      acc1 += sample<DIM>(s, P, fmaf(t1, dx, jx), fmaf(t1, dy, jy), fmaf(t1, dz, jz));
      acc2 += sample<DIM>(s, P, fmaf(t2, dx, jx), fmaf(t2, dy, jy), fmaf(t2, dz, jz));
      acc3 += sample<DIM>(s, P, fmaf(t3, dx, jx), fmaf(t3, dy, jy), fmaf(t3, dz, jz));
    }
  } else {
    const float inv = 1.0f / (float)S;
#pragma unroll 4
    for (int i = 0; i < S; ++i) {
      const float t = ((float)i + 0.5f) * inv;
      acc0 += sample<DIM>(s, P, fmaf(t, dx, jx), fmaf(t, dy, jy), fmaf(t, dz, jz));
    }
  }
  return (acc0 + acc1) + (acc2 + acc3);
}

// MODE 0: march, sigma_t in shared memory; 1: march, sigma_t from global;
// 2: closed form tau = sigma_c r.
template <int DIM, int MODE, int S_CT>
__global__ void __launch_bounds__(kPairThreads) k_pairs_f32(PairArgs a) {
  extern __shared__ float4 smem4[];
  float4 *srcs = smem4;                                  // [kPairThreads]
  float *lat = reinterpret_cast<float *>(smem4 + kPairThreads);
  const float *sig = (MODE == 0) ? lat : a.sig;
  const int tid = threadIdx.x;
  if (MODE == 0) {
    const float4 *g4 = reinterpret_cast<const float4 *>(a.sig);
    long n4 = a.lattice / 4;
    for (long i = tid; i < n4; i += blockDim.x) reinterpret_cast<float4 *>(lat)[i] = g4[i];
    for (long i = n4 * 4 + tid; i < a.lattice; i += blockDim.x) lat[i] = a.sig[i];
    __syncthreads();
  }
  const int n = a.n;
  const long items = (long)a.tiles * a.splits;
  for (long item = blockIdx.x; item < items; item += gridDim.x) {
    const int tile = (int)(item % a.tiles);
    const int split = (int)(item / a.tiles);
    const long j_raw = (long)tile * kPairThreads + tid;
    const bool valid = j_raw < a.N;
    const long j = valid ? j_raw : a.N - 1;
    const float jx = (float)(j % n);
    const float jy = (float)((j / n) % n);
    const float jz = DIM == 3 ? (float)(j / ((long)n * n)) : 0.f;
    const long k_begin = (long)split * a.chunk;
    const long k_end = min(a.N, k_begin + a.chunk);
    double dsum = 0.0;
    for (long k0 = k_begin; k0 < k_end; k0 += kPairThreads) {
      const int cnt = (int)min((long)kPairThreads, k_end - k0);
      __syncthreads();
      if (tid < cnt) {
        long k = k0 + tid;
        float kx = (float)(k % n), ky = (float)((k / n) % n);
        float kz = DIM == 3 ? (float)(k / ((long)n * n)) : 0.f;
        srcs[tid] = make_float4(kx, ky, kz, a.src[k]);
      }
      __syncthreads();
      for (int c0 = 0; c0 < cnt; c0 += 64) {
        const int c1 = min(cnt, c0 + 64);
        float fsum = 0.f;
        for (int c = c0; c < c1; ++c) {
          const float4 q = srcs[c];
          const float dx = q.x - jx, dy = q.y - jy, dz = q.z - jz;
          const float r2 = DIM == 3 ? fmaf(dz, dz, fmaf(dy, dy, dx * dx)) : fmaf(dy, dy, dx * dx);
          const float inv_r = rsqrtf(r2);
          const float r = r2 * inv_r;
          float e2;  // -tau * log2(e)
          if (MODE == 2) {
            e2 = -a.tau_scale2 * r;
          } else {
            const float acc = march<DIM, S_CT>(sig, a.P, a.S, jx, jy, jz, dx, dy, dz);
            e2 = -a.tau_scale2 * acc * r;
          }
          const float ker = DIM == 3 ? inv_r * inv_r : inv_r;
          const float w = a.wcoef * exp2f(e2) * ker;
          fsum = (r2 > 0.f) ? fmaf(w, q.w, fsum) : fsum;
        }
        dsum += (double)fsum;
      }
    }
    if (valid) a.partial[(long)split * a.N + j] = dsum;
  }
}

// FP64 path: every pair in FP64, sigma_t read from the padded FP64 lattice.
struct PairArgs64 {
  const double *sig;
  const double *src;
  double *partial;
  long N;
  int n, P, tiles, splits, chunk, S, closed;
  double h, sigma_c, wcoef;
};

template <int DIM>
__device__ double sample64(const double *__restrict__ s, int P, const double *p) {
  int i0[3];
  double w[3];
  for (int d = 0; d < DIM; ++d) {
    double f = floor(p[d]);
    i0[d] = (int)f;
    w[d] = p[d] - f;
  }
  if (DIM == 2) {
    const double *r0 = s + (long)i0[1] * P + i0[0];
    double lo = (1.0 - w[0]) * r0[0] + w[0] * r0[1];
    double hi = (1.0 - w[0]) * r0[P] + w[0] * r0[P + 1];
    return (1.0 - w[1]) * lo + w[1] * hi;
  }
  double out = 0.0;
  for (int cz = 0; cz < 2; ++cz)
    for (int cy = 0; cy < 2; ++cy)
      for (int cx = 0; cx < 2; ++cx) {
        double ww = (cx ? w[0] : 1.0 - w[0]) * (cy ? w[1] : 1.0 - w[1]) * (cz ? w[2] : 1.0 - w[2]);
        out += ww * s[((long)(i0[2] + cz) * P + (i0[1] + cy)) * P + (i0[0] + cx)];
      }
  return out;
}

template <int DIM>
__global__ void __launch_bounds__(kPairThreads) k_pairs_f64(PairArgs64 a) {
  const int tid = threadIdx.x;
  const int n = a.n;
  const long items = (long)a.tiles * a.splits;
  for (long item = blockIdx.x; item < items; item += gridDim.x) {
    const int tile = (int)(item % a.tiles);
    const int split = (int)(item / a.tiles);
    const long j = (long)tile * kPairThreads + tid;
    if (j >= a.N) continue;
    double uj[3] = {(double)(j % n), (double)((j / n) % n),
                    DIM == 3 ? (double)(j / ((long)n * n)) : 0.0};
    const long k_begin = (long)split * a.chunk;
    const long k_end = min(a.N, k_begin + a.chunk);
    double sum = 0.0;
    for (long k = k_begin; k < k_end; ++k) {
      if (k == j) continue;
      double uk[3] = {(double)(k % n), (double)((k / n) % n),
                      DIM == 3 ? (double)(k / ((long)n * n)) : 0.0};
      double r2 = 0.0;
      for (int d = 0; d < DIM; ++d) r2 += (uk[d] - uj[d]) * (uk[d] - uj[d]);
      double r = sqrt(r2);
      double tau;
      if (a.closed) {
        tau = a.sigma_c * a.h * r;
      } else {
        double acc = 0.0, p[3];
        for (int i = 0; i < a.S; ++i) {
          double t = (i + 0.5) / a.S;
          for (int d = 0; d < DIM; ++d) p[d] = uj[d] + t * (uk[d] - uj[d]);
          acc += sample64<DIM>(a.sig, a.P, p);
        }
        tau = a.h * r * acc / a.S;
      }
      double ker = DIM == 3 ? 1.0 / r2 : 1.0 / r;
      sum += a.wcoef * exp(-tau) * ker * a.src[k];
    }
    a.partial[(long)split * a.N + j] = sum;
  }
}

__global__ void k_source_prep_f32(long N, int op, const double *__restrict__ ss,
                                  const double *__restrict__ g, float *__restrict__ s) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x)
    s[i] = (float)(op == VIE_OP_A_RAW ? g[i] : ss[i] * g[i]);
}

__global__ void k_source_prep_f64(long N, int op, const double *__restrict__ ss,
                                  const double *__restrict__ g, double *__restrict__ s) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x)
    s[i] = op == VIE_OP_A_RAW ? g[i] : ss[i] * g[i];
}

// y_j = sum_split partial[split][j] + d_j s_j, then the requested operator.
__global__ void k_reduce(long N, int splits, int op, const double *__restrict__ partial,
                         const double *__restrict__ diag, const double *__restrict__ ss,
                         const double *__restrict__ g, double *__restrict__ y) {
  for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < N; j += (long)gridDim.x * blockDim.x) {
    double s = op == VIE_OP_A_RAW ? g[j] : ss[j] * g[j];
    double acc = diag[j] * s;
    for (int p = 0; p < splits; ++p) acc += partial[(long)p * N + j];
    y[j] = op == VIE_OP_I_MINUS_K ? g[j] - acc : acc;
  }
}

__global__ void k_pad_sigma(int dim, int n, const double *__restrict__ sig, float *__restrict__ o32,
                            double *__restrict__ o64) {
  const int P = n + 1;
  long total = dim == 2 ? (long)P * P : (long)P * P * P;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    long px = i % P, py = (i / P) % P, pz = dim == 3 ? i / ((long)P * P) : 0;
    px = min(px, (long)n - 1);
    py = min(py, (long)n - 1);
    pz = min(pz, (long)n - 1);
    double v = sig[(pz * n + py) * n + px];
    o32[i] = (float)v;
    o64[i] = v;
  }
}

// ---- self cell (M-iii with the singular integral computed explicitly)
// Gauss-Legendre nodes/weights on [-1, 1], filled by the host.
constexpr int kGL = 32;
__constant__ double c_gl_x[kGL];
__constant__ double c_gl_w[kGL];

// (1 - e^{-s R}) / s, the radial integral of e^{-s rho} over [0, R].
__device__ double radial(double s, double R) { return s == 0.0 ? R : -expm1(-s * R) / s; }

// 2D: d = (1/2pi) * 8 * int_0^{pi/4} radial(sigma, a sec th) dth, a = h/2.
// 3D: d = (1/4pi) * 48 * int_0^{pi/4} dphi int_a^{a sqrt(1+sec^2 phi)}
//          a radial(sigma, rho) / rho^2 drho
// (polar / face parametrisation of the square / cube about its centre).
__global__ void k_selfcell(int dim, long N, double h, const double *__restrict__ sig,
                           double *__restrict__ d) {
  for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < N; j += (long)gridDim.x * blockDim.x) {
    const double s = sig[j], a = 0.5 * h, q = 0.25 * kPi;
    double I = 0.0;
    if (dim == 2) {
      for (int i = 0; i < kGL; ++i) {
        double th = 0.5 * q * (c_gl_x[i] + 1.0);
        I += c_gl_w[i] * radial(s, a / cos(th));
      }
      d[j] = 8.0 * (0.5 * q * I) / (2.0 * kPi);
    } else {
      for (int i = 0; i < kGL; ++i) {
        double ph = 0.5 * q * (c_gl_x[i] + 1.0);
        double sec = 1.0 / cos(ph);
        double rmax = a * sqrt(1.0 + sec * sec);
        double inner = 0.0;
        for (int k = 0; k < kGL; ++k) {
          double rho = a + 0.5 * (rmax - a) * (c_gl_x[k] + 1.0);
          inner += c_gl_w[k] * a * radial(s, rho) / (rho * rho);
        }
        I += c_gl_w[i] * 0.5 * (rmax - a) * inner;
      }
      d[j] = 48.0 * (0.5 * q * I) / (4.0 * kPi);
    }
  }
}

int grid_for(long n, int threads) {
  long b = (n + threads - 1) / threads;
  return (int)std::max(1L, std::min(b, 4096L));
}

// Gauss-Legendre rule by Newton iteration on the Legendre polynomial P_m,
// started from the asymptotic root estimate cos(pi (i - 1/4) / (m + 1/2)).
void gauss_legendre(int m, std::vector<double> &x, std::vector<double> &w) {
  x.assign(m, 0.0);
  w.assign(m, 0.0);
  for (int i = 0; i < m; ++i) {
    double z = cos(kPi * (i + 0.75) / (m + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= m; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = m * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

template <int DIM, int MODE>
const void *pair_kernel_ptr(int steps) {
  if (steps == 64) return (const void *)k_pairs_f32<DIM, MODE, 64>;
  return (const void *)k_pairs_f32<DIM, MODE, 0>;
}

const void *pair_kernel(int dim, int mode, int steps) {
  if (dim == 2) {
    if (mode == 0) return pair_kernel_ptr<2, 0>(steps);
    if (mode == 1) return pair_kernel_ptr<2, 1>(steps);
    return (const void *)k_pairs_f32<2, 2, 0>;
  }
  if (mode == 0) return pair_kernel_ptr<3, 0>(steps);
  if (mode == 1) return pair_kernel_ptr<3, 1>(steps);
  return (const void *)k_pairs_f32<3, 2, 0>;
}

int kernel_mode(const PairPlan &p, int tau_closed) { return tau_closed ? 2 : (p.smem_sigma ? 0 : 1); }

}  // namespace

vie_status plan_pairs(const Medium &m, int steps, int tau_closed, int precision, int device,
                      PairPlan *plan) {
  DevProps prop;
  VIE_TRY(get_dev_props(device, &prop));
  PairPlan p{};
  p.tiles = (int)((m.N + kPairThreads - 1) / kPairThreads);
  size_t lattice = m.dim == 2 ? (size_t)m.P * m.P : (size_t)m.P * m.P * m.P;
  size_t stage = sizeof(float4) * kPairThreads;
  int bps = 1;
  if (precision == VIE_PREC_FP64) {
    p.smem_sigma = 0;
    p.smem_bytes = 0;
    VIE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &bps, m.dim == 2 ? k_pairs_f64<2> : k_pairs_f64<3>, kPairThreads, 0));
  } else {
    size_t want = stage + lattice * sizeof(float);
    p.smem_sigma = (!tau_closed && want <= (size_t)prop.sharedMemPerBlockOptin) ? 1 : 0;
    p.smem_bytes = p.smem_sigma ? want : stage;
    const void *k = pair_kernel(m.dim, kernel_mode(p, tau_closed), steps);
    VIE_TRY(raise_smem_limit(k, (size_t)((int)p.smem_bytes)));
    VIE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, kPairThreads, p.smem_bytes));
  }
  bps = std::max(1, bps);
  long slots = (long)bps * prop.multiProcessorCount;
  // About eight work items per resident CTA slot keeps the tail short while
  // each split still covers many sources.
  long want_items = 8 * slots;
  long splits = std::max(1L, (want_items + p.tiles - 1) / p.tiles);
  splits = std::min(splits, std::max(1L, m.N / 64));
  p.splits = (int)splits;
  p.chunk = (int)((m.N + splits - 1) / splits);
  p.splits = (int)((m.N + p.chunk - 1) / p.chunk);
  long items = (long)p.tiles * p.splits;
  long per = (items + slots - 1) / slots;
  p.grid = (int)((items + per - 1) / per);
  *plan = p;
  return VIE_OK;
}

vie_status launch_pairs(const Medium &m, const PairPlan &plan, int steps, int tau_closed,
                        int precision, const void *src, double *partial, cudaStream_t st) {
  const double h = 1.0 / m.n;
  if (precision == VIE_PREC_FP64) {
    PairArgs64 a;
    a.sig = m.sig64;
    a.src = (const double *)src;
    a.partial = partial;
    a.N = m.N;
    a.n = m.n;
    a.P = m.P;
    a.tiles = plan.tiles;
    a.splits = plan.splits;
    a.chunk = plan.chunk;
    a.S = steps;
    a.closed = tau_closed;
    a.h = h;
    a.sigma_c = m.sigma_c;
    a.wcoef = m.dim == 2 ? h / (2.0 * kPi) : h / (4.0 * kPi);
    if (m.dim == 2)
      k_pairs_f64<2><<<plan.grid, kPairThreads, 0, st>>>(a);
    else
      k_pairs_f64<3><<<plan.grid, kPairThreads, 0, st>>>(a);
    VIE_CHECK_LAUNCH("k_pairs_f64");
    return VIE_OK;
  }
  PairArgs a;
  a.sig = m.sig32;
  a.src = (const float *)src;
  a.partial = partial;
  a.N = m.N;
  a.n = m.n;
  a.P = m.P;
  a.tiles = plan.tiles;
  a.splits = plan.splits;
  a.chunk = plan.chunk;
  a.S = steps;
  a.lattice = m.dim == 2 ? (long)m.P * m.P : (long)m.P * m.P * m.P;
  a.tau_scale2 = tau_closed ? (float)(h * m.sigma_c * 1.4426950408889634)
                            : (float)(h / steps * 1.4426950408889634);
  a.wcoef = (float)(m.dim == 2 ? h / (2.0 * kPi) : h / (4.0 * kPi));
  const void *k = pair_kernel(m.dim, kernel_mode(plan, tau_closed), steps);
  void *args[] = {&a};
  VIE_CUDA(cudaLaunchKernel(k, dim3(plan.grid), dim3(kPairThreads), args, plan.smem_bytes, st));
  count_launch();
  return VIE_OK;
}

// The limit a kernel has been raised to, per device, is remembered, so that
// launches on hot paths do not query the function's attributes every time.
vie_status raise_smem_limit(const void *k, size_t bytes) {
  struct Seen {
    int device;
    const void *kernel;
    size_t bytes;
  };
  static std::mutex mu;
  static std::vector<Seen> seen;
  int dev = 0;
  VIE_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  for (const Seen &e : seen)
    if (e.device == dev && e.kernel == k && e.bytes >= bytes) return VIE_OK;
  cudaFuncAttributes at;
  VIE_CUDA(cudaFuncGetAttributes(&at, k));
  if ((size_t)at.maxDynamicSharedSizeBytes < bytes)
    VIE_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  seen.push_back({dev, k, std::max(bytes, (size_t)at.maxDynamicSharedSizeBytes)});
  return VIE_OK;
}

vie_status launch_source_prep(long N, int op, const double *sigma_s, const double *g,
                              int precision, void *src, cudaStream_t st) {
  if (precision == VIE_PREC_FP64)
    k_source_prep_f64<<<grid_for(N, 256), 256, 0, st>>>(N, op, sigma_s, g, (double *)src);
  else
    k_source_prep_f32<<<grid_for(N, 256), 256, 0, st>>>(N, op, sigma_s, g, (float *)src);
  VIE_CHECK_LAUNCH("k_source_prep");
  return VIE_OK;
}

vie_status launch_reduce(long N, int splits, int op, const double *partial, const double *diag,
                         const double *sigma_s, const double *g, double *y, cudaStream_t st) {
  k_reduce<<<grid_for(N, 256), 256, 0, st>>>(N, splits, op, partial, diag, sigma_s, g, y);
  VIE_CHECK_LAUNCH("k_reduce");
  return VIE_OK;
}

vie_status launch_pad_sigma(int dim, int n, const double *sig, float *out32, double *out64,
                            cudaStream_t st) {
  long P = n + 1;
  long total = dim == 2 ? P * P : P * P * P;
  k_pad_sigma<<<grid_for(total, 256), 256, 0, st>>>(dim, n, sig, out32, out64);
  VIE_CHECK_LAUNCH("k_pad_sigma");
  return VIE_OK;
}

vie_status launch_selfcell(int dim, int n, const double *sigma_t, double *diag, cudaStream_t st) {
  // The rule lives in __constant__ memory, which is per device: upload it
  // once for every device the library runs on (under a lock: host threads
  // may make their first calls on a device at the same time).
  static std::mutex rule_mu;
  static bool have_rule[256] = {};
  int dev = 0;
  VIE_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return VIE_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lock(rule_mu);
    if (!have_rule[dev]) {
      std::vector<double> x, w;
      gauss_legendre(kGL, x, w);
      VIE_CUDA(cudaMemcpyToSymbol(c_gl_x, x.data(), sizeof(double) * kGL));
      VIE_CUDA(cudaMemcpyToSymbol(c_gl_w, w.data(), sizeof(double) * kGL));
      have_rule[dev] = true;
    }
  }
  long N = dim == 2 ? (long)n * n : (long)n * n * n;
  k_selfcell<<<grid_for(N, 128), 128, 0, st>>>(dim, N, 1.0 / n, sigma_t, diag);
  VIE_CHECK_LAUNCH("k_selfcell");
  return VIE_OK;
}

}  // namespace vie
