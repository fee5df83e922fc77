// FP64 Krylov building blocks for GMRES(m) (Algorithm 1, S.2; Section 5).
//
// Arnoldi uses classical Gram-Schmidt applied twice (CGS2): h = V^T w,
// w -= V h, repeated, so each pass is two bandwidth-bound sweeps over the
// basis instead of k dependent ones.  Dot products are block partials summed
// in a fixed order by a second kernel, so results do not depend on timing.
// Givens rotations and the triangular solve are tiny and run in one thread.
#include <math.h>

#include "vie_internal.cuh"

namespace vie {

namespace {

constexpr int kDotThreads = 256;

__device__ __forceinline__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

// part[b * nv + i] = sum over this block's slice of V_i . w
__global__ void __launch_bounds__(kDotThreads) k_dots(const double *__restrict__ V, int nv, long ldv,
                                                      const double *__restrict__ w, long N,
                                                      double *__restrict__ part) {
  __shared__ double red[kDotThreads / 32];
  const long stride = (long)gridDim.x * blockDim.x;
  const long i0 = blockIdx.x * (long)blockDim.x + threadIdx.x;
  for (int v = 0; v < nv; ++v) {
    const double *x = V + (long)v * ldv;
    double s = 0.0;
    for (long i = i0; i < N; i += stride) s += x[i] * w[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[(long)blockIdx.x * nv + v] = s;
  }
}

__global__ void k_dots_finish(const double *__restrict__ part, int blocks, int nv,
                              double *__restrict__ out, int accumulate) {
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < blocks; ++b) s += part[(long)b * nv + v];
    out[v] = accumulate ? out[v] + s : s;
  }
}

// w -= sum_v h_v V_v
__global__ void k_orth_update(const double *__restrict__ V, int nv, long ldv,
                              const double *__restrict__ h, double *__restrict__ w, long N) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    double acc = w[i];
    for (int v = 0; v < nv; ++v) acc -= h[v] * V[(long)v * ldv + i];
    w[i] = acc;
  }
}

// x += sum_v y_v V_v
__global__ void k_lincomb_add(const double *__restrict__ V, int nv, long ldv,
                              const double *__restrict__ y, double *__restrict__ x, long N) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    double acc = x[i];
    for (int v = 0; v < nv; ++v) acc += y[v] * V[(long)v * ldv + i];
    x[i] = acc;
  }
}

// y = x / norm, norm = sqrt(*n2) if use_sqrt else *n2; a zero norm gives y = 0.
__global__ void k_scale(const double *__restrict__ x, const double *__restrict__ n2, int use_sqrt,
                        double *__restrict__ y, long N) {
  double nrm = use_sqrt ? sqrt(*n2) : *n2;
  double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x)
    y[i] = x[i] * inv;
}

__global__ void k_axpby(double a, const double *__restrict__ x, double b,
                        const double *__restrict__ y, double *__restrict__ z, long N) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x)
    z[i] = a * x[i] + b * y[i];
}

// Column k of the Hessenberg matrix H ((m+1) x m, column-major): entries
// 0..k from hcol, entry k+1 = sqrt(hk1sq).  Apply the k earlier rotations,
// build rotation k, rotate the residual vector gv, and write
// |gv[k+1]| / bnorm to *est.  One thread.
__device__ void givens_step(double *H, int m, int k, const double *hcol, double hk1sq, double *cs, double *sn,
                            double *gv, double bnorm, double *est) {
  double *c = H + (long)k * (m + 1);
  for (int i = 0; i <= k; ++i) c[i] = hcol[i];
  c[k + 1] = sqrt(hk1sq);
  for (int i = 0; i < k; ++i) {
    double a = c[i], b = c[i + 1];
    c[i] = cs[i] * a + sn[i] * b;
    c[i + 1] = -sn[i] * a + cs[i] * b;
  }
  double a = c[k], b = c[k + 1];
  double den = hypot(a, b);
  double cc = den > 0.0 ? a / den : 1.0, ss = den > 0.0 ? b / den : 0.0;
  cs[k] = cc;
  sn[k] = ss;
  c[k] = den;
  c[k + 1] = 0.0;
  double g = gv[k];
  gv[k] = cc * g;
  gv[k + 1] = -ss * g;
  *est = fabs(gv[k + 1]) / bnorm;
}

__global__ void k_givens(double *H, int m, int k, const double *hcol, const double *hk1sq,
                         double *cs, double *sn, double *gv, double bnorm, double *est) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  givens_step(H, m, k, hcol, *hk1sq, cs, sn, gv, bnorm, est);
}

// k_dots and k_dots_finish in one launch: the last block to finish (by an
// atomic ticket, reset for the next launch) sums the block partials in block
// order, the same order as k_dots_finish: out1[v] = s and/or out2[v] += s.
// With gv != nullptr (nv = 1, V = w) the sum is ||w||^2 and the last block
// then takes the Givens step of column k with it.
__global__ void __launch_bounds__(kDotThreads) k_dots_last(const double *__restrict__ V, int nv, long ldv,
                                                           const double *__restrict__ w, long N, double *part,
                                                           int *ticket, double *out1, double *out2, double *H,
                                                           int m, int k, const double *hcol, double *cs,
                                                           double *sn, double *gv, double bnorm, double *est) {
  __shared__ double red[kDotThreads / 32];
  __shared__ int last;
  const long stride = (long)gridDim.x * blockDim.x;
  const long i0 = blockIdx.x * (long)blockDim.x + threadIdx.x;
  for (int v = 0; v < nv; ++v) {
    const double *x = V + (long)v * ldv;
    double sum = 0.0;
    for (long i = i0; i < N; i += stride) sum += x[i] * w[i];
    sum = block_sum(sum, red);
    if (threadIdx.x == 0) part[(long)blockIdx.x * nv + v] = sum;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    double sum = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) sum += __ldcg(part + (long)b * nv + v);
    if (out1) out1[v] = sum;
    if (out2) out2[v] += sum;
    if (gv && v == 0) givens_step(H, m, k, hcol, sum, cs, sn, gv, bnorm, est);
  }
  if (threadIdx.x == 0) *ticket = 0;
}

// Solve the k x k upper-triangular system R y = gv[0..k-1], R = H[0..k-1][0..k-1].
__global__ void k_backsolve(const double *H, int m, int k, const double *gv, double *y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double s = gv[i];
    for (int q = i + 1; q < k; ++q) s -= H[(long)q * (m + 1) + i] * y[q];
    double r = H[(long)i * (m + 1) + i];
    y[i] = r != 0.0 ? s / r : 0.0;
  }
}

int grid_for(long n, int threads) {
  long b = (n + threads - 1) / threads;
  return (int)(b < 1 ? 1 : (b > 2048 ? 2048 : b));
}

}  // namespace

int dot_blocks(long N) {
  long b = (N + 4 * kDotThreads - 1) / (4 * kDotThreads);
  return (int)(b < 1 ? 1 : (b > 304 ? 304 : b));
}

vie_status launch_dots(const double *V, int nv, long ldv, const double *w, long N, double *part,
                       int blocks, cudaStream_t st) {
  k_dots<<<blocks, kDotThreads, 0, st>>>(V, nv, ldv, w, N, part);
  VIE_CHECK_LAUNCH("k_dots");
  return VIE_OK;
}

vie_status launch_dots_last(const double *V, int nv, long ldv, const double *w, long N, double *part,
                            int blocks, int *ticket, double *out1, double *out2, cudaStream_t st) {
  k_dots_last<<<blocks, kDotThreads, 0, st>>>(V, nv, ldv, w, N, part, ticket, out1, out2, nullptr, 0, 0,
                                              nullptr, nullptr, nullptr, nullptr, 0.0, nullptr);
  VIE_CHECK_LAUNCH("k_dots_last");
  return VIE_OK;
}

vie_status launch_norm2_givens(const double *w, long N, double *part, int blocks, int *ticket, double *norm2,
                               double *H, int m, int k, const double *hcol, double *cs, double *sn, double *gv,
                               double bnorm, double *est, cudaStream_t st) {
  k_dots_last<<<blocks, kDotThreads, 0, st>>>(w, 1, N, w, N, part, ticket, norm2, nullptr, H, m, k, hcol, cs, sn,
                                              gv, bnorm, est);
  VIE_CHECK_LAUNCH("k_dots_last");
  return VIE_OK;
}

vie_status launch_dots_finish(const double *part, int blocks, int nv, double *out, int accumulate,
                              cudaStream_t st) {
  k_dots_finish<<<1, 256, 0, st>>>(part, blocks, nv, out, accumulate);
  VIE_CHECK_LAUNCH("k_dots_finish");
  return VIE_OK;
}

vie_status launch_orth_update(const double *V, int nv, long ldv, const double *h, double *w,
                              long N, cudaStream_t st) {
  k_orth_update<<<grid_for(N, 256), 256, 0, st>>>(V, nv, ldv, h, w, N);
  VIE_CHECK_LAUNCH("k_orth_update");
  return VIE_OK;
}

vie_status launch_lincomb_add(const double *V, int nv, long ldv, const double *y, double *x,
                              long N, cudaStream_t st) {
  k_lincomb_add<<<grid_for(N, 256), 256, 0, st>>>(V, nv, ldv, y, x, N);
  VIE_CHECK_LAUNCH("k_lincomb_add");
  return VIE_OK;
}

vie_status launch_scale(const double *x, const double *norm2, int use_sqrt, double *y, long N,
                        cudaStream_t st) {
  k_scale<<<grid_for(N, 256), 256, 0, st>>>(x, norm2, use_sqrt, y, N);
  VIE_CHECK_LAUNCH("k_scale");
  return VIE_OK;
}

vie_status launch_axpby(double a, const double *x, double b, const double *y, double *z, long N,
                        cudaStream_t st) {
  k_axpby<<<grid_for(N, 256), 256, 0, st>>>(a, x, b, y, z, N);
  VIE_CHECK_LAUNCH("k_axpby");
  return VIE_OK;
}

vie_status launch_givens(double *H, int m, int k, const double *hcol, const double *hk1sq,
                         double *cs, double *sn, double *gv, double bnorm, double *est,
                         cudaStream_t st) {
  k_givens<<<1, 32, 0, st>>>(H, m, k, hcol, hk1sq, cs, sn, gv, bnorm, est);
  VIE_CHECK_LAUNCH("k_givens");
  return VIE_OK;
}

vie_status launch_backsolve(const double *H, int m, int k, const double *gv, double *y,
                            cudaStream_t st) {
  k_backsolve<<<1, 32, 0, st>>>(H, m, k, gv, y);
  VIE_CHECK_LAUNCH("k_backsolve");
  return VIE_OK;
}

}  // namespace vie
