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

// Block sum in a fixed order, valid in thread 0: every thread's value goes to
// shared memory, lane l of warp 0 adds values l, l + 32, ... in turn, and a
// shuffle tree over warp 0 finishes.  GB300's FP64 pipe is narrow, and a
// shuffle tree in every warp cost more FP64 adds than the dot products.
__device__ __forceinline__ double block_sum(double v, double *red) {
  __syncthreads();  // an earlier call may still be reading red
  red[threadIdx.x] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    for (int i = threadIdx.x; i < (int)blockDim.x; i += 32) s += red[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;
}

// part[b * nv + i] = sum over this block's slice of V_i . w
__global__ void __launch_bounds__(kDotThreads) k_dots(const double *__restrict__ V, int nv, long ldv,
                                                      const double *__restrict__ w, long N,
                                                      double *__restrict__ part) {
  __shared__ double red[kDotThreads];
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
  __shared__ double s_inv;  // one square root and divide per block, not per thread
  if (threadIdx.x == 0) {
    const double nrm = use_sqrt ? sqrt(*n2) : *n2;
    s_inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  }
  __syncthreads();
  const double inv = s_inv;
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
  __shared__ double red[kDotThreads];
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

// ---- R solves in lockstep (blockIdx.y = right-hand side r).  Each kernel
// does for every r with act[r] != 0 what its single-vector form above does,
// in the same order, so a batched solve of one right-hand side reproduces
// the single solve's arithmetic.  Vector i of r's basis sits at
// V + r ldv_r + i N; r's small arrays at r times their length.

// out1[r][v] = V_r[v] . w_r (v < nv) and/or out2[r][v] += it; with gvmode the
// single dot (nv = 1, V = w) is ||w_r||^2 and the last block of r then takes
// r's Givens step of column k.
__global__ void __launch_bounds__(kDotThreads) k_bdots_last(KBatch b, const double *__restrict__ V, long ldv_r,
                                                            int nv, const double *__restrict__ w, long ldw_r,
                                                            double *out1, double *out2, int gvmode, int k) {
  __shared__ double red[kDotThreads];
  __shared__ int last;
  const int r = blockIdx.y;
  if (!b.act[r]) return;
  const long N = b.N;
  const int m = b.m;
  const double *Vr = V + (long)r * ldv_r;
  const double *wr = w + (long)r * ldw_r;
  double *part = b.part + (long)r * gridDim.x * (m + 1);
  const long stride = (long)gridDim.x * blockDim.x;
  const long i0 = blockIdx.x * (long)blockDim.x + threadIdx.x;
  for (int v = 0; v < nv; ++v) {
    const double *x = Vr + (long)v * N;
    double sum = 0.0;
    for (long i = i0; i < N; i += stride) sum += x[i] * wr[i];
    sum = block_sum(sum, red);
    if (threadIdx.x == 0) part[(long)blockIdx.x * nv + v] = sum;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(b.ticket + r, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    double sum = 0.0;
    for (int q = 0; q < (int)gridDim.x; ++q) sum += __ldcg(part + (long)q * nv + v);
    if (out1) out1[(long)r * (m + 1) + v] = sum;
    if (out2) out2[(long)r * (m + 1) + v] += sum;
    if (gvmode && v == 0) {
      b.scal[r * 8 + 2] = sum;
      givens_step(b.H + (long)r * (m + 1) * m, m, k, b.hcol + (long)r * (m + 1), sum, b.cs + (long)r * m,
                  b.sn + (long)r * m, b.gv + (long)r * (m + 1), b.bnorm[r], b.scal + r * 8 + 3);
    }
  }
  if (threadIdx.x == 0) b.ticket[r] = 0;
}

// ||w_r||^2 into scal[r][slot] (no Givens step)
__global__ void __launch_bounds__(kDotThreads) k_bnorm2(KBatch b, const double *__restrict__ w, long ldw_r,
                                                        int slot) {
  __shared__ double red[kDotThreads];
  __shared__ int last;
  const int r = blockIdx.y;
  if (!b.act[r]) return;
  const long N = b.N;
  const double *wr = w + (long)r * ldw_r;
  double *part = b.part + (long)r * gridDim.x * (b.m + 1);
  double sum = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x)
    sum += wr[i] * wr[i];
  sum = block_sum(sum, red);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = sum;
    __threadfence();
    last = atomicAdd(b.ticket + r, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)gridDim.x; ++q) t += __ldcg(part + q);
    b.scal[r * 8 + slot] = t;
    b.ticket[r] = 0;
  }
}

// w_r -= sum_{v < nv} h_r[v] V_r[v]
__global__ void k_borth_update(KBatch b, const double *__restrict__ V, long ldv_r, int nv,
                               const double *__restrict__ h, double *__restrict__ w, long ldw_r) {
  const int r = blockIdx.y;
  if (!b.act[r]) return;
  const long N = b.N;
  const double *Vr = V + (long)r * ldv_r;
  const double *hr = h + (long)r * (b.m + 1);
  double *wr = w + (long)r * ldw_r;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    double acc = wr[i];
    for (int v = 0; v < nv; ++v) acc -= hr[v] * Vr[(long)v * N + i];
    wr[i] = acc;
  }
}

// y_r = x_r / norm_r, norm_r = sqrt(scal[r][slot]) if use_sqrt else scal[r][slot]
__global__ void k_bscale(KBatch b, const double *__restrict__ x, long ldx_r, int slot, int use_sqrt,
                         double *__restrict__ y, long ldy_r) {
  const int r = blockIdx.y;
  if (!b.act[r]) return;
  __shared__ double s_inv;  // one square root and divide per block, not per thread
  if (threadIdx.x == 0) {
    const double n2 = b.scal[r * 8 + slot];
    const double nrm = use_sqrt ? sqrt(n2) : n2;
    s_inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  }
  __syncthreads();
  const double inv = s_inv;
  const double *xr = x + (long)r * ldx_r;
  double *yr = y + (long)r * ldy_r;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < b.N; i += (long)gridDim.x * blockDim.x)
    yr[i] = xr[i] * inv;
}

// z_r = a x_r + c y_r
__global__ void k_baxpby(KBatch b, double a, const double *__restrict__ x, long ldx_r, double c,
                         const double *__restrict__ y, long ldy_r, double *__restrict__ z, long ldz_r) {
  const int r = blockIdx.y;
  if (!b.act[r]) return;
  const double *xr = x + (long)r * ldx_r, *yr = y + (long)r * ldy_r;
  double *zr = z + (long)r * ldz_r;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < b.N; i += (long)gridDim.x * blockDim.x)
    zr[i] = a * xr[i] + c * yr[i];
}

// r's triangular solve of its kk[r] columns (one thread per r), then x_r +=
// sum_{v < kk[r]} y_r[v] B_r[v] (B: V or the flexible directions Z)
__global__ void k_bbacksolve(KBatch b, const int *__restrict__ kk) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= b.R || !b.act[r]) return;
  const int m = b.m, k = kk[r];
  const double *H = b.H + (long)r * (m + 1) * m, *gv = b.gv + (long)r * (m + 1);
  double *y = b.yv + (long)r * m;
  for (int i = k - 1; i >= 0; --i) {
    double s = gv[i];
    for (int q = i + 1; q < k; ++q) s -= H[(long)q * (m + 1) + i] * y[q];
    const double d = H[(long)i * (m + 1) + i];
    y[i] = d != 0.0 ? s / d : 0.0;
  }
}

__global__ void k_blincomb_add(KBatch b, const double *__restrict__ B, long ldb_r, const int *__restrict__ kk,
                               double *__restrict__ x, long ldx_r) {
  const int r = blockIdx.y;
  if (!b.act[r]) return;
  const int k = kk[r];
  const double *Br = B + (long)r * ldb_r, *y = b.yv + (long)r * b.m;
  double *xr = x + (long)r * ldx_r;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < b.N; i += (long)gridDim.x * blockDim.x) {
    double acc = xr[i];
    for (int v = 0; v < k; ++v) acc += y[v] * Br[(long)v * b.N + i];
    xr[i] = acc;
  }
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

// ---- lockstep batch launchers (KBatch: vie_internal.cuh)
static dim3 bgrid(long N, int R, int threads) {
  long gx = (N + threads - 1) / threads;
  gx = gx < 1 ? 1 : (gx > 2048 / (R < 8 ? R : 8) ? 2048 / (R < 8 ? R : 8) : gx);
  return dim3((unsigned)gx, (unsigned)R);
}

vie_status launch_bdots(const KBatch &b, const double *V, long ldv_r, int nv, const double *w, long ldw_r,
                        double *out1, double *out2, cudaStream_t st) {
  k_bdots_last<<<dim3((unsigned)b.blocks, (unsigned)b.R), kDotThreads, 0, st>>>(b, V, ldv_r, nv, w, ldw_r, out1,
                                                                                out2, 0, 0);
  VIE_CHECK_LAUNCH("k_bdots_last");
  return VIE_OK;
}

vie_status launch_bnorm2_givens(const KBatch &b, const double *w, long ldw_r, int k, cudaStream_t st) {
  k_bdots_last<<<dim3((unsigned)b.blocks, (unsigned)b.R), kDotThreads, 0, st>>>(b, w, ldw_r, 1, w, ldw_r,
                                                                                nullptr, nullptr, 1, k);
  VIE_CHECK_LAUNCH("k_bdots_last");
  return VIE_OK;
}

vie_status launch_bnorm2(const KBatch &b, const double *w, long ldw_r, int slot, cudaStream_t st) {
  k_bnorm2<<<dim3((unsigned)b.blocks, (unsigned)b.R), kDotThreads, 0, st>>>(b, w, ldw_r, slot);
  VIE_CHECK_LAUNCH("k_bnorm2");
  return VIE_OK;
}

vie_status launch_borth_update(const KBatch &b, const double *V, long ldv_r, int nv, const double *h, double *w,
                               long ldw_r, cudaStream_t st) {
  k_borth_update<<<bgrid(b.N, b.R, 256), 256, 0, st>>>(b, V, ldv_r, nv, h, w, ldw_r);
  VIE_CHECK_LAUNCH("k_borth_update");
  return VIE_OK;
}

vie_status launch_bscale(const KBatch &b, const double *x, long ldx_r, int slot, int use_sqrt, double *y,
                         long ldy_r, cudaStream_t st) {
  k_bscale<<<bgrid(b.N, b.R, 256), 256, 0, st>>>(b, x, ldx_r, slot, use_sqrt, y, ldy_r);
  VIE_CHECK_LAUNCH("k_bscale");
  return VIE_OK;
}

vie_status launch_baxpby(const KBatch &b, double a, const double *x, long ldx_r, double c, const double *y,
                         long ldy_r, double *z, long ldz_r, cudaStream_t st) {
  k_baxpby<<<bgrid(b.N, b.R, 256), 256, 0, st>>>(b, a, x, ldx_r, c, y, ldy_r, z, ldz_r);
  VIE_CHECK_LAUNCH("k_baxpby");
  return VIE_OK;
}

vie_status launch_bupdate(const KBatch &b, const double *B, long ldb_r, const int *kk, double *x, long ldx_r,
                          cudaStream_t st) {
  k_bbacksolve<<<(b.R + 31) / 32, 32, 0, st>>>(b, kk);
  VIE_CHECK_LAUNCH("k_bbacksolve");
  k_blincomb_add<<<bgrid(b.N, b.R, 256), 256, 0, st>>>(b, B, ldb_r, kk, x, ldx_r);
  VIE_CHECK_LAUNCH("k_blincomb_add");
  return VIE_OK;
}

}  // namespace vie
