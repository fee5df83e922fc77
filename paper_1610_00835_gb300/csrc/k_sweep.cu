// Step two of Algorithm 1 (S.3): the scattering-free transport solve along
// backward characteristics, Eq. EQ:ERT Intgrl with q = Q = sigma_s U + f:
//   Phi(x, v) = int_0^L exp(-int_0^l sigma_t(x - l' v) dl') Q(x - l v) dl,
// L the distance from x to the boundary along -v.  One thread per
// (direction, cell) ray.  The ray is cut into ns = ceil(2 n L - 1e-6) equal
// steps (at most h/2 each); the step count is decided in FP64 with
// correctly rounded operations so that it does not depend on instruction
// selection.  On each step sigma_t~ and Q~ (bilinear / trilinear in the cell
// values, clamped to the hull of the centres) are frozen at the step midpoint
// and the step is integrated exactly:
//   Phi += e^{-tau} Q~ (1 - e^{-sigma~ D}) / sigma~,  tau += sigma~ D.
#include <math.h>

#include "vie_internal.cuh"

namespace vie {

namespace {

// Q = sigma_s U + f on the padded lattice (edge copies in the pad).
__global__ void k_make_q(int dim, int n, const double *__restrict__ ss, const double *__restrict__ U,
                         const double *__restrict__ f, float *__restrict__ q) {
  const int P = n + 1;
  long total = dim == 2 ? (long)P * P : (long)P * P * P;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    long px = min(i % P, (long)n - 1), py = min((i / P) % P, (long)n - 1);
    long pz = dim == 3 ? min(i / ((long)P * P), (long)n - 1) : 0;
    long j = (pz * n + py) * n + px;
    q[i] = (float)(ss[j] * U[j] + f[j]);
  }
}

// Interpolate the padded lattice `s` at lattice coordinate u (clamped to
// [0, n-1] per axis).
template <int DIM>
__device__ __forceinline__ float interp(const float *__restrict__ s, int n, int P, const float *u) {
  int i0[3];
  float a[3];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    float c = fminf(fmaxf(u[d], 0.f), (float)(n - 1));
    float fl = floorf(c);
    i0[d] = (int)fl;
    a[d] = c - fl;
  }
  if (DIM == 2) {
    const float *r0 = s + i0[1] * P + i0[0];
    float lo = fmaf(a[0], __ldg(r0 + 1) - __ldg(r0), __ldg(r0));
    float hi = fmaf(a[0], __ldg(r0 + P + 1) - __ldg(r0 + P), __ldg(r0 + P));
    return fmaf(a[1], hi - lo, lo);
  } else {
    const float *r0 = s + (i0[2] * P + i0[1]) * P + i0[0];
    const float *r1 = r0 + P * P;
    float a0 = fmaf(a[0], __ldg(r0 + 1) - __ldg(r0), __ldg(r0));
    float a1 = fmaf(a[0], __ldg(r0 + P + 1) - __ldg(r0 + P), __ldg(r0 + P));
    float b0 = fmaf(a[0], __ldg(r1 + 1) - __ldg(r1), __ldg(r1));
    float b1 = fmaf(a[0], __ldg(r1 + P + 1) - __ldg(r1 + P), __ldg(r1 + P));
    float c0 = fmaf(a[1], a1 - a0, a0);
    float c1 = fmaf(a[1], b1 - b0, b0);
    return fmaf(a[2], c1 - c0, c0);
  }
}

template <int DIM>
__global__ void __launch_bounds__(256) k_sweep(int n, const float *__restrict__ sig,
                                               const float *__restrict__ q,
                                               const float *__restrict__ dirs, int M,
                                               float *__restrict__ Phi) {
  const long N = DIM == 2 ? (long)n * n : (long)n * n * n;
  const long rays = N * (long)M;
  const int P = n + 1;
  const double h = 1.0 / n;
  for (long id = blockIdx.x * (long)blockDim.x + threadIdx.x; id < rays;
       id += (long)gridDim.x * blockDim.x) {
    const long j = id % N;
    const int m = (int)(id / N);
    long idx[3] = {j % n, (j / n) % n, DIM == 3 ? j / ((long)n * n) : 0};
    double x[3], v[3];
    double L = INFINITY;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      x[d] = __dmul_rn(__dadd_rn((double)idx[d], 0.5), h);
      v[d] = (double)dirs[m * DIM + d];
      if (v[d] > 0.0) L = fmin(L, __ddiv_rn(x[d], v[d]));
      else if (v[d] < 0.0) L = fmin(L, __ddiv_rn(__dsub_rn(1.0, x[d]), -v[d]));
    }
    // |v| = 1 gives L <= sqrt(dim); the cap only bounds the loop for
    // directions that are not unit vectors (undefined input).
    if (!(L <= 2.0)) L = 2.0;
    double steps = ceil(__dsub_rn(__dmul_rn(L, 2.0 * n), 1e-6));
    long ns = steps < 1.0 ? 1 : (long)steps;
    const float dl = (float)(L / (double)ns);
    // Lattice coordinates of the midpoints: u(s) = x/h - 1/2 - (s + 1/2) dl v / h.
    float u0[3], du[3];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      u0[d] = (float)(x[d] * n - 0.5);
      du[d] = (float)(-(double)dl * v[d] * n);
    }
    float tau = 0.f, acc = 0.f;
    for (long s = 0; s < ns; ++s) {
      const float t = (float)s + 0.5f;
      float u[3];
#pragma unroll
      for (int d = 0; d < DIM; ++d) u[d] = fmaf(t, du[d], u0[d]);
      const float sg = interp<DIM>(sig, n, P, u);
      const float qq = interp<DIM>(q, n, P, u);
      const float seg = sg > 0.f ? -expm1f(-sg * dl) / sg : dl;
      acc = fmaf(expf(-tau) * qq, seg, acc);
      tau = fmaf(sg, dl, tau);
    }
    Phi[(long)m * N + j] = acc;
  }
}

int grid_for(long n, int threads) {
  long b = (n + threads - 1) / threads;
  return (int)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

}  // namespace

vie_status launch_make_q(int dim, int n, const double *sigma_s, const double *U, const double *f,
                         float *qpad, cudaStream_t st) {
  long P = n + 1;
  long total = dim == 2 ? P * P : P * P * P;
  k_make_q<<<grid_for(total, 256), 256, 0, st>>>(dim, n, sigma_s, U, f, qpad);
  VIE_CHECK_LAUNCH("k_make_q");
  return VIE_OK;
}

vie_status launch_sweep(int dim, int n, const float *sigpad, const float *qpad, const float *dirs,
                        int M, float *Phi, cudaStream_t st) {
  long N = dim == 2 ? (long)n * n : (long)n * n * n;
  long rays = N * M;
  if (dim == 2)
    k_sweep<2><<<grid_for(rays, 256), 256, 0, st>>>(n, sigpad, qpad, dirs, M, Phi);
  else
    k_sweep<3><<<grid_for(rays, 256), 256, 0, st>>>(n, sigpad, qpad, dirs, M, Phi);
  VIE_CHECK_LAUNCH("k_sweep");
  return VIE_OK;
}

}  // namespace vie
