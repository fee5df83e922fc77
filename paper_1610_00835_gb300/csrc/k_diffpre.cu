// Diffusion preconditioner of Section 4.4 (Eq. EQ:DA), 2D.
//
// Diffusion approximation on the unit square: -div(kappa grad U) + mu_a U = f
// with kappa = 1 / (d mu), mu_a = mu - mu_s, and U + l dU/dn = 0 on the
// boundary, l = 2 / (d mu) (d = 2).  Second-order finite volumes on the n x n
// cells: an interior face carries the harmonic mean of its cells' kappa and
// the flux kappa_f (U_c - U_nb) / h; a boundary face eliminates the boundary
// value through the Robin condition, leaving the outward flux
// 2 kappa_c U_c / (h + 2 l_c).  Per cell area, row c of D is
//     diag_c U_c - sum_nb a_nb U_nb,  a_nb = kappa_f / h^2,
//     diag_c = mu_a,c + sum a_nb + (boundary faces) 2 kappa_c / (h (h + 2 l_c)).
//
// As the right preconditioner of (I - K) U = b it applies
//     M(r) = r + D^{-1}(sigma_s r)
// (the diffusion limit of A is (D + Sigma_s)^{-1}, so (I - A Sigma_s)^{-1} is
// close to I + D^{-1} Sigma_s), with D^{-1} one V-cycle of geometric
// multigrid from a zero guess: levels n, n/2, ... while the size is even and
// above 8 (coarse mu and mu_s the means of the 2 x 2 children, the operator
// rediscretised); red-black Gauss-Seidel, 2 sweeps before and after the
// correction; restriction = mean of the children's residuals; bilinear
// prolongation in the cell centres; 200 red-black sweeps on the coarsest grid
// in one CTA.  FP64 (the grids are small).  The V-cycle runs on fixed
// buffers, so it is captured once into a CUDA graph; an application is the
// source kernel, the graph and the finishing kernel.
#include <math.h>

#include <algorithm>
#include <vector>

#include "vie_internal.cuh"

namespace vie {

namespace {

constexpr int kPre = 2, kPost = 2, kCoarseSweeps = 200;
constexpr int kT = 256;

__device__ __forceinline__ double neighbour_sum(const double *__restrict__ c, const double *__restrict__ u, int n,
                                               long N, int ix, int iy, long j) {
  double s = 0.0;
  if (ix > 0) s += c[N + j] * u[j - 1];
  if (ix < n - 1) s += c[2 * N + j] * u[j + 1];
  if (iy > 0) s += c[3 * N + j] * u[j - n];
  if (iy < n - 1) s += c[4 * N + j] * u[j + n];
  return s;
}

// one colour of a red-black Gauss-Seidel sweep (red: ix + iy even); plane 5
// of c holds 1 / diag
__global__ void k_dp_rbgs(int n, const double *__restrict__ c, const double *__restrict__ f, double *__restrict__ u,
                          int colour) {
  const long N = (long)n * n;
  for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < N; j += (long)gridDim.x * blockDim.x) {
    const int ix = (int)(j % n), iy = (int)(j / n);
    if (((ix + iy) & 1) != colour) continue;
    u[j] = (f[j] + neighbour_sum(c, u, n, N, ix, iy, j)) * c[5 * N + j];
  }
}

// f_coarse = mean over the 2 x 2 children of the fine residual f - D u
__global__ void k_dp_restrict(int n, const double *__restrict__ c, const double *__restrict__ f,
                              const double *__restrict__ u, double *__restrict__ fc) {
  const int nc = n / 2;
  const long N = (long)n * n, Nc = (long)nc * nc;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < Nc; t += (long)gridDim.x * blockDim.x) {
    const int I = (int)(t % nc), J = (int)(t / nc);
    double acc = 0.0;
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        const int ix = 2 * I + a, iy = 2 * J + b;
        const long j = (long)iy * n + ix;
        acc += f[j] - (c[j] * u[j] - neighbour_sum(c, u, n, N, ix, iy, j));
      }
    fc[t] = 0.25 * acc;
  }
}

// u_fine += bilinear interpolation of the coarse correction (a neighbour
// outside the coarse grid replaced by the coarse cell itself)
__global__ void k_dp_prolong(int nc, const double *__restrict__ e, double *__restrict__ u) {
  const int n = 2 * nc;
  const long N = (long)n * n;
  for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < N; j += (long)gridDim.x * blockDim.x) {
    const int fx = (int)(j % n), fy = (int)(j / n);
    const int I = fx >> 1, J = fy >> 1;
    const int I2 = (fx & 1) ? min(I + 1, nc - 1) : max(I - 1, 0);
    const int J2 = (fy & 1) ? min(J + 1, nc - 1) : max(J - 1, 0);
    u[j] += (9.0 * e[(long)J * nc + I] + 3.0 * e[(long)J * nc + I2] + 3.0 * e[(long)J2 * nc + I] +
             e[(long)J2 * nc + I2]) / 16.0;
  }
}

__global__ void k_dp_zero(long N, double *__restrict__ u) {
  for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < N; j += (long)gridDim.x * blockDim.x) u[j] = 0.0;
}

// the coarsest grid: zero guess, kCoarseSweeps red-black sweeps, one CTA
__global__ void k_dp_coarse(int n, const double *__restrict__ c, const double *__restrict__ f, double *__restrict__ u) {
  const long N = (long)n * n;
  for (long j = threadIdx.x; j < N; j += blockDim.x) u[j] = 0.0;
  __syncthreads();
  for (int s = 0; s < kCoarseSweeps; ++s)
    for (int colour = 0; colour < 2; ++colour) {
      for (long j = threadIdx.x; j < N; j += blockDim.x) {
        const int ix = (int)(j % n), iy = (int)(j / n);
        if (((ix + iy) & 1) == colour) u[j] = (f[j] + neighbour_sum(c, u, n, N, ix, iy, j)) * c[5 * N + j];
      }
      __syncthreads();
    }
}

__global__ void k_dp_source(long N, const double *__restrict__ ss, const double *__restrict__ v,
                            double *__restrict__ f) {
  for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < N; j += (long)gridDim.x * blockDim.x)
    f[j] = ss[j] * v[j];
}

__global__ void k_dp_finish(long N, const double *__restrict__ v, const double *__restrict__ e,
                            double *__restrict__ z) {
  for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < N; j += (long)gridDim.x * blockDim.x)
    z[j] = v[j] + e[j];
}

int blocks_for(long N) { return (int)std::max(1L, std::min((N + kT - 1) / kT, 2048L)); }

// the coefficient planes of an n x n level with cell values mu, mu_a (FP64, host)
void level_coefficients(int n, const std::vector<double> &mu, const std::vector<double> &mua,
                        std::vector<double> &c) {
  const long N = (long)n * n;
  const double h = 1.0 / n;
  c.assign(6 * N, 0.0);
  for (int iy = 0; iy < n; ++iy)
    for (int ix = 0; ix < n; ++ix) {
      const long j = (long)iy * n + ix;
      const double kc = 1.0 / (2.0 * mu[j]), lc = 2.0 / (2.0 * mu[j]);
      double diag = mua[j];
      const int nx[4] = {ix - 1, ix + 1, ix, ix}, ny[4] = {iy, iy, iy - 1, iy + 1};
      for (int q = 0; q < 4; ++q) {
        if (nx[q] >= 0 && nx[q] < n && ny[q] >= 0 && ny[q] < n) {
          const double kn = 1.0 / (2.0 * mu[(long)ny[q] * n + nx[q]]);
          const double a = 2.0 * kc * kn / (kc + kn) / (h * h);
          c[(q + 1) * N + j] = a;
          diag += a;
        } else {
          diag += 2.0 * kc / (h * (h + 2.0 * lc));
        }
      }
      c[j] = diag;
      c[5 * N + j] = 1.0 / diag;
    }
}

// the V-cycle on the level buffers (kernels only; captured into the graph)
cudaError_t enqueue_vcycle(const DiffPre &dp, cudaStream_t st, int *kernels) {
  const DiffLevel *lv = dp.lv;
  const int L = dp.L;
  int k = 0;
  for (int l = 0; l + 1 < L; ++l) {
    const long N = (long)lv[l].n * lv[l].n;
    k_dp_zero<<<blocks_for(N), kT, 0, st>>>(N, lv[l].u);
    ++k;
    for (int s = 0; s < kPre; ++s)
      for (int colour = 0; colour < 2; ++colour, ++k)
        k_dp_rbgs<<<blocks_for(N), kT, 0, st>>>(lv[l].n, lv[l].c, lv[l].f, lv[l].u, colour);
    k_dp_restrict<<<blocks_for(N / 4), kT, 0, st>>>(lv[l].n, lv[l].c, lv[l].f, lv[l].u, lv[l + 1].f);
    ++k;
  }
  {
    // one CTA just large enough for the coarsest grid: its barriers stay cheap
    const long Nc = (long)lv[L - 1].n * lv[L - 1].n;
    const int threads = (int)std::min(1024L, std::max(32L, (Nc + 31) / 32 * 32));
    k_dp_coarse<<<1, threads, 0, st>>>(lv[L - 1].n, lv[L - 1].c, lv[L - 1].f, lv[L - 1].u);
  }
  ++k;
  for (int l = L - 2; l >= 0; --l) {
    const long N = (long)lv[l].n * lv[l].n;
    k_dp_prolong<<<blocks_for(N), kT, 0, st>>>(lv[l + 1].n, lv[l + 1].u, lv[l].u);
    ++k;
    for (int s = 0; s < kPost; ++s)
      for (int colour = 0; colour < 2; ++colour, ++k)
        k_dp_rbgs<<<blocks_for(N), kT, 0, st>>>(lv[l].n, lv[l].c, lv[l].f, lv[l].u, colour);
  }
  *kernels = k;
  return cudaGetLastError();
}

}  // namespace

vie_status diffusion_prepare(DiffPre *dp, int n, const double *sigma_t, const double *sigma_s,
                             const double *sigma_s_dev, cudaStream_t st) {
  diffusion_release(dp);
  const long N = (long)n * n;
  std::vector<double> mu(sigma_t, sigma_t + N), mua((size_t)N);
  for (long j = 0; j < N; ++j) {
    if (!(sigma_t[j] > 0.0)) {
      set_error("vie_set_diffusion_preconditioner: sigma_t must be > 0 in every cell (kappa = 1 / (2 sigma_t))");
      return VIE_ERR_INVALID_ARG;
    }
    mua[j] = sigma_t[j] - sigma_s[j];
  }
  std::vector<double> c;
  int ln = n;
  for (;;) {
    level_coefficients(ln, mu, mua, c);
    const long M = (long)ln * ln;
    DiffLevel &L = dp->lv[dp->L++];  // owned by dp from here: released on failure
    L.n = ln;
    VIE_CUDA(vie_malloc((void **)&L.c, sizeof(double) * 6 * M));
    VIE_CUDA(vie_malloc((void **)&L.f, sizeof(double) * M));
    VIE_CUDA(vie_malloc((void **)&L.u, sizeof(double) * M));
    VIE_CUDA(cudaMemcpyAsync(L.c, c.data(), sizeof(double) * 6 * M, cudaMemcpyHostToDevice, st));
    VIE_CUDA(cudaStreamSynchronize(st));
    if (ln % 2 || ln <= 8 || dp->L == kDiffMaxLevels) break;
    const int nc = ln / 2;
    std::vector<double> mc((size_t)nc * nc), ac((size_t)nc * nc);
    for (int J = 0; J < nc; ++J)
      for (int I = 0; I < nc; ++I) {
        const long a = (long)(2 * J) * ln + 2 * I, b = a + ln;
        mc[(long)J * nc + I] = 0.25 * (mu[a] + mu[b] + mu[a + 1] + mu[b + 1]);
        ac[(long)J * nc + I] = 0.25 * (mua[a] + mua[b] + mua[a + 1] + mua[b + 1]);
      }
    mu.swap(mc);
    mua.swap(ac);
    ln = nc;
  }
  dp->ss = sigma_s_dev;
  dp->n = n;
  // the V-cycle as a graph on a private capture stream
  VIE_CUDA(cudaStreamCreateWithFlags(&dp->cap, cudaStreamNonBlocking));
  VIE_CUDA(cudaStreamBeginCapture(dp->cap, cudaStreamCaptureModeThreadLocal));
  int kernels = 0;
  const cudaError_t ek = enqueue_vcycle(*dp, dp->cap, &kernels);
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(dp->cap, &graph);
  if (ek != cudaSuccess || ec != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(ek != cudaSuccess ? ek : ec, "diffusion V-cycle capture");
  }
  dp->graph = graph;
  VIE_CUDA(cudaGraphInstantiate(&dp->exec, graph, 0));
  dp->graph_kernels = kernels;
  dp->on = 1;
  return VIE_OK;
}

void diffusion_release(DiffPre *dp) {
  if (dp->exec) cudaGraphExecDestroy(dp->exec);
  if (dp->graph) cudaGraphDestroy(dp->graph);
  if (dp->cap) cudaStreamDestroy(dp->cap);
  for (int l = 0; l < dp->L; ++l) {
    if (dp->lv[l].c) vie_free(dp->lv[l].c);
    if (dp->lv[l].f) vie_free(dp->lv[l].f);
    if (dp->lv[l].u) vie_free(dp->lv[l].u);
  }
  *dp = DiffPre{};
}

vie_status diffusion_precondition(const DiffPre &dp, const double *v, double *z, cudaStream_t st) {
  const DiffLevel *lv = dp.lv;
  const long N = (long)dp.n * dp.n;
  k_dp_source<<<blocks_for(N), kT, 0, st>>>(N, dp.ss, v, lv[0].f);
  VIE_CHECK_LAUNCH("k_dp_source");
  VIE_CUDA(cudaGraphLaunch(dp.exec, st));
  for (int i = 0; i < dp.graph_kernels; ++i) count_launch();
  k_dp_finish<<<blocks_for(N), kT, 0, st>>>(N, v, lv[0].u, z);
  VIE_CHECK_LAUNCH("k_dp_finish");
  return VIE_OK;
}

}  // namespace vie
