// FFT preconditioner of Section 4.4 (Eqs. EQ: FFT and EQ:SOL FFT), 2D.
//
// The medium's coefficients are replaced by their means mu = mean sigma_t and
// mu_s = mean sigma_s.  With constant coefficients the discrete operator is a
// convolution, U - mu_s W * U = b, W the homogeneous medium's matrix A as a
// function of the displacement D (M-iii: h e^{-mu h|D|} / (2 pi |D|), the
// self-cell integral at D = 0; M-ii: e^{-mu h|D|} (h / 2 pi) G(D), G the
// closed-form cell integral).  Extended periodically to an m x m torus (m the
// power of two at or above 2 n: the paper's [0, 2]^2) with the vector
// extended by zero, the operator is diagonal in Fourier space, so
//     z = P F^{-1}( F(P^{-1} b) / lambda ),  lambda = F(delta - mu_s W~).
// W~ is even, so lambda is real; 1 / lambda is computed once on the host in
// FP64 and stored in FP32.
//
// Apply: three launches of length-m complex FFTs in shared memory, one line
// per CTA.  Rows: the n grid rows, zero-extended, forward (decimation in time
// from bit-reversed order).  Columns: each of the m columns (rows past n are
// zero), forward, times 1 / lambda, inverse by decimation in frequency (the
// result lands in bit-reversed order; only the n grid rows are stored).  Rows
// again: inverse, the n grid columns stored in FP64 with the 1 / m^2 of the
// two inverse transforms.  Twiddles e^{-2 pi i k / m} come from a host FP64
// table.  FP32 throughout: a preconditioner of flexible GMRES needs no more.
#include <math.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "vie_internal.cuh"

namespace vie {

namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// decimation in time: x in bit-reversed order in, natural order out
__device__ void fft_dit(float2 *x, int m, const float2 *__restrict__ tw, bool inverse) {
  for (int half = 1; half < m; half <<= 1) {
    const int step = m / (2 * half);
    for (int b = threadIdx.x; b < m / 2; b += blockDim.x) {
      const int pos = b & (half - 1), i = (b - pos) * 2 + pos, j = i + half;
      float2 w = tw[pos * step];
      if (inverse) w.y = -w.y;
      const float2 a = x[i], t = cmul(x[j], w);
      x[i] = make_float2(a.x + t.x, a.y + t.y);
      x[j] = make_float2(a.x - t.x, a.y - t.y);
    }
    __syncthreads();
  }
}

// decimation in frequency: natural order in, bit-reversed order out
__device__ void fft_dif(float2 *x, int m, const float2 *__restrict__ tw, bool inverse) {
  for (int half = m / 2; half >= 1; half >>= 1) {
    const int step = m / (2 * half);
    for (int b = threadIdx.x; b < m / 2; b += blockDim.x) {
      const int pos = b & (half - 1), i = (b - pos) * 2 + pos, j = i + half;
      float2 w = tw[pos * step];
      if (inverse) w.y = -w.y;
      const float2 a = x[i], c = x[j];
      x[i] = make_float2(a.x + c.x, a.y + c.y);
      x[j] = cmul(make_float2(a.x - c.x, a.y - c.y), w);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int bitrev(int i, int logm) { return (int)(__brev((unsigned)i) >> (32 - logm)); }

// row y < n: zero-extended b row, forward transform, into buf[y][0, m)
__global__ void k_fft_rows_fwd(int n, int m, int logm, const double *__restrict__ v,
                               const float2 *__restrict__ tw, float2 *__restrict__ buf) {
  extern __shared__ float2 x[];
  const int y = blockIdx.x;
  for (int i = threadIdx.x; i < m; i += blockDim.x)
    x[bitrev(i, logm)] = make_float2(i < n ? (float)v[(long)y * n + i] : 0.f, 0.f);
  __syncthreads();
  fft_dit(x, m, tw, false);
  for (int i = threadIdx.x; i < m; i += blockDim.x) buf[(long)y * m + i] = x[i];
}

// column kx: rows past n are zero; forward, times 1 / lambda, inverse; rows < n back
__global__ void k_fft_cols(int n, int m, int logm, float2 *__restrict__ buf, const float *__restrict__ inv_lambda,
                           const float2 *__restrict__ tw) {
  extern __shared__ float2 x[];
  const int kx = blockIdx.x;
  for (int i = threadIdx.x; i < m; i += blockDim.x)
    x[bitrev(i, logm)] = i < n ? buf[(long)i * m + kx] : make_float2(0.f, 0.f);
  __syncthreads();
  fft_dit(x, m, tw, false);
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const float s = inv_lambda[(long)i * m + kx];
    x[i] = make_float2(x[i].x * s, x[i].y * s);
  }
  __syncthreads();
  fft_dif(x, m, tw, true);
  for (int i = threadIdx.x; i < n; i += blockDim.x) buf[(long)i * m + kx] = x[bitrev(i, logm)];
}

// row y < n: inverse transform, the n grid columns out in FP64
__global__ void k_fft_rows_inv(int n, int m, int logm, const float2 *__restrict__ buf, const float2 *__restrict__ tw,
                               float scale, double *__restrict__ z) {
  extern __shared__ float2 x[];
  const int y = blockIdx.x;
  for (int i = threadIdx.x; i < m; i += blockDim.x) x[i] = buf[(long)y * m + i];
  __syncthreads();
  fft_dif(x, m, tw, true);
  for (int i = threadIdx.x; i < n; i += blockDim.x) z[(long)y * n + i] = (double)(x[bitrev(i, logm)].x * scale);
}

// ---- host: the symbol in FP64

// in-place radix-2 FFT of a complex FP64 line (forward, e^{-2 pi i k/m});
// w holds e^{-2 pi i k/m} for k < m/2
void host_fft(std::vector<std::complex<double>> &a, const std::vector<std::complex<double>> &w) {
  const size_t m = a.size();
  for (size_t i = 1, j = 0; i < m; ++i) {
    size_t bit = m >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  for (size_t len = 2; len <= m; len <<= 1) {
    const size_t step = m / len;
    for (size_t b = 0; b < m; b += len)
      for (size_t k = 0; k < len / 2; ++k) {
        const std::complex<double> u = a[b + k], t = a[b + k + len / 2] * w[k * step];
        a[b + k] = u + t;
        a[b + k + len / 2] = u - t;
      }
  }
}

// self-cell integral int_{[-h/2,h/2]^2} e^{-mu |z|} / (2 pi |z|) dz: in polar
// coordinates over the square's eight triangles,
//   (4 / pi) int_0^{pi/4} (1 - e^{-mu a / cos t}) / mu dt,  a = h / 2,
// by composite Simpson (the integrand is analytic on the interval)
double host_selfcell(double h, double mu) {
  const int K = 2048;
  const double a = 0.5 * h, L = 0.25 * kPi;
  auto f = [&](double t) {
    const double R = a / cos(t);
    return mu * R < 1e-8 ? R * (1.0 - 0.5 * mu * R) : (1.0 - exp(-mu * R)) / mu;
  };
  double acc = f(0.0) + f(L);
  for (int i = 1; i < K; ++i) acc += (i & 1 ? 4.0 : 2.0) * f(L * i / K);
  return 4.0 / kPi * acc * (L / K) / 3.0;
}

}  // namespace

vie_status fft_prepare(FftPre *fp, int n, double mu, double mu_s, int mii, cudaStream_t st) {
  fft_release(fp);
  int m = 1, logm = 0;
  while (m < 2 * n) {
    m *= 2;
    ++logm;
  }
  if (logm > 12) {
    set_error("vie_set_fft_preconditioner: grid too large (n <= 2048)");
    return VIE_ERR_UNSUPPORTED;
  }
  const double h = 1.0 / n;
  // W~ on the torus, displacement (dx, dy) in [-m/2, m/2)
  std::vector<std::complex<double>> W((size_t)m * m);
  for (int iy = 0; iy < m; ++iy)
    for (int ix = 0; ix < m; ++ix) {
      const int dx = ix < m / 2 ? ix : ix - m, dy = iy < m / 2 ? iy : iy - m;
      const double r = sqrt((double)dx * dx + (double)dy * dy);
      double w;
      if (mii)
        w = exp(-mu * h * r) * h * unit_cell_integral(dx, dy) / (2.0 * kPi);
      else if (dx == 0 && dy == 0)
        w = host_selfcell(h, mu);
      else
        w = h * exp(-mu * h * r) / (2.0 * kPi * r);
      W[(size_t)iy * m + ix] = w;
    }
  std::vector<std::complex<double>> line((size_t)m), wt((size_t)m / 2);
  for (int k = 0; k < m / 2; ++k) wt[k] = std::polar(1.0, -2.0 * kPi * k / m);
  for (int iy = 0; iy < m; ++iy) {
    std::copy(W.begin() + (size_t)iy * m, W.begin() + (size_t)(iy + 1) * m, line.begin());
    host_fft(line, wt);
    std::copy(line.begin(), line.end(), W.begin() + (size_t)iy * m);
  }
  for (int ix = 0; ix < m; ++ix) {
    for (int iy = 0; iy < m; ++iy) line[iy] = W[(size_t)iy * m + ix];
    host_fft(line, wt);
    for (int iy = 0; iy < m; ++iy) W[(size_t)iy * m + ix] = line[iy];
  }
  std::vector<float> inv((size_t)m * m);
  for (size_t i = 0; i < inv.size(); ++i) {
    const double lam = 1.0 - mu_s * W[i].real();  // W~ even: the transform is real
    if (!(lam > 0.0)) {
      set_error("vie_set_fft_preconditioner: the periodic operator is not positive (mean sigma_s > mean "
                "sigma_t?)");
      return VIE_ERR_INVALID_ARG;
    }
    inv[i] = (float)(1.0 / lam);
  }
  std::vector<float2> tw((size_t)m / 2);
  for (int k = 0; k < m / 2; ++k) tw[k] = make_float2((float)wt[k].real(), (float)wt[k].imag());
  VIE_CUDA(vie_malloc((void **)&fp->inv_lambda, sizeof(float) * inv.size()));
  VIE_CUDA(vie_malloc((void **)&fp->tw, sizeof(float2) * tw.size()));
  VIE_CUDA(vie_malloc((void **)&fp->buf, sizeof(float2) * (size_t)n * m));
  VIE_CUDA(cudaMemcpyAsync(fp->inv_lambda, inv.data(), sizeof(float) * inv.size(), cudaMemcpyHostToDevice, st));
  VIE_CUDA(cudaMemcpyAsync(fp->tw, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice, st));
  VIE_CUDA(cudaStreamSynchronize(st));
  const size_t smem = sizeof(float2) * (size_t)m;
  if (smem > 48 * 1024) {
    VIE_TRY(raise_smem_limit((const void *)k_fft_rows_fwd, (size_t)((int)smem)));
    VIE_TRY(raise_smem_limit((const void *)k_fft_cols, (size_t)((int)smem)));
    VIE_TRY(raise_smem_limit((const void *)k_fft_rows_inv, (size_t)((int)smem)));
  }
  fp->n = n;
  fp->m = m;
  fp->logm = logm;
  fp->mu = mu;
  fp->mu_s = mu_s;
  fp->on = 1;
  return VIE_OK;
}

void fft_release(FftPre *fp) {
  if (fp->inv_lambda) vie_free(fp->inv_lambda);
  if (fp->tw) vie_free(fp->tw);
  if (fp->buf) vie_free(fp->buf);
  *fp = FftPre{};
}

vie_status fft_precondition(const FftPre &fp, const double *v, double *z, cudaStream_t st) {
  const int n = fp.n, m = fp.m;
  const int threads = std::min(m / 2, 256);
  const size_t smem = sizeof(float2) * (size_t)m;
  k_fft_rows_fwd<<<n, threads, smem, st>>>(n, m, fp.logm, v, fp.tw, fp.buf);
  VIE_CHECK_LAUNCH("k_fft_rows_fwd");
  k_fft_cols<<<m, threads, smem, st>>>(n, m, fp.logm, fp.buf, fp.inv_lambda, fp.tw);
  VIE_CHECK_LAUNCH("k_fft_cols");
  k_fft_rows_inv<<<n, threads, smem, st>>>(n, m, fp.logm, fp.buf, fp.tw, 1.0f / ((float)m * (float)m), z);
  VIE_CHECK_LAUNCH("k_fft_rows_inv");
  return VIE_OK;
}

}  // namespace vie
