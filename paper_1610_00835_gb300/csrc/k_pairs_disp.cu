// Displacement-major pair kernel: 2D, FP32 tiles, S = 64 march steps.
//
// It computes the operator of k_apply.cu (Section 2, Eq. EQ:Kernel; Section
// 3.2, M-iii): y_j = sum_{k != j} A_jk s_k.  On a uniform grid the segment
// from cell j to cell j + D (D = (dx, dy) in cells) has its midpoint samples
// at u_j + (i + 1/2) D / S: their integer parts and bilinear weights depend on
// D and i only.  A warp therefore takes one displacement D and a block of
// 32 x 8 targets (32 consecutive x per warp, 8 consecutive y per thread):
// per sample, one thread x-interpolates the 9 lattice rows its 8 targets
// touch (the two rows of target q + 1 overlap those of target q) and
// combines neighbouring rows with the warp-uniform y weight.
//
// Work units are (D, 32 x 8 block of the targets j with j + D inside the
// grid) for D in a half plane (dy > 0, or dy = 0 and dx > 0): A_jk = A_kj, so
// each unordered pair is marched once and feeds y_j (weight s_{j+D}) and
// y_{j+D} (weight s_j).  Units are sorted by the size of their displacement's
// rectangle, largest first, and warps take them four at a time from a global
// counter.  Each CTA sums into a private copy of y in shared memory held in
// 64-bit fixed point: every term w s is rounded once to a multiple of
// 1/scale, scale the power of two at or below 2^62 / (max|s| R) with R a
// bound on every row sum of A,
// and integer atomic adds are exact in any order.  The result is therefore
// bitwise reproducible whatever the schedule, and the accumulation error is
// below N 2^-63 max|s| R.  Each CTA writes its copy (int64) to its
// partial-sum slot; k_disp_reduce adds the slots in int64 (exact, since the
// sum of the magnitudes of all terms of a target is below 2^62), converts
// once to FP64 and adds the self cell.
//
// Rows of targets beyond the rectangle (ragged blocks) are computed and
// discarded; the lattice carries 8 extra rows so that their samples stay in
// bounds, and lanes beyond it use the last valid column.
#include <math.h>

#include <algorithm>
#include <vector>

#include "march.cuh"
#include "vie_internal.cuh"

namespace vie {

namespace {

using namespace march;

constexpr int kR = 8;          // targets per thread (stacked in y)
constexpr int kThreads = 1024;
constexpr int kExtraRows = 8;

struct DispArgs {
  const float *lat;            // [(n + 1 + kExtraRows)][ldp] padded sigma_t, ldp = n + 1
  const float *src;            // s_k, FP32 [N]
  unsigned *smax;              // bits of max |s_k| (set by the source kernel)
  double *scale_out;           // fixed-point scale of this apply (for the reduce)
  double rbound;               // bound on sum_k A_jk for every j
  double *partial;             // [gridDim.x][N]
  const short4 *units;         // (dx, dy, bx, by)
  int *counter;                // [2]
  long n_units;
  int n, ldp;
  long lat_elems;
  float tau_scale2, wcoef, h;
};

template <int OFF>
__device__ __forceinline__ float lds1(unsigned addr) {
  float v;
  asm("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(addr), "n"(OFF));
  return v;
}

// L[r] = x-interpolation of lattice row (row of addr) + r, r < R; rows LDP floats apart.
template <int LDP, int R>
struct Rows {
  static __device__ __forceinline__ void load(unsigned addr, float ax, float *L) {
    Rows<LDP, R - 1>::load(addr, ax, L);
    const float v0 = lds1<4 * LDP * (R - 1)>(addr), v1 = lds1<4 * LDP * (R - 1) + 4>(addr);
    L[R - 1] = fmaf(ax, v1 - v0, v0);
  }
};
template <int LDP>
struct Rows<LDP, 0> {
  static __device__ __forceinline__ void load(unsigned, float, float *) {}
};

template <int LDP>
__global__ void __launch_bounds__(kThreads, 1) k_pairs_disp(DispArgs a) {
  extern __shared__ float4 smem4[];
  unsigned long long *ysh = reinterpret_cast<unsigned long long *>(smem4);  // [N] fixed point
  const int n = a.n;
  const long N = (long)n * n;
  float *lat = reinterpret_cast<float *>(ysh + N + (N & 1));  // 16-byte aligned for float4 staging
  const int tid = threadIdx.x, lane = tid & 31;
  {
    const float4 *g4 = reinterpret_cast<const float4 *>(a.lat);
    float4 *l4 = reinterpret_cast<float4 *>(lat);
    const long n4 = a.lat_elems / 4;
    for (long i = tid; i < n4; i += kThreads) l4[i] = g4[i];
    for (long i = n4 * 4 + tid; i < a.lat_elems; i += kThreads) lat[i] = a.lat[i];
    for (long i = tid; i < N; i += kThreads) ysh[i] = 0ull;
  }
  __syncthreads();
  // power-of-two scale: 2^k <= 2^62 / (max|s| R), so w * scale is exact
  const float smax = __uint_as_float(*a.smax);
  const double scale_d =
      smax > 0.f ? ldexp(1.0, ilogb(4.611686018427387904e18 / ((double)smax * a.rbound))) : 1.0;
  const float scale = (float)scale_d;
  const int ldp = LDP > 0 ? LDP : a.ldp;
  const unsigned lat_base = (unsigned)__cvta_generic_to_shared(lat);
  // element (x, y) at lat_base + 4 (x + ldp y); x, y taken as biased float bits
  const unsigned base = lat_base - 4u * kTwo23Bits * (1u + (unsigned)ldp);
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
    const short4 un = a.units[u0++];
    const int dx = un.x, dy = un.y;
    const int xlo = dx < 0 ? -dx : 0, xhi = dx > 0 ? n - dx : n;
    const int ylo = dy < 0 ? -dy : 0, yhi = dy > 0 ? n - dy : n;
    const int xr = xlo + un.z * 32 + lane;
    const bool xvalid = xr < xhi;
    const int x = xvalid ? xr : xhi - 1;
    const int y0 = ylo + un.w * kR;
    const float sx = dx * (1.0f / kS), sy = dy * (1.0f / kS);
    float px = fmaf(0.5f, sx, (float)x), py = fmaf(0.5f, sy, (float)y0);
    float acc[kR];
#pragma unroll
    for (int q = 0; q < kR; ++q) acc[q] = 0.f;
#pragma unroll 4
    for (int i = 0; i < kS; ++i) {
      const float bx = __fadd_rd(px, kTwo23), by = __fadd_rd(py, kTwo23);
      const float ax = px - (bx - kTwo23), ay = py - (by - kTwo23);
      const unsigned addr = base + 4u * __float_as_uint(bx) + (4u * (unsigned)ldp) * __float_as_uint(by);
      float L[kR + 1];
      if (LDP > 0) {
        Rows<(LDP > 0 ? LDP : 1), kR + 1>::load(addr, ax, L);
      } else {
#pragma unroll
        for (int r = 0; r <= kR; ++r) {
          float v0, v1;
          const unsigned ar = addr + 4u * ldp * r;
          asm("ld.shared.f32 %0, [%1];" : "=f"(v0) : "r"(ar));
          asm("ld.shared.f32 %0, [%1+4];" : "=f"(v1) : "r"(ar));
          L[r] = fmaf(ax, v1 - v0, v0);
        }
      }
      const float w0 = 1.0f - ay;
#pragma unroll
      for (int q = 0; q < kR; ++q) acc[q] = fmaf(ay, L[q + 1], fmaf(w0, L[q], acc[q]));
      px += sx;
      py += sy;
    }
    const float r2 = (float)(dx * dx + dy * dy);
    const float inv_r = rsqrtf(r2);
    const float tscale = -a.tau_scale2 * r2 * inv_r;  // -(h/S) log2(e) r
    const float wk = a.wcoef * inv_r;
#pragma unroll
    for (int q = 0; q < kR; ++q) {
      const int y = y0 + q;
      if (xvalid && y < yhi) {
        const long j = (long)y * n + x;
        const long k = j + (long)dy * n + dx;
        const float w = wk * exp2f(tscale * acc[q]) * scale;
        atomicAdd(&ysh[j], (unsigned long long)__float2ll_rn(w * __ldg(a.src + k)));
        atomicAdd(&ysh[k], (unsigned long long)__float2ll_rn(w * __ldg(a.src + j)));
      }
    }
  }
  __syncthreads();
  unsigned long long *out = reinterpret_cast<unsigned long long *>(a.partial) + (long)blockIdx.x * N;
  for (long i = tid; i < N; i += kThreads) out[i] = ysh[i];
  if (blockIdx.x == 0 && tid == 0) *a.scale_out = scale_d;
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(a.counter + 1, 1) == (int)gridDim.x - 1) {
      a.counter[0] = 0;
      a.counter[1] = 0;
      *a.smax = 0u;  // every CTA read it before this, the next source kernel sets it
      __threadfence();
    }
  }
}

// the padded FP32 lattice (stride P = n + 1) with kExtraRows more rows
// repeating row n
__global__ void k_make_rows(int n, const float *__restrict__ pad, int rows, float *__restrict__ out) {
  const int P = n + 1;
  const long total = (long)rows * P;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int y = (int)(i / P), x = (int)(i % P);
    out[i] = pad[(long)min(y, P - 1) * P + x];
  }
}

// y_j = (sum_slot part[slot][j]) / scale + d_j s_j, integer sum over the slots
__global__ void k_disp_reduce(long N, int slots, int op, const unsigned long long *__restrict__ part,
                              const double *__restrict__ scale, const double *__restrict__ diag,
                              const double *__restrict__ ss, const double *__restrict__ g,
                              double *__restrict__ y) {
  const double inv = 1.0 / *scale;
  for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < N; j += (long)gridDim.x * blockDim.x) {
    unsigned long long acc = 0ull;
    for (int p = 0; p < slots; ++p) acc += part[(long)p * N + j];
    const double sj = op == VIE_OP_A_RAW ? g[j] : ss[j] * g[j];
    const double v = (double)(long long)acc * inv + diag[j] * sj;
    y[j] = op == VIE_OP_I_MINUS_K ? g[j] - v : v;
  }
}

// s = sigma_s g (or g) in FP32, and max |s| (float bits, atomicMax)
__global__ void k_disp_source(long N, int op, const double *__restrict__ ss, const double *__restrict__ g,
                              float *__restrict__ s, unsigned *__restrict__ smax) {
  unsigned m = 0u;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    const float v = (float)(op == VIE_OP_A_RAW ? g[i] : ss[i] * g[i]);
    s[i] = v;
    m = max(m, __float_as_uint(fabsf(v)));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(smax, m);
}

typedef void (*DispKernel)(DispArgs);

DispKernel pick_disp(int ldp) {
  switch (ldp) {
    case 65: return k_pairs_disp<65>;
    case 129: return k_pairs_disp<129>;
    default: return k_pairs_disp<0>;
  }
}

}  // namespace

size_t disp_smem_bytes(int n) {
  const long rows = n + 1 + kExtraRows;
  return sizeof(float) * (size_t)rows * (n + 1) + sizeof(unsigned long long) * (size_t)n * n + 16;
}

vie_status disp_prepare(DispPlan *dp, int n, const float *sig_padded, int device, cudaStream_t st) {
  dp->usable = 0;
  if (n < 2) return VIE_OK;
  cudaDeviceProp prop;
  VIE_CUDA(cudaGetDeviceProperties(&prop, device));
  const size_t smem = disp_smem_bytes(n);
  if (smem > (size_t)prop.sharedMemPerBlockOptin) return VIE_OK;
  const int ldp = n + 1, rows = n + 1 + kExtraRows;
  DispKernel k = pick_disp(ldp);
  VIE_CUDA(cudaFuncSetAttribute((const void *)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int bps = 0;
  VIE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, kThreads, smem));
  if (bps < 1) return VIE_OK;
  // work units, largest displacement rectangles first
  struct D {
    int dx, dy;
    long area;
  };
  std::vector<D> ds;
  for (int dy = 0; dy < n; ++dy)
    for (int dx = -(n - 1); dx < n; ++dx) {
      if (dy == 0 && dx <= 0) continue;
      ds.push_back({dx, dy, (long)(n - std::abs(dx)) * (n - dy)});
    }
  std::stable_sort(ds.begin(), ds.end(), [](const D &p, const D &q) { return p.area > q.area; });
  std::vector<short4> units;
  for (const D &d : ds) {
    const int wx = n - std::abs(d.dx), wy = n - d.dy;
    const int bxs = (wx + 31) / 32, bys = (wy + kR - 1) / kR;
    for (int by = 0; by < bys; ++by)
      for (int bx = 0; bx < bxs; ++bx)
        units.push_back(make_short4((short)d.dx, (short)d.dy, (short)bx, (short)by));
  }
  VIE_CUDA(cudaMalloc((void **)&dp->units, sizeof(short4) * units.size()));
  VIE_CUDA(cudaMemcpy(dp->units, units.data(), sizeof(short4) * units.size(), cudaMemcpyHostToDevice));
  VIE_CUDA(cudaMalloc((void **)&dp->counter, 2 * sizeof(int)));
  VIE_CUDA(cudaMemset(dp->counter, 0, 2 * sizeof(int)));
  const long lat_elems = (long)rows * ldp;
  VIE_CUDA(cudaMalloc((void **)&dp->lattice, sizeof(float) * lat_elems));
  k_make_rows<<<(int)std::min((lat_elems + 255) / 256, 4096L), 256, 0, st>>>(n, sig_padded, rows,
                                                                              (float *)dp->lattice);
  VIE_CHECK_LAUNCH("k_make_rows");
  VIE_CUDA(cudaMalloc((void **)&dp->smax, sizeof(unsigned)));
  VIE_CUDA(cudaMemset(dp->smax, 0, sizeof(unsigned)));
  VIE_CUDA(cudaMalloc((void **)&dp->scale, sizeof(double)));
  // every row sum of A is below sum over all nonzero displacements of h / (2 pi r)
  double rb = 0.0;
  for (int dy = -(n - 1); dy < n; ++dy)
    for (int dx = -(n - 1); dx < n; ++dx)
      if (dx || dy) rb += 1.0 / sqrt((double)dx * dx + (double)dy * dy);
  dp->rbound = rb / (2.0 * kPi * n);
  dp->n_units = (long)units.size();
  dp->lat_elems = lat_elems;
  dp->ldp = ldp;
  dp->smem = smem;
  dp->grid = bps * prop.multiProcessorCount;
  dp->kernel = (const void *)k;
  dp->usable = 1;
  return VIE_OK;
}

void disp_release(DispPlan *dp) {
  if (dp->units) cudaFree(dp->units);
  if (dp->counter) cudaFree(dp->counter);
  if (dp->lattice) cudaFree(dp->lattice);
  if (dp->smax) cudaFree(dp->smax);
  if (dp->scale) cudaFree(dp->scale);
  dp->smax = nullptr;
  dp->scale = nullptr;
  dp->units = nullptr;
  dp->counter = nullptr;
  dp->lattice = nullptr;
  dp->usable = 0;
}

vie_status disp_source(const DispPlan &dp, long N, int op, const double *sigma_s, const double *g,
                       float *src, cudaStream_t st) {
  const int blocks = (int)std::min((N + 255) / 256, 1024L);
  k_disp_source<<<blocks, 256, 0, st>>>(N, op, sigma_s, g, src, dp.smax);
  VIE_CHECK_LAUNCH("k_disp_source");
  return VIE_OK;
}

vie_status disp_reduce(const DispPlan &dp, long N, int op, const double *partial, const double *diag,
                       const double *sigma_s, const double *g, double *y, cudaStream_t st) {
  const int blocks = (int)std::min((N + 255) / 256, 4096L);
  k_disp_reduce<<<blocks, 256, 0, st>>>(N, dp.grid, op, (const unsigned long long *)partial, dp.scale, diag,
                                        sigma_s, g, y);
  VIE_CHECK_LAUNCH("k_disp_reduce");
  return VIE_OK;
}

vie_status disp_launch(const DispPlan &dp, int n, float tau_scale2, float wcoef, const float *src,
                       double *partial, cudaStream_t st) {
  DispArgs a;
  a.lat = (const float *)dp.lattice;
  a.src = src;
  a.smax = dp.smax;
  a.scale_out = dp.scale;
  a.rbound = dp.rbound;
  a.partial = partial;
  a.units = (const short4 *)dp.units;
  a.counter = dp.counter;
  a.n_units = dp.n_units;
  a.n = n;
  a.ldp = dp.ldp;
  a.lat_elems = dp.lat_elems;
  a.tau_scale2 = tau_scale2;
  a.wcoef = wcoef;
  a.h = 1.0f / n;
  void *args[] = {&a};
  VIE_CUDA(cudaLaunchKernel(dp.kernel, dim3(dp.grid), dim3(kThreads), args, dp.smem, st));
  count_launch();
  return VIE_OK;
}

}  // namespace vie
