// Assembly of the discrete operator K (Section 3.2, Eq. EQ: LINEAR SYSTEM:
// K = [K_jk omega_k]) into device memory, for reuse across applies: the
// paper caches its kernel evaluations for the same reason (Section 4.2, last
// paragraph: line integrals cached during setup and reused by GMRES).
//
// K_jk = A_jk sigma_s,k (j != k), K_jj = d_j sigma_s,j, row-major with row
// stride LDK (a multiple of 64 elements, padding columns zero).  Storage is
// FP32, or BF16 hi/lo pairs hi = bf16(K), lo = bf16(K - hi) for the
// split-precision tensor-core product.
//
// The pair weights come from the same S = 64 FP32x2 march as the symmetric
// apply (march.cuh), on the same tile-pair work list: each unordered pair is
// marched once and written twice.  K[k][j] (row k, consecutive j across the
// threads of a warp) is stored directly; K[j][k] goes through a 32 x 33
// per-warp transpose in shared memory so that both stores are coalesced.
#include <cuda_bf16.h>

#include <algorithm>

#include "march.cuh"
#include "vie_internal.cuh"

namespace vie {

namespace {

using namespace march;

constexpr int kG = 128;  // targets per tile = threads per group

struct AsmArgs {
  const float *sig;        // re-strided lattice (global), copied to shared memory
  const double *sigma_s;   // [N]
  float *k32;              // FP32 output or null
  __nv_bfloat16 *khi, *klo;// BF16 split output or null
  long ldk;                // row stride (elements)
  const int2 *items;
  int *counter;
  long N;
  int n, n_items, ldp, plane, groups;
  long lattice;
  float tau_scale2, wcoef;
};

__device__ __forceinline__ void gsync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(kG) : "memory");
}

__device__ __forceinline__ void store_entry(const AsmArgs &a, long row, long col, float v) {
  const long idx = row * a.ldk + col;
  if (a.k32) a.k32[idx] = v;
  if (a.khi) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    a.khi[idx] = hi;
    a.klo[idx] = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
}

template <int DIM, int LDP, int PLANE>
__global__ void __launch_bounds__(1024, 1) k_assemble_sym(AsmArgs a) {
  extern __shared__ float4 smem[];
  const int groups = a.groups;
  float4 *srcs_all = smem;                                            // [groups][kG]
  float *tr_all = reinterpret_cast<float *>(smem + groups * kG);      // [groups][4][32][33]
  int *slot_all = reinterpret_cast<int *>(tr_all + groups * 4 * 32 * 33);
  float *lat = reinterpret_cast<float *>(slot_all + 4 * groups);
  const int tid = threadIdx.x, nthreads = blockDim.x;
  const int grp = tid / kG, t = tid % kG, warp = t / 32, lane = t % 32;
  float4 *srcs = srcs_all + grp * kG;
  float *tr = tr_all + (grp * 4 + warp) * 32 * 33;
  int *slot = slot_all + 4 * grp;
  if (LDP >= 0) {  // LDP < 0: the lattice stays in global memory
    const float4 *g4 = reinterpret_cast<const float4 *>(a.sig);
    const long n4 = a.lattice / 4;
    float4 *l4 = reinterpret_cast<float4 *>(lat);
    for (long i = tid; i < n4; i += nthreads) l4[i] = g4[i];
    for (long i = n4 * 4 + tid; i < a.lattice; i += nthreads) lat[i] = a.sig[i];
  }
  __syncthreads();
  const Geo geo = make_geo((unsigned)__cvta_generic_to_shared(lat), DIM, LDP > 0 ? LDP : a.ldp,
                           PLANE > 0 ? PLANE : a.plane);
  GeoG geog;
  geog.base = a.sig;
  geog.ldp = a.ldp;
  geog.bias = kTwo23Bits * (1u + (unsigned)a.ldp);
  const int n = a.n;
  const long N = a.N, nn = (long)n * n;
  for (;;) {
    if (t == 0) *slot = atomicAdd(a.counter, 1);
    gsync(grp);
    const int it = *slot;
    gsync(grp);
    if (it >= a.n_items) break;
    const int2 ab = a.items[it];
    const long j_raw = (long)ab.x * kG + t;
    const bool jvalid = j_raw < N;
    const long j = jvalid ? j_raw : N - 1;
    const float jx = (float)(j % n), jy = (float)((j / n) % n);
    const float jz = DIM == 3 ? (float)(j / nn) : 0.f;
    const float ssj = (float)a.sigma_s[j];
    {
      const long k = (long)ab.y * kG + t;
      const long kc = k < N ? k : N - 1;
      srcs[t] = make_float4((float)(kc % n), (float)((kc / n) % n),
                            DIM == 3 ? (float)(kc / nn) : 0.f, (float)a.sigma_s[kc]);
    }
    gsync(grp);
    const bool diag_item = ab.x == ab.y;
#pragma unroll 1
    for (int c0 = 0; c0 < kG; c0 += 32) {
#pragma unroll 1
      for (int cc = 0; cc < 32; ++cc) {
        const int c = c0 + cc;
        const float4 q = srcs[c];
        const float dx = q.x - jx, dy = q.y - jy, dz = q.z - jz;
        const float r2 = DIM == 3 ? fmaf(dz, dz, fmaf(dy, dy, dx * dx)) : fmaf(dy, dy, dx * dx);
        const float inv_r = rsqrtf(r2);
        const float r = r2 * inv_r;
        const float acc = LDP < 0 ? march64_g(geog, jx, jy, dx, dy)
                                  : march64<DIM, (LDP < 0 ? 0 : LDP), PLANE>(geo, jx, jy, jz, dx, dy, dz);
        const float ker = DIM == 3 ? inv_r * inv_r : inv_r;
        float w = a.wcoef * exp2f(-a.tau_scale2 * acc * r) * ker;
        w = r2 > 0.f ? w : 0.f;
        const long k = (long)ab.y * kG + c;
        // row k, column j: consecutive j across the warp
        if (jvalid && k < N && k != j) store_entry(a, k, j, w * ssj);
        if (!diag_item) tr[cc * 33 + lane] = w;
      }
      if (!diag_item) {
        __syncwarp();
        // row j_r (r-th target of this warp), columns k = 128 b + c0 + lane
        const long k = (long)ab.y * kG + c0 + lane;
        const float ssk = srcs[c0 + lane].w;
#pragma unroll 4
        for (int r = 0; r < 32; ++r) {
          const long jr = (long)ab.x * kG + warp * 32 + r;
          if (jr < N && k < N) store_entry(a, jr, k, tr[lane * 33 + r] * ssk);
        }
        __syncwarp();
      }
    }
    gsync(grp);
  }
  if (t == 0) {
    __threadfence();
    const int done = atomicAdd(a.counter + 1, 1);
    if (done == (int)gridDim.x * groups - 1) {
      a.counter[0] = 0;
      a.counter[1] = 0;
      __threadfence();
    }
  }
}

// K_jj = d_j sigma_s,j
__global__ void k_assemble_diag(long N, long ldk, const double *__restrict__ diag,
                                const double *__restrict__ ss, float *k32, __nv_bfloat16 *khi,
                                __nv_bfloat16 *klo) {
  for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < N; j += (long)gridDim.x * blockDim.x) {
    const float v = (float)(diag[j] * ss[j]);
    const long idx = j * ldk + j;
    if (k32) k32[idx] = v;
    if (khi) {
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      khi[idx] = hi;
      klo[idx] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
  }
}

typedef void (*AsmKernel)(AsmArgs);

AsmKernel pick_asm(int dim, int ldp, int plane, int global) {
  if (global) return k_assemble_sym<2, -1, 0>;
  if (dim == 2) {
    switch (ldp) {
      case 33: return k_assemble_sym<2, 33, 0>;
      case 65: return k_assemble_sym<2, 65, 0>;
      case 97: return k_assemble_sym<2, 97, 0>;
      case 129: return k_assemble_sym<2, 129, 0>;
      case 161: return k_assemble_sym<2, 161, 0>;
      case 193: return k_assemble_sym<2, 193, 0>;
      case 225: return k_assemble_sym<2, 225, 0>;
      default: return k_assemble_sym<2, 0, 0>;
    }
  }
  if (ldp == 33 && plane == 33 * 33) return k_assemble_sym<3, 33, 33 * 33>;
  return k_assemble_sym<3, 0, 0>;
}

}  // namespace

long assembled_ldk(long N) { return (N + 63) / 64 * 64; }

vie_status launch_assemble(const SymPlan &sp, int dim, int n, long N, const double *sigma_s,
                           const double *diag, float *k32, void *khi, void *klo, int device,
                           cudaStream_t st) {
  if (!sp.usable) {
    set_error("vie_assemble: grid too large for the shared-memory assembly kernel");
    return VIE_ERR_UNSUPPORTED;
  }
  const long ldk = assembled_ldk(N);
  const size_t kbytes = sizeof(float) * (size_t)N * ldk;
  if (k32) VIE_CUDA(cudaMemsetAsync(k32, 0, kbytes, st));
  if (khi) {
    VIE_CUDA(cudaMemsetAsync(khi, 0, kbytes / 2, st));
    VIE_CUDA(cudaMemsetAsync(klo, 0, kbytes / 2, st));
  }
  DevProps prop;
  VIE_TRY(get_dev_props(device, &prop));
  const size_t per_group = sizeof(float4) * kG + sizeof(float) * 4 * 32 * 33 + 4 * sizeof(int);
  const size_t lat_bytes = sp.global_lattice ? 0 : sizeof(float) * sp.lattice_elems;
  int groups = (int)std::min<size_t>(8, (prop.sharedMemPerBlockOptin - lat_bytes) / per_group);
  if (groups < 1) {
    set_error("vie_assemble: lattice too large for the assembly kernel");
    return VIE_ERR_UNSUPPORTED;
  }
  const size_t smem = per_group * groups + lat_bytes + 64;
  AsmKernel k = pick_asm(dim, sp.ldp, sp.plane, sp.global_lattice);
  VIE_TRY(raise_smem_limit((const void *)k, (size_t)((int)smem)));
  int bps = 0;
  VIE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, kG * groups, smem));
  if (bps < 1) {
    set_error("vie_assemble: assembly kernel does not fit on an SM");
    return VIE_ERR_UNSUPPORTED;
  }
  AsmArgs a;
  a.sig = sp.lattice;
  a.sigma_s = sigma_s;
  a.k32 = k32;
  a.khi = (__nv_bfloat16 *)khi;
  a.klo = (__nv_bfloat16 *)klo;
  a.ldk = ldk;
  a.items = sp.items;
  a.counter = sp.counter;
  a.N = N;
  a.n = n;
  a.n_items = sp.n_items;
  a.ldp = sp.ldp;
  a.plane = sp.plane;
  a.groups = groups;
  a.lattice = sp.lattice_elems;
  const double h = 1.0 / n;
  a.tau_scale2 = (float)(h / kS * 1.4426950408889634);
  a.wcoef = (float)(dim == 2 ? h / (2.0 * kPi) : h / (4.0 * kPi));
  const int grid = (int)std::min<long>((long)bps * prop.multiProcessorCount,
                                       (sp.n_items + groups - 1) / groups);
  void *args[] = {&a};
  VIE_CUDA(cudaLaunchKernel((const void *)k, dim3(grid), dim3(kG * groups), args, smem, st));
  count_launch();
  const long b = (N + 255) / 256;
  k_assemble_diag<<<(int)std::min(b, 4096L), 256, 0, st>>>(N, ldk, diag, sigma_s, k32,
                                                           (__nv_bfloat16 *)khi,
                                                           (__nv_bfloat16 *)klo);
  VIE_CHECK_LAUNCH("k_assemble_diag");
  return VIE_OK;
}

}  // namespace vie
