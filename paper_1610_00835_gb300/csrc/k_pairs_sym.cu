// Symmetric on-the-fly pair kernel for FP32 tiles with S = 64 march steps.
//
// What it computes is the operator of k_apply.cu (Section 2, Eq. EQ:Kernel;
// Section 3.2, M-iii): y_j = sum_{k != j} A_jk s_k with
//   A_jk = h^d exp(-tau_jk) / (|S^{d-1}| r_jk^{d-1}),
//   tau_jk = (r_jk / S) sum_{i<S} sigma_t~(u_j + (i+1/2)/S (u_k - u_j)).
// The midpoint samples of the segment j -> k are those of k -> j in reverse
// order, so A_jk = A_kj: each unordered pair is marched once and feeds both
// y_j (row sum, weight s_k) and y_k (column sum, weight s_j).
//
// Work decomposition: targets are cut into tiles of G = 128 cells; an item is
// a tile pair (a, b) with a <= b.  A group of 128 threads (4 warps) takes
// items from a global counter; thread t owns target j = 128 a + t and walks
// the 128 sources of tile b.  Row sums go to partial[b][j]; column sums are
// reduced across the group (warp shuffles, then 4 warps in shared memory) and
// go to partial[a][k].  Every (slot, target) of partial[T][N] is written
// exactly once (target j of tile a is a row target of items (a, b >= a) and a
// column target of items (c < a, a)), so the reduce kernel needs no zeroing.
// A CTA holds 8 groups that share one copy of the padded sigma_t lattice in
// shared memory.  The last group to run out of items resets the counter for
// the next launch; no thread ever waits on another CTA.
//
// The march arithmetic (FP32x2 packed sample pairs) is in march.cuh.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "march.cuh"
#include "vie_internal.cuh"

namespace vie {

namespace {

using namespace march;

constexpr int kG = 128;                // targets per tile = threads per group
constexpr int kGroups = 8;             // groups per CTA
constexpr int kCtaThreads = kG * kGroups;

struct SymArgs {
  const float *sig;    // padded lattice (global), copied to shared memory
  const float *src;    // s_k, FP32 [N]
  double *partial;     // [T][N]
  const int2 *items;   // (a, b), a <= b
  int *counter;        // [2]: next item, finished groups
  long N;
  int n, T, n_items, ldp, plane;
  long lattice;        // elements of the shared lattice
  float tau_scale2;    // (h / S) log2(e)
  float wcoef;         // h / (2 pi) or h / (4 pi)
};

__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(kG) : "memory");
}

template <int DIM, int LDP, int PLANE>
__global__ void __launch_bounds__(kCtaThreads, 1) k_pairs_sym(SymArgs a) {
  extern __shared__ float4 smem[];
  // per group: sources [kG] float4, column sums [4][kG] float, item slot
  float4 *srcs_all = smem;
  float *col_all = reinterpret_cast<float *>(smem + kGroups * kG);
  int *item_all = reinterpret_cast<int *>(col_all + kGroups * 4 * kG);
  float *lat = reinterpret_cast<float *>(item_all + 4 * kGroups);
  const int tid = threadIdx.x;
  const int grp = tid / kG, t = tid % kG, warp = t / 32, lane = t % 32;
  float4 *srcs = srcs_all + grp * kG;
  float *colw = col_all + grp * 4 * kG;
  int *item_slot = item_all + 4 * grp;

  // stage the lattice (whole CTA); LDP < 0: the lattice stays in global memory
  if (LDP >= 0) {
    const float4 *g4 = reinterpret_cast<const float4 *>(a.sig);
    const long n4 = a.lattice / 4;
    float4 *l4 = reinterpret_cast<float4 *>(lat);
    for (long i = tid; i < n4; i += kCtaThreads) l4[i] = g4[i];
    for (long i = n4 * 4 + tid; i < a.lattice; i += kCtaThreads) lat[i] = a.sig[i];
  }
  __syncthreads();

  const Geo geo = make_geo((unsigned)__cvta_generic_to_shared(lat), DIM,
                           LDP > 0 ? LDP : a.ldp, PLANE > 0 ? PLANE : a.plane);
  GeoG geog;
  geog.base = a.sig;
  geog.ldp = a.ldp;
  geog.bias = kTwo23Bits * (1u + (unsigned)a.ldp);
  const int n = a.n;
  const long N = a.N;
  const long nn = (long)n * n;

  for (;;) {
    if (t == 0) *item_slot = atomicAdd(a.counter, 1);
    group_sync(grp);
    const int it = *item_slot;
    group_sync(grp);
    if (it >= a.n_items) break;
    const int2 ab = a.items[it];
    const long j_raw = (long)ab.x * kG + t;
    const bool jvalid = j_raw < N;
    const long j = jvalid ? j_raw : N - 1;
    const float jx = (float)(j % n), jy = (float)((j / n) % n);
    const float jz = DIM == 3 ? (float)(j / nn) : 0.f;
    const float sj = jvalid ? a.src[j] : 0.f;
    {
      const long k = (long)ab.y * kG + t;
      const bool kvalid = k < N;
      const long kc = kvalid ? k : N - 1;
      srcs[t] = make_float4((float)(kc % n), (float)((kc / n) % n),
                            DIM == 3 ? (float)(kc / nn) : 0.f, kvalid ? a.src[kc] : 0.f);
    }
    group_sync(grp);
    const bool diag_item = ab.x == ab.y;
    double dsum = 0.0;
#pragma unroll 1
    for (int c0 = 0; c0 < kG; c0 += 64) {
      float fsum = 0.f;
#pragma unroll 1
      for (int c = c0; c < c0 + 64; ++c) {
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
        fsum = fmaf(w, q.w, fsum);
        if (!diag_item) {
          float cs = w * sj;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
          if (lane == 0) colw[warp * kG + c] = cs;
        }
      }
      dsum += (double)fsum;
    }
    if (jvalid) a.partial[(long)ab.y * N + j] = dsum;
    if (!diag_item) {
      group_sync(grp);
      const long k = (long)ab.y * kG + t;
      if (k < N) {
        const float s = (colw[t] + colw[kG + t]) + (colw[2 * kG + t] + colw[3 * kG + t]);
        a.partial[(long)ab.x * N + k] = (double)s;
      }
    }
    group_sync(grp);
  }
  // The last group to finish resets the counter for the next launch.
  if (t == 0) {
    __threadfence();
    const int done = atomicAdd(a.counter + 1, 1);
    if (done == (int)gridDim.x * kGroups - 1) {
      a.counter[0] = 0;
      a.counter[1] = 0;
      __threadfence();
    }
  }
}

typedef void (*SymKernel)(SymArgs);

// Instantiated lattice strides: 2D LDP = n + 1 rounded up to these; 3D uses
// LDP = PLANE / LDP = 33 (n <= 32).  Other sizes take the runtime-stride one.
SymKernel pick(int dim, int P, int *ldp, int *plane) {
  if (dim == 2) {
    static const int sizes[] = {33, 65, 97, 129, 161, 193, 225};
    for (int s : sizes)
      if (P <= s) {
        *ldp = s;
        *plane = 0;
        switch (s) {
          case 33: return k_pairs_sym<2, 33, 0>;
          case 65: return k_pairs_sym<2, 65, 0>;
          case 97: return k_pairs_sym<2, 97, 0>;
          case 129: return k_pairs_sym<2, 129, 0>;
          case 161: return k_pairs_sym<2, 161, 0>;
          case 193: return k_pairs_sym<2, 193, 0>;
          default: return k_pairs_sym<2, 225, 0>;
        }
      }
    *ldp = P;
    *plane = 0;
    return k_pairs_sym<2, 0, 0>;
  }
  if (P == 33) {
    *ldp = 33;
    *plane = 33 * 33;
    return k_pairs_sym<3, 33, 33 * 33>;
  }
  *ldp = P;
  *plane = P * P;
  return k_pairs_sym<3, 0, 0>;
}

// Copy the padded lattice (stride P) into stride (ldp, plane) layout.
__global__ void k_restride(int dim, int P, int ldp, int plane, const float *__restrict__ in,
                           float *__restrict__ out, long total_out) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total_out;
       i += (long)gridDim.x * blockDim.x) {
    long z = dim == 3 ? i / plane : 0;
    long rem = i - z * (long)(dim == 3 ? plane : 0);
    long y = rem / ldp, x = rem % ldp;
    long xs = x < P ? x : P - 1, ys = y < P ? y : P - 1, zs = z < P ? z : P - 1;
    out[i] = in[(zs * P + ys) * P + xs];
  }
}

}  // namespace

size_t sym_smem_bytes(int dim, int n, int *ldp_out, int *plane_out) {
  int ldp = 0, plane = 0;
  pick(dim, n + 1, &ldp, &plane);
  const long P = n + 1;
  const long lattice = dim == 2 ? (long)ldp * P : (long)plane * P;
  if (ldp_out) *ldp_out = ldp;
  if (plane_out) *plane_out = plane;
  return sizeof(float4) * kGroups * kG + sizeof(float) * kGroups * 4 * kG +
         sizeof(int) * 4 * kGroups + sizeof(float) * lattice;
}

static size_t sym_group_bytes() {
  return sizeof(float4) * kGroups * kG + sizeof(float) * kGroups * 4 * kG + sizeof(int) * 4 * kGroups;
}

vie_status sym_prepare(SymPlan *sp, int dim, int n, long N, const float *sig_padded,
                       int device, cudaStream_t st) {
  DevProps prop;
  VIE_TRY(get_dev_props(device, &prop));
  int ldp = 0, plane = 0;
  SymKernel k = pick(dim, n + 1, &ldp, &plane);
  size_t smem = sym_smem_bytes(dim, n, nullptr, nullptr);
  sp->usable = 0;
  sp->global_lattice = 0;
  if (smem > (size_t)prop.sharedMemPerBlockOptin) {
    if (dim != 2) return VIE_OK;
    // 2D lattice too large for shared memory: read it through L1
    k = k_pairs_sym<2, -1, 0>;
    ldp = n + 1;
    plane = 0;
    smem = sym_group_bytes();
    sp->global_lattice = 1;
  }
  VIE_TRY(raise_smem_limit((const void *)k, (size_t)((int)smem)));
  int bps = 0;
  VIE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, kCtaThreads, smem));
  if (bps < 1) return VIE_OK;
  const long P = n + 1;
  const long lattice = dim == 2 ? (long)ldp * P : (long)plane * P;
  sp->T = (int)((N + kG - 1) / kG);
  sp->n_items = sp->T * (sp->T + 1) / 2;
  std::vector<int2> items;
  items.reserve(sp->n_items);
  for (int a = 0; a < sp->T; ++a)
    for (int b = a; b < sp->T; ++b) items.push_back(make_int2(a, b));
  VIE_CUDA(vie_malloc((void **)&sp->items, sizeof(int2) * items.size()));
  VIE_CUDA(cudaMemcpy(sp->items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice));
  VIE_CUDA(vie_malloc((void **)&sp->counter, 2 * sizeof(int)));
  VIE_CUDA(cudaMemset(sp->counter, 0, 2 * sizeof(int)));
  VIE_CUDA(vie_malloc((void **)&sp->lattice, sizeof(float) * lattice));
  {
    long b = (lattice + 255) / 256;
    k_restride<<<(int)std::min(b, 4096L), 256, 0, st>>>(dim, (int)P, ldp, plane, sig_padded,
                                                        sp->lattice, lattice);
    VIE_CHECK_LAUNCH("k_restride");
  }
  sp->lattice_elems = lattice;
  sp->ldp = ldp;
  sp->plane = plane;
  sp->smem = smem;
  sp->grid = (int)std::min<long>((long)bps * prop.multiProcessorCount,
                                 (sp->n_items + kGroups - 1) / kGroups);
  sp->kernel = (const void *)k;
  sp->usable = 1;
  return VIE_OK;
}

void sym_release(SymPlan *sp) {
  if (sp->items) vie_free(sp->items);
  if (sp->counter) vie_free(sp->counter);
  if (sp->lattice) vie_free(sp->lattice);
  sp->items = nullptr;
  sp->counter = nullptr;
  sp->lattice = nullptr;
  sp->usable = 0;
}

vie_status sym_launch(const SymPlan &sp, int dim, int n, long N, float tau_scale2, float wcoef,
                      const float *src, double *partial, cudaStream_t st) {
  SymArgs a;
  a.sig = sp.lattice;
  a.src = src;
  a.partial = partial;
  a.items = sp.items;
  a.counter = sp.counter;
  a.N = N;
  a.n = n;
  a.T = sp.T;
  a.n_items = sp.n_items;
  a.ldp = sp.ldp;
  a.plane = sp.plane;
  a.lattice = sp.lattice_elems;
  a.tau_scale2 = tau_scale2;
  a.wcoef = wcoef;
  (void)dim;
  void *args[] = {&a};
  VIE_CUDA(cudaLaunchKernel(sp.kernel, dim3(sp.grid), dim3(kCtaThreads), args, sp.smem, st));
  count_launch();
  return VIE_OK;
}

}  // namespace vie

namespace vie {

// Plan the symmetric kernel on caller-provided device memory: nothing is
// allocated.  lattice_mem must hold sym_smem_bytes()' lattice part
// (LDP (n+1) floats in 2D, PLANE (n+1) in 3D); items_mem T (T+1)/2 int2
// (filled by the caller in the order a = 0.., b = a..T-1); counter_mem two
// ints set to zero by the caller before the launch.
// Resident CTAs per SM of a symmetric-kernel variant, per device: computed
// once (occupancy query and shared-memory opt-in), then read from the cache.
struct OccEntry {
  int device;
  const void *kernel;
  size_t smem;
  int bps;
};

vie_status sym_occupancy(int device, const void *k, size_t smem, int *bps) {
  static std::mutex mu;
  static std::vector<OccEntry> cache;
  std::lock_guard<std::mutex> lock(mu);
  for (const OccEntry &e : cache)
    if (e.device == device && e.kernel == k && e.smem == smem) {
      *bps = e.bps;
      return VIE_OK;
    }
  VIE_TRY(raise_smem_limit(k, (size_t)((int)smem)));
  int b = 0;
  VIE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, kCtaThreads, smem));
  cache.push_back({device, k, smem, b});
  *bps = b;
  return VIE_OK;
}

vie_status sym_plan_external(SymPlan *sp, int dim, int n, long N, const float *sig_padded,
                             int device, int2 *items_mem, int *counter_mem, float *lattice_mem,
                             long max_lattice, int max_T, cudaStream_t st) {
  int optin = 0, sms = 0;
  VIE_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  VIE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  int ldp = 0, plane = 0;
  SymKernel k = pick(dim, n + 1, &ldp, &plane);
  const size_t smem = sym_smem_bytes(dim, n, nullptr, nullptr);
  sp->usable = 0;
  if (smem > (size_t)optin) return VIE_OK;
  const long P = n + 1;
  const long lattice = dim == 2 ? (long)ldp * P : (long)plane * P;
  const int T = (int)((N + kG - 1) / kG);
  // the caller's buffers must hold the re-strided lattice and T target tiles
  // before anything is launched into them
  if (lattice > max_lattice || T > max_T) return VIE_OK;
  int bps = 0;
  VIE_TRY(sym_occupancy(device, (const void *)k, smem, &bps));
  if (bps < 1) return VIE_OK;
  sp->T = T;
  sp->n_items = sp->T * (sp->T + 1) / 2;
  sp->items = items_mem;
  sp->counter = counter_mem;
  sp->lattice = lattice_mem;
  {
    long b = (lattice + 255) / 256;
    k_restride<<<(int)std::min(b, 4096L), 256, 0, st>>>(dim, (int)P, ldp, plane, sig_padded,
                                                        lattice_mem, lattice);
    VIE_CHECK_LAUNCH("k_restride");
  }
  sp->lattice_elems = lattice;
  sp->ldp = ldp;
  sp->plane = plane;
  sp->smem = smem;
  sp->grid = (int)std::min<long>((long)bps * sms, (sp->n_items + kGroups - 1) / kGroups);
  sp->kernel = (const void *)k;
  sp->usable = 1;
  return VIE_OK;
}

}  // namespace vie
