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
// March arithmetic: two consecutive samples share every FP32x2 instruction
// (sm_100 family packed add/fma).  In lattice units the sample positions are
// multiples of 1/128 below 2^13 and advance by exact adds.  floor(p) is the
// round-toward-minus-infinity sum p + 2^23; its bit pattern is 0x4B000000 +
// floor(p), used directly as the integer index (the bias is folded into the
// shared-memory base address).
#include <math.h>

#include <algorithm>
#include <vector>

#include "vie_internal.cuh"

namespace vie {

namespace {

typedef unsigned long long u64;

constexpr int kG = 128;                // targets per tile = threads per group
constexpr int kGroups = 8;             // groups per CTA
constexpr int kCtaThreads = kG * kGroups;
constexpr int kS = 64;                 // march steps of this kernel
constexpr float kTwo23 = 8388608.0f;
constexpr unsigned kTwo23Bits = 0x4B000000u;

__device__ __forceinline__ u64 pk(float lo, float hi) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk(u64 r, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}
__device__ __forceinline__ void upku(u64 r, unsigned &lo, unsigned &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "l"(r));
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
  u64 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 addrm2(u64 a, u64 b) {
  u64 r;
  asm("add.rm.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
  u64 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
  u64 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
template <int OFF>
__device__ __forceinline__ float lds(unsigned addr) {
  float v;
  asm("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(addr), "n"(OFF));
  return v;
}
__device__ __forceinline__ float lds_rt(unsigned addr) {
  float v;
  asm("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
  return v;
}

// Lattice geometry: element (x, y, z) sits at x + LDP*y + PLANE*z.  LDP = 0
// selects runtime strides.
struct Geo {
  unsigned base;  // shared byte address of element 0 minus the 2^23 bias
  int ldp, plane; // runtime strides (elements)
};

// Sum of the multilinear interpolant at the two lattice points held in
// (px, py, pz) (one sample per 32-bit half).
template <int DIM, int LDP, int PLANE>
__device__ __forceinline__ u64 sample_pair(const Geo &g, u64 m2, u64 px, u64 py, u64 pz) {
  const u64 bx = addrm2(px, m2), by = addrm2(py, m2);
  const u64 ax = sub2(px, sub2(bx, m2)), ay = sub2(py, sub2(by, m2));
  unsigned x0, x1, y0, y1;
  upku(bx, x0, x1);
  upku(by, y0, y1);
  const int ldp = LDP > 0 ? LDP : g.ldp;
  unsigned a0 = g.base + 4u * x0 + (4u * (unsigned)ldp) * y0;
  unsigned a1 = g.base + 4u * x1 + (4u * (unsigned)ldp) * y1;
  if (DIM == 3) {
    const u64 bz = addrm2(pz, m2);
    const u64 az = sub2(pz, sub2(bz, m2));
    unsigned z0, z1;
    upku(bz, z0, z1);
    const int plane = PLANE > 0 ? PLANE : g.plane;
    a0 += (4u * (unsigned)plane) * z0;
    a1 += (4u * (unsigned)plane) * z1;
    float c[2][8];
    if (LDP > 0) {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const unsigned a = s ? a1 : a0;
        c[s][0] = lds<0>(a);
        c[s][1] = lds<4>(a);
        c[s][2] = lds<4 * LDP>(a);
        c[s][3] = lds<4 * LDP + 4>(a);
        c[s][4] = lds<4 * PLANE>(a);
        c[s][5] = lds<4 * PLANE + 4>(a);
        c[s][6] = lds<4 * PLANE + 4 * LDP>(a);
        c[s][7] = lds<4 * PLANE + 4 * LDP + 4>(a);
      }
    } else {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const unsigned a = s ? a1 : a0;
        const unsigned b = a + 4u * g.ldp, p = a + 4u * g.plane, q = b + 4u * g.plane;
        c[s][0] = lds_rt(a);
        c[s][1] = lds_rt(a + 4);
        c[s][2] = lds_rt(b);
        c[s][3] = lds_rt(b + 4);
        c[s][4] = lds_rt(p);
        c[s][5] = lds_rt(p + 4);
        c[s][6] = lds_rt(q);
        c[s][7] = lds_rt(q + 4);
      }
    }
    u64 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = pk(c[0][e], c[1][e]);
    const u64 e00 = fma2(ax, sub2(v[1], v[0]), v[0]);
    const u64 e10 = fma2(ax, sub2(v[3], v[2]), v[2]);
    const u64 e01 = fma2(ax, sub2(v[5], v[4]), v[4]);
    const u64 e11 = fma2(ax, sub2(v[7], v[6]), v[6]);
    const u64 f0 = fma2(ay, sub2(e10, e00), e00);
    const u64 f1 = fma2(ay, sub2(e11, e01), e01);
    return fma2(az, sub2(f1, f0), f0);
  } else {
    float c[2][4];
    if (LDP > 0) {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const unsigned a = s ? a1 : a0;
        c[s][0] = lds<0>(a);
        c[s][1] = lds<4>(a);
        c[s][2] = lds<4 * LDP>(a);
        c[s][3] = lds<4 * LDP + 4>(a);
      }
    } else {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const unsigned a = s ? a1 : a0;
        const unsigned b = a + 4u * g.ldp;
        c[s][0] = lds_rt(a);
        c[s][1] = lds_rt(a + 4);
        c[s][2] = lds_rt(b);
        c[s][3] = lds_rt(b + 4);
      }
    }
    const u64 v00 = pk(c[0][0], c[1][0]), v10 = pk(c[0][1], c[1][1]);
    const u64 v01 = pk(c[0][2], c[1][2]), v11 = pk(c[0][3], c[1][3]);
    const u64 lo = fma2(ax, sub2(v10, v00), v00);
    const u64 hi = fma2(ax, sub2(v11, v01), v01);
    return fma2(ay, sub2(hi, lo), lo);
  }
}

// Sum of the S = 64 samples of sigma_t~ from lattice point j towards j + d.
template <int DIM, int LDP, int PLANE>
__device__ __forceinline__ float march64(const Geo &g, float jx, float jy, float jz, float dx,
                                         float dy, float dz) {
  const u64 m2 = pk(kTwo23, kTwo23);
  const float sx = dx * (1.0f / kS), sy = dy * (1.0f / kS), sz = dz * (1.0f / kS);
  u64 px = pk(fmaf(0.5f, sx, jx), fmaf(1.5f, sx, jx));
  u64 py = pk(fmaf(0.5f, sy, jy), fmaf(1.5f, sy, jy));
  u64 pz = DIM == 3 ? pk(fmaf(0.5f, sz, jz), fmaf(1.5f, sz, jz)) : 0ull;
  const u64 tx = pk(2.f * sx, 2.f * sx), ty = pk(2.f * sy, 2.f * sy);
  const u64 tz = DIM == 3 ? pk(2.f * sz, 2.f * sz) : 0ull;
  u64 acc0 = 0ull, acc1 = 0ull;  // +0.0f pairs
#pragma unroll
  for (int i = 0; i < kS / 2; ++i) {
    const u64 v = sample_pair<DIM, LDP, PLANE>(g, m2, px, py, pz);
    if (i & 1)
      acc1 = add2(acc1, v);
    else
      acc0 = add2(acc0, v);
    px = add2(px, tx);
    py = add2(py, ty);
    if (DIM == 3) pz = add2(pz, tz);
  }
  float a, b, c, d;
  upk(acc0, a, b);
  upk(acc1, c, d);
  return (a + b) + (c + d);
}

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

  // stage the lattice (whole CTA)
  {
    const float4 *g4 = reinterpret_cast<const float4 *>(a.sig);
    const long n4 = a.lattice / 4;
    float4 *l4 = reinterpret_cast<float4 *>(lat);
    for (long i = tid; i < n4; i += kCtaThreads) l4[i] = g4[i];
    for (long i = n4 * 4 + tid; i < a.lattice; i += kCtaThreads) lat[i] = a.sig[i];
  }
  __syncthreads();

  Geo geo;
  {
    const unsigned lat_addr = (unsigned)__cvta_generic_to_shared(lat);
    const unsigned ldp = LDP > 0 ? LDP : a.ldp, plane = PLANE > 0 ? PLANE : a.plane;
    // element index = (x - B) + ldp (y - B) + plane (z - B) with B = 0x4B000000
    unsigned bias = kTwo23Bits * (1u + ldp + (DIM == 3 ? plane : 0u));
    geo.base = lat_addr - 4u * bias;
    geo.ldp = (int)ldp;
    geo.plane = (int)plane;
  }
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
        const float acc = march64<DIM, LDP, PLANE>(geo, jx, jy, jz, dx, dy, dz);
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

vie_status sym_prepare(SymPlan *sp, int dim, int n, long N, const float *sig_padded,
                       int device, cudaStream_t st) {
  cudaDeviceProp prop;
  VIE_CUDA(cudaGetDeviceProperties(&prop, device));
  int ldp = 0, plane = 0;
  SymKernel k = pick(dim, n + 1, &ldp, &plane);
  size_t smem = sym_smem_bytes(dim, n, nullptr, nullptr);
  sp->usable = 0;
  if (smem > (size_t)prop.sharedMemPerBlockOptin) return VIE_OK;
  VIE_CUDA(cudaFuncSetAttribute((const void *)k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
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
  VIE_CUDA(cudaMalloc((void **)&sp->items, sizeof(int2) * items.size()));
  VIE_CUDA(cudaMemcpy(sp->items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice));
  VIE_CUDA(cudaMalloc((void **)&sp->counter, 2 * sizeof(int)));
  VIE_CUDA(cudaMemset(sp->counter, 0, 2 * sizeof(int)));
  VIE_CUDA(cudaMalloc((void **)&sp->lattice, sizeof(float) * lattice));
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
  if (sp->items) cudaFree(sp->items);
  if (sp->counter) cudaFree(sp->counter);
  if (sp->lattice) cudaFree(sp->lattice);
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
vie_status sym_plan_external(SymPlan *sp, int dim, int n, long N, const float *sig_padded,
                             int device, int2 *items_mem, int *counter_mem, float *lattice_mem,
                             cudaStream_t st) {
  cudaDeviceProp prop;
  VIE_CUDA(cudaGetDeviceProperties(&prop, device));
  int ldp = 0, plane = 0;
  SymKernel k = pick(dim, n + 1, &ldp, &plane);
  const size_t smem = sym_smem_bytes(dim, n, nullptr, nullptr);
  sp->usable = 0;
  if (smem > (size_t)prop.sharedMemPerBlockOptin) return VIE_OK;
  VIE_CUDA(cudaFuncSetAttribute((const void *)k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  int bps = 0;
  VIE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, kCtaThreads, smem));
  if (bps < 1) return VIE_OK;
  const long P = n + 1;
  const long lattice = dim == 2 ? (long)ldp * P : (long)plane * P;
  sp->T = (int)((N + kG - 1) / kG);
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
  sp->grid = (int)std::min<long>((long)bps * prop.multiProcessorCount,
                                 (sp->n_items + kGroups - 1) / kGroups);
  sp->kernel = (const void *)k;
  sp->usable = 1;
  return VIE_OK;
}

}  // namespace vie
