// Device helpers of the S = 64 FP32x2 march, shared by the symmetric apply
// kernel (k_pairs_sym.cu) and the assembly kernel (k_assemble.cu).
//
// Two consecutive midpoint samples share every packed FP32x2 instruction
// (sm_100 family add/sub/fma .f32x2).  In lattice units the sample positions
// are multiples of 1/128 below 2^13 and advance by exact adds; floor(p) is
// the round-toward-minus-infinity sum p + 2^23, whose bit pattern is
// 0x4B000000 + floor(p) and serves directly as the integer index (the bias is
// folded into the shared-memory base address).
#pragma once

#include "vie_internal.cuh"

namespace vie {
namespace march {

constexpr int kS = 64;                 // march steps
constexpr float kTwo23 = 8388608.0f;
constexpr unsigned kTwo23Bits = 0x4B000000u;

typedef unsigned long long u64;


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


// 2D lattice read from global memory (through L1) for grids whose lattice
// does not fit in shared memory.  Same arithmetic as sample_pair<2, 0, 0>.
struct GeoG {
  const float *base;  // element 0
  unsigned bias;      // 0x4B000000 (1 + ldp), subtracted from the biased index
  int ldp;
};

__device__ __forceinline__ u64 sample_pair_g(const GeoG &g, u64 m2, u64 px, u64 py) {
  const u64 bx = addrm2(px, m2), by = addrm2(py, m2);
  const u64 ax = sub2(px, sub2(bx, m2)), ay = sub2(py, sub2(by, m2));
  unsigned x0, x1, y0, y1;
  upku(bx, x0, x1);
  upku(by, y0, y1);
  const float *p0 = g.base + (x0 + (unsigned)g.ldp * y0 - g.bias);
  const float *p1 = g.base + (x1 + (unsigned)g.ldp * y1 - g.bias);
  const u64 v00 = pk(__ldg(p0), __ldg(p1)), v10 = pk(__ldg(p0 + 1), __ldg(p1 + 1));
  const u64 v01 = pk(__ldg(p0 + g.ldp), __ldg(p1 + g.ldp));
  const u64 v11 = pk(__ldg(p0 + g.ldp + 1), __ldg(p1 + g.ldp + 1));
  const u64 lo = fma2(ax, sub2(v10, v00), v00);
  const u64 hi = fma2(ax, sub2(v11, v01), v01);
  return fma2(ay, sub2(hi, lo), lo);
}

__device__ __forceinline__ float march64_g(const GeoG &g, float jx, float jy, float dx, float dy) {
  const u64 m2 = pk(kTwo23, kTwo23);
  const float sx = dx * (1.0f / kS), sy = dy * (1.0f / kS);
  u64 px = pk(fmaf(0.5f, sx, jx), fmaf(1.5f, sx, jx));
  u64 py = pk(fmaf(0.5f, sy, jy), fmaf(1.5f, sy, jy));
  const u64 tx = pk(2.f * sx, 2.f * sx), ty = pk(2.f * sy, 2.f * sy);
  u64 acc0 = 0ull, acc1 = 0ull;
#pragma unroll
  for (int i = 0; i < kS / 2; ++i) {
    const u64 v = sample_pair_g(g, m2, px, py);
    if (i & 1)
      acc1 = add2(acc1, v);
    else
      acc0 = add2(acc0, v);
    px = add2(px, tx);
    py = add2(py, ty);
  }
  float a, b, c, d;
  upk(acc0, a, b);
  upk(acc1, c, d);
  return (a + b) + (c + d);
}

// Base address of a lattice at shared address lat_addr with strides (ldp,
// plane): element (x, y, z) is read at base + 4 (X + ldp Y + plane Z), X, Y, Z
// the biased float bits 0x4B000000 + coordinate.
__device__ __forceinline__ Geo make_geo(unsigned lat_addr, int dim, unsigned ldp, unsigned plane) {
  Geo g;
  const unsigned bias = kTwo23Bits * (1u + ldp + (dim == 3 ? plane : 0u));
  g.base = lat_addr - 4u * bias;
  g.ldp = (int)ldp;
  g.plane = (int)plane;
  return g;
}

}  // namespace march
}  // namespace vie
