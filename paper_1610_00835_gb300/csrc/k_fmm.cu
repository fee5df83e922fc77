// Interpolation-based FMM of Section 3.3 (Fong-Darve; Eqs. EQ: CHEB,
// EQ:Kernel Approx, EQ: SUMMATION, EQ: M2L, EQ: L2L) as an assembled operator
// for 2D grids, with every kernel evaluation cached, as the paper does for
// its GMRES iterations.
//
// y = A s for the M-iii matrix A: the near field (each leaf and its 3 x 3
// neighbourhood of leaves) from the entries A_jk themselves, the far field
// through Chebyshev interpolation of
//     K(x, y) = h^2 exp(-tau(x, y)) / (2 pi |x - y|)
// on a quadtree (leaves of b x b cells, n = 2^L b, b >= 8 and as small as the
// factors of two allow; level l has 2^l x 2^l boxes, far field from l = 2):
//     P2M  W_leaf = P s_leaf                      P [p^2][b^2]  = S_p(leaf cell, node)
//     M2M  W_parent = sum_q C_q W_child(q)        C_q [p^2][p^2] = S_p(parent^{-1} child node, node)
//     M2L  L_B = sum_{C in IL(B)} K_BC W_C        K_BC [p^2][p^2]: 27 blocks per box
//     L2L  L_child(q) += C_q^T L_parent
//     L2P  y_leaf += P^T L_leaf
// S_p is Eq. EQ: CHEB with the first-kind points cos((2i - 1) pi / (2p)); P
// and C_q do not depend on the box or the level, so they are built once on
// the host in FP64.  The interaction list IL(B) is the 27 children of the
// neighbours of B's parent that are not neighbours of B; its offsets depend
// only on B's position in its parent.  tau between Chebyshev nodes is the
// S-step midpoint march of the bilinear sigma_t with the sample points
// clamped to the hull of the cell centres (nodes near the boundary lie
// outside it).  Setup fills the near blocks and the M2L blocks on the device
// (FP32); an apply is 2 L - 1 launches of small dense products that read the
// cached blocks once (M2L of all levels in one of them).
#include <math.h>

#include <algorithm>
#include <vector>

#include "vie_internal.cuh"

namespace vie {

namespace {

constexpr int kIL = 27;  // interaction-list slots per box

// far-field offsets (dx, dy) of the interaction list of a box at position
// (qx, qy) in its parent: x in [-2 - qx, 3 - qx], y likewise, minus the 3 x 3
__host__ __device__ __forceinline__ void il_offset(int qx, int qy, int slot, int *dx, int *dy) {
  int k = 0;
  for (int oy = -2 - qy; oy <= 3 - qy; ++oy)
    for (int ox = -2 - qx; ox <= 3 - qx; ++ox) {
      if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1) continue;
      if (k == slot) {
        *dx = ox;
        *dy = oy;
        return;
      }
      ++k;
    }
  *dx = *dy = 0;
}

// bilinear sigma_t~ at lattice coordinates (cell centre j at (ix, iy)),
// clamped to [0, n - 1]; s is the (n + 1)^2 padded lattice
__device__ __forceinline__ float sample_clamped(const float *__restrict__ s, int n, int P, float gx, float gy) {
  gx = fminf(fmaxf(gx, 0.f), (float)(n - 1));
  gy = fminf(fmaxf(gy, 0.f), (float)(n - 1));
  const float fx = floorf(gx), fy = floorf(gy);
  const int ix = (int)fx, iy = (int)fy;
  const float ax = gx - fx, ay = gy - fy;
  const float *r0 = s + (long)iy * P + ix;
  const float lo = fmaf(ax, r0[1] - r0[0], r0[0]);
  const float hi = fmaf(ax, r0[P + 1] - r0[P], r0[P]);
  return fmaf(ay, hi - lo, lo);
}

// h^2 e^{-tau} / (2 pi r) between lattice points a and b (cells; r > 0)
__device__ __forceinline__ float kernel_entry(const float *__restrict__ sig, int n, int P, int S, int closed,
                                              float sigma_c, float ax, float ay, float bx, float by) {
  const float h = 1.0f / (float)n;
  const float dx = bx - ax, dy = by - ay;
  const float r = sqrtf(dx * dx + dy * dy);
  float tau;
  if (closed) {
    tau = sigma_c * h * r;
  } else {
    float acc0 = 0.f, acc1 = 0.f;
    const float inv = 1.0f / (float)S;
    int i = 0;
    for (; i + 1 < S; i += 2) {
      const float t0 = ((float)i + 0.5f) * inv, t1 = ((float)i + 1.5f) * inv;
      acc0 += sample_clamped(sig, n, P, fmaf(t0, dx, ax), fmaf(t0, dy, ay));
      acc1 += sample_clamped(sig, n, P, fmaf(t1, dx, ax), fmaf(t1, dy, ay));
    }
    if (i < S) acc0 += sample_clamped(sig, n, P, fmaf(((float)i + 0.5f) * inv, dx, ax), fmaf(((float)i + 0.5f) * inv, dy, ay));
    tau = h * r * inv * (acc0 + acc1);
  }
  return h * expf(-tau) / (2.0f * 3.14159265358979f * r);
}

struct FillArgs {
  const float *sig;     // padded FP32 sigma_t lattice, (n + 1)^2
  const double *diag;   // self cells
  int n, P, S, closed;
  float sigma_c;
};

// near blocks, stored transposed: near[leaf][slot][k][j] (slot = (oy+1)*3 + ox+1)
__global__ void k_fmm_near_fill(FillArgs a, int L, int b, float *__restrict__ near) {
  const int nl = 1 << L, bb = b * b;
  const long total = (long)nl * nl * 9 * bb * bb;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const int j = (int)(e % bb);
    long t = e / bb;
    const int k = (int)(t % bb);
    t /= bb;
    const int slot = (int)(t % 9);
    const long leaf = t / 9;
    const int bx = (int)(leaf % nl), by = (int)(leaf / nl);
    const int cx = bx + slot % 3 - 1, cy = by + slot / 3 - 1;
    float v = 0.f;
    if (cx >= 0 && cx < nl && cy >= 0 && cy < nl) {
      const int jx = bx * b + j % b, jy = by * b + j / b;
      const int kx = cx * b + k % b, ky = cy * b + k / b;
      if (jx == kx && jy == ky)
        v = (float)a.diag[(long)jy * a.n + jx];
      else
        v = kernel_entry(a.sig, a.n, a.P, a.S, a.closed, a.sigma_c, (float)jx, (float)jy, (float)kx, (float)ky);
    }
    near[e] = v;
  }
}

// M2L blocks of one level: m2l[box][slot][m'][m] (transposed: for each source
// node m', the p^2 target rows contiguous)
__global__ void k_fmm_m2l_fill(FillArgs a, int level, int p, const float *__restrict__ z, float *__restrict__ m2l) {
  const int nb = 1 << level, P2 = p * p;
  const long total = (long)nb * nb * kIL * P2 * P2;
  const float w = (float)a.n / (float)nb;  // box side in cells
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const int m = (int)(e % P2);
    long t = e / P2;
    const int mp = (int)(t % P2);
    t /= P2;
    const int slot = (int)(t % kIL);
    const long box = t / kIL;
    const int bx = (int)(box % nb), by = (int)(box / nb);
    int ox, oy;
    il_offset(bx & 1, by & 1, slot, &ox, &oy);
    const int cx = bx + ox, cy = by + oy;
    float v = 0.f;
    if (cx >= 0 && cx < nb && cy >= 0 && cy < nb) {
      // node positions in lattice coordinates (cell centre j at index j)
      const float tx = bx * w + 0.5f * w * (z[m % p] + 1.f) - 0.5f;
      const float ty = by * w + 0.5f * w * (z[m / p] + 1.f) - 0.5f;
      const float sx = cx * w + 0.5f * w * (z[mp % p] + 1.f) - 0.5f;
      const float sy = cy * w + 0.5f * w * (z[mp / p] + 1.f) - 0.5f;
      v = kernel_entry(a.sig, a.n, a.P, a.S, a.closed, a.sigma_c, tx, ty, sx, sy);
    }
    m2l[e] = v;
  }
}

// P2M: W[leaf][m] = sum_k Pm[m][k] s_leaf[k]; one CTA per leaf
__global__ void k_fmm_p2m(int n, int L, int b, int P2, const float *__restrict__ Pm, const float *__restrict__ s,
                          float *__restrict__ W) {
  extern __shared__ float sh[];
  const int nl = 1 << L, bb = b * b;
  const int bx = blockIdx.x % nl, by = blockIdx.x / nl;
  for (int k = threadIdx.x; k < bb; k += blockDim.x) sh[k] = s[(long)(by * b + k / b) * n + bx * b + k % b];
  __syncthreads();
  for (int m = threadIdx.x; m < P2; m += blockDim.x) {
    float acc = 0.f;
    for (int k = 0; k < bb; ++k) acc = fmaf(Pm[m * bb + k], sh[k], acc);
    W[(long)blockIdx.x * P2 + m] = acc;
  }
}

// M2M: parent boxes at level l from their children at l + 1
__global__ void k_fmm_m2m(int level, int P2, const float *__restrict__ Cq, const float *__restrict__ Wc,
                          float *__restrict__ Wp) {
  extern __shared__ float sh[];
  const int nb = 1 << level;
  const int bx = blockIdx.x % nb, by = blockIdx.x / nb;
  for (int i = threadIdx.x; i < 4 * P2; i += blockDim.x) {
    const int q = i / P2, mp = i % P2;
    const long child = (long)(2 * by + q / 2) * (2 * nb) + 2 * bx + q % 2;
    sh[i] = Wc[child * P2 + mp];
  }
  __syncthreads();
  for (int m = threadIdx.x; m < P2; m += blockDim.x) {
    float acc = 0.f;
    for (int q = 0; q < 4; ++q)
      for (int mp = 0; mp < P2; ++mp) acc = fmaf(Cq[((long)q * P2 + m) * P2 + mp], sh[q * P2 + mp], acc);
    Wp[(long)blockIdx.x * P2 + m] = acc;
  }
}

// M2L of every level in one launch (the levels do not depend on each other):
// CTA t takes box t - first[l] of the level l with first[l] <= t < first[l + 1],
// the small coarse levels first, so that their latency hides behind the
// streaming of the large fine level.  Lc[B] = sum over the interaction list of
// K_BC W_C.
struct M2LArgs {
  int L;
  long first[32];     // first CTA of each level
  long node_off[32];  // W and Lc offsets of each level
  long m2l_off[32];   // M2L block offsets of each level
};

__global__ void k_fmm_m2l(M2LArgs a, int P2, const float *__restrict__ m2l_all, const float *__restrict__ W_all,
                          float *__restrict__ Lc_all) {
  extern __shared__ float sh[];
  int level = 2;
  while (level < a.L && (long)blockIdx.x >= a.first[level + 1]) ++level;
  const long box = (long)blockIdx.x - a.first[level];
  const float *m2l = m2l_all + a.m2l_off[level];
  const float *W = W_all + a.node_off[level];
  float *Lc = Lc_all + a.node_off[level];
  const int nb = 1 << level;
  const int bx = (int)(box % nb), by = (int)(box / nb);
  for (int i = threadIdx.x; i < kIL * P2; i += blockDim.x) {
    const int slot = i / P2, mp = i % P2;
    int ox, oy;
    il_offset(bx & 1, by & 1, slot, &ox, &oy);
    const int cx = bx + ox, cy = by + oy;
    sh[i] = (cx >= 0 && cx < nb && cy >= 0 && cy < nb) ? W[((long)cy * nb + cx) * P2 + mp] : 0.f;
  }
  __syncthreads();
  // blockDim / P2 groups of P2 threads each take every parts-th source node
  const float *blk = m2l + box * kIL * P2 * P2;
  float *red = sh + kIL * P2;
  const int parts = blockDim.x / P2, m = threadIdx.x % P2, part = threadIdx.x / P2;
  // four independent chains keep four streaming loads in flight per thread
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
  if (part < parts) {
    const int I = kIL * P2;
    int i = part;
    for (; i + 3 * parts < I; i += 4 * parts) {
      a0 = fmaf(__ldcs(blk + (long)i * P2 + m), sh[i], a0);
      a1 = fmaf(__ldcs(blk + (long)(i + parts) * P2 + m), sh[i + parts], a1);
      a2 = fmaf(__ldcs(blk + (long)(i + 2 * parts) * P2 + m), sh[i + 2 * parts], a2);
      a3 = fmaf(__ldcs(blk + (long)(i + 3 * parts) * P2 + m), sh[i + 3 * parts], a3);
    }
    for (; i < I; i += parts) a0 = fmaf(__ldcs(blk + (long)i * P2 + m), sh[i], a0);
  }
  red[threadIdx.x] = (a0 + a1) + (a2 + a3);
  __syncthreads();
  if (threadIdx.x < P2) {
    float t = 0.f;
    for (int q = 0; q < parts; ++q) t += red[q * P2 + threadIdx.x];
    Lc[box * P2 + threadIdx.x] = t;
  }
}

// L2L: child boxes at level l + 1 take their parent's interpolated L
__global__ void k_fmm_l2l(int level, int P2, const float *__restrict__ Cq, const float *__restrict__ Lp,
                          float *__restrict__ Lch) {
  extern __shared__ float sh[];
  const int nc = 2 << level;  // children per side
  const int cx = blockIdx.x % nc, cy = blockIdx.x / nc;
  const int q = (cx & 1) + 2 * (cy & 1);
  const long parent = (long)(cy >> 1) * (nc >> 1) + (cx >> 1);
  for (int m = threadIdx.x; m < P2; m += blockDim.x) sh[m] = Lp[parent * P2 + m];
  __syncthreads();
  for (int mp = threadIdx.x; mp < P2; mp += blockDim.x) {
    float acc = 0.f;
    for (int m = 0; m < P2; ++m) acc = fmaf(Cq[((long)q * P2 + m) * P2 + mp], sh[m], acc);
    Lch[(long)blockIdx.x * P2 + mp] += acc;
  }
}

// leaves: near field from the cached blocks plus L2P; y (FP64) by op
__global__ void k_fmm_leaf(int n, int L, int b, int P2, const float *__restrict__ near, const float *__restrict__ Pm,
                           const float *__restrict__ s, const float *__restrict__ Lc, int op,
                           const double *__restrict__ g, double *__restrict__ y) {
  extern __shared__ float sh[];  // [9][b^2] sources, then [P2] L
  const int nl = 1 << L, bb = b * b;
  const int bx = blockIdx.x % nl, by = blockIdx.x / nl;
  for (int i = threadIdx.x; i < 9 * bb; i += blockDim.x) {
    const int slot = i / bb, k = i % bb;
    const int cx = bx + slot % 3 - 1, cy = by + slot / 3 - 1;
    sh[i] = (cx >= 0 && cx < nl && cy >= 0 && cy < nl) ? s[(long)(cy * b + k / b) * n + cx * b + k % b] : 0.f;
  }
  for (int m = threadIdx.x; m < P2; m += blockDim.x) sh[9 * bb + m] = Lc ? Lc[(long)blockIdx.x * P2 + m] : 0.f;
  __syncthreads();
  // blockDim / bb groups of bb threads each take every parts-th source cell;
  // group 0 adds the far field (L2P)
  const float *blk = near + (long)blockIdx.x * 9 * bb * bb;
  float *red = sh + 9 * bb + P2;
  const int parts = blockDim.x / bb, j = threadIdx.x % bb, part = threadIdx.x / bb;
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
  if (part < parts) {
    const int I = 9 * bb;
    int i = part;
    for (; i + 3 * parts < I; i += 4 * parts) {
      a0 = fmaf(__ldcs(blk + (long)i * bb + j), sh[i], a0);
      a1 = fmaf(__ldcs(blk + (long)(i + parts) * bb + j), sh[i + parts], a1);
      a2 = fmaf(__ldcs(blk + (long)(i + 2 * parts) * bb + j), sh[i + 2 * parts], a2);
      a3 = fmaf(__ldcs(blk + (long)(i + 3 * parts) * bb + j), sh[i + 3 * parts], a3);
    }
    for (; i < I; i += parts) a0 = fmaf(__ldcs(blk + (long)i * bb + j), sh[i], a0);
    if (part == 0)
      for (int m = 0; m < P2; ++m) a1 = fmaf(Pm[m * bb + j], sh[9 * bb + m], a1);
  }
  red[threadIdx.x] = (a0 + a1) + (a2 + a3);
  __syncthreads();
  if (threadIdx.x < bb) {
    double v = 0.0;
    for (int q = 0; q < parts; ++q) v += (double)red[q * bb + threadIdx.x];
    const long jj = (long)(by * b + threadIdx.x / b) * n + bx * b + threadIdx.x % b;
    y[jj] = op == VIE_OP_I_MINUS_K ? g[jj] - v : v;
  }
}

// ---- host: the interpolation matrices in FP64

double s1(int p, double u, double v) {
  u = std::min(1.0, std::max(-1.0, u));
  const double tu = acos(u), tv = acos(v);
  double acc = 1.0 / p;
  for (int k = 1; k < p; ++k) acc += 2.0 / p * cos(k * tu) * cos(k * tv);
  return acc;
}

int blocks_for(long total) { return (int)std::max(1L, std::min((total + 255) / 256, 152L * 64)); }

}  // namespace

void fmm_leaf_levels(int n, int *L, int *b) {
  int l = 0;
  while (n % (2 << l) == 0 && n / (2 << l) >= 8) ++l;
  *L = l;
  *b = n >> l;
}

vie_status fmm_prepare(FmmPlan *fp, int n, int p, const float *sig32, const double *diag, int steps, int closed,
                       double sigma_c, cudaStream_t st) {
  fmm_release(fp);
  int L, b;
  fmm_leaf_levels(n, &L, &b);
  if (L < 2) {
    set_error("vie_assemble_fmm: the grid has no far field (n must be 2^L b with L >= 2 and b >= 8)");
    return VIE_ERR_UNSUPPORTED;
  }
  if (p < 2 || p > 12) {
    set_error("vie_assemble_fmm: order must be in 2..12");
    return VIE_ERR_INVALID_ARG;
  }
  const int P2 = p * p, bb = b * b, nl = 1 << L;
  std::vector<double> z(p);
  for (int i = 0; i < p; ++i) z[i] = cos((2.0 * (i + 1) - 1.0) * kPi / (2.0 * p));
  // P[m][k]: leaf cell k = kx + b ky at u = 2 (kx + 1/2) / b - 1
  std::vector<float> Pm((size_t)P2 * bb), Cq((size_t)4 * P2 * P2), zf(p);
  for (int m = 0; m < P2; ++m)
    for (int k = 0; k < bb; ++k) {
      const double u = 2.0 * (k % b + 0.5) / b - 1.0, v = 2.0 * (k / b + 0.5) / b - 1.0;
      Pm[(size_t)m * bb + k] = (float)(s1(p, u, z[m % p]) * s1(p, v, z[m / p]));
    }
  // C_q[m][m']: child q's node m' in its parent's coordinates
  for (int q = 0; q < 4; ++q)
    for (int m = 0; m < P2; ++m)
      for (int mp = 0; mp < P2; ++mp) {
        const double u = -1.0 + (q % 2) + 0.5 * (z[mp % p] + 1.0);
        const double v = -1.0 + (q / 2) + 0.5 * (z[mp / p] + 1.0);
        Cq[((size_t)q * P2 + m) * P2 + mp] = (float)(s1(p, u, z[m % p]) * s1(p, v, z[m / p]));
      }
  for (int i = 0; i < p; ++i) zf[i] = (float)z[i];
  fp->n = n;
  fp->p = p;
  fp->L = L;
  fp->b = b;
  long nodes = 0;
  for (int l = 2; l <= L; ++l) {
    fp->node_off[l] = nodes;
    nodes += (long)P2 << (2 * l);
  }
  long m2l_total = 0;
  for (int l = 2; l <= L; ++l) {
    fp->m2l_off[l] = m2l_total;
    m2l_total += ((long)kIL * P2 * P2) << (2 * l);
  }
  const long near_total = (long)nl * nl * 9 * bb * bb;
  VIE_CUDA(vie_malloc((void **)&fp->near, sizeof(float) * near_total));
  VIE_CUDA(vie_malloc((void **)&fp->m2l, sizeof(float) * m2l_total));
  VIE_CUDA(vie_malloc((void **)&fp->W, sizeof(float) * nodes));
  VIE_CUDA(vie_malloc((void **)&fp->Lc, sizeof(float) * nodes));
  VIE_CUDA(vie_malloc((void **)&fp->Pm, sizeof(float) * Pm.size()));
  VIE_CUDA(vie_malloc((void **)&fp->Cq, sizeof(float) * Cq.size()));
  VIE_CUDA(vie_malloc((void **)&fp->z, sizeof(float) * p));
  VIE_CUDA(cudaMemcpyAsync(fp->Pm, Pm.data(), sizeof(float) * Pm.size(), cudaMemcpyHostToDevice, st));
  VIE_CUDA(cudaMemcpyAsync(fp->Cq, Cq.data(), sizeof(float) * Cq.size(), cudaMemcpyHostToDevice, st));
  VIE_CUDA(cudaMemcpyAsync(fp->z, zf.data(), sizeof(float) * p, cudaMemcpyHostToDevice, st));
  FillArgs a{sig32, diag, n, n + 1, steps, closed, (float)sigma_c};
  k_fmm_near_fill<<<blocks_for(near_total), 256, 0, st>>>(a, L, b, fp->near);
  VIE_CHECK_LAUNCH("k_fmm_near_fill");
  for (int l = 2; l <= L; ++l) {
    const long cnt = ((long)kIL * P2 * P2) << (2 * l);
    k_fmm_m2l_fill<<<blocks_for(cnt), 256, 0, st>>>(a, l, p, fp->z, fp->m2l + fp->m2l_off[l]);
    VIE_CHECK_LAUNCH("k_fmm_m2l_fill");
  }
  VIE_CUDA(cudaStreamSynchronize(st));
  fp->near_floats = near_total;
  fp->m2l_floats = m2l_total;
  fp->on = 1;
  return VIE_OK;
}

void fmm_release(FmmPlan *fp) {
  if (fp->near) vie_free(fp->near);
  if (fp->m2l) vie_free(fp->m2l);
  if (fp->W) vie_free(fp->W);
  if (fp->Lc) vie_free(fp->Lc);
  if (fp->Pm) vie_free(fp->Pm);
  if (fp->Cq) vie_free(fp->Cq);
  if (fp->z) vie_free(fp->z);
  *fp = FmmPlan{};
}

vie_status fmm_apply(const FmmPlan &fp, int op, const float *s, const double *g, double *y, cudaStream_t st) {
  const int n = fp.n, L = fp.L, b = fp.b, P2 = fp.p * fp.p, bb = b * b;
  const int nl = 1 << L;
  const int t = 128, tm = std::max(P2, 256 / P2 * P2), tl = std::max(bb, 256 / bb * bb);
  // upward pass
  k_fmm_p2m<<<nl * nl, t, sizeof(float) * bb, st>>>(n, L, b, P2, fp.Pm, s, fp.W + fp.node_off[L]);
  VIE_CHECK_LAUNCH("k_fmm_p2m");
  for (int l = L - 1; l >= 2; --l) {
    k_fmm_m2m<<<1 << (2 * l), t, sizeof(float) * 4 * P2, st>>>(l, P2, fp.Cq, fp.W + fp.node_off[l + 1],
                                                              fp.W + fp.node_off[l]);
    VIE_CHECK_LAUNCH("k_fmm_m2m");
  }
  // interactions (all levels in one launch), then the downward pass
  {
    M2LArgs a;
    a.L = L;
    long first = 0;
    for (int l = 2; l <= L; ++l) {
      a.first[l] = first;
      a.node_off[l] = fp.node_off[l];
      a.m2l_off[l] = fp.m2l_off[l];
      first += 1L << (2 * l);
    }
    a.first[L + 1] = first;
    k_fmm_m2l<<<(unsigned)first, tm, sizeof(float) * (kIL * P2 + tm), st>>>(a, P2, fp.m2l, fp.W, fp.Lc);
    VIE_CHECK_LAUNCH("k_fmm_m2l");
  }
  for (int l = 2; l < L; ++l) {
    k_fmm_l2l<<<1 << (2 * (l + 1)), t, sizeof(float) * P2, st>>>(l, P2, fp.Cq, fp.Lc + fp.node_off[l],
                                                                  fp.Lc + fp.node_off[l + 1]);
    VIE_CHECK_LAUNCH("k_fmm_l2l");
  }
  k_fmm_leaf<<<nl * nl, tl, sizeof(float) * (9 * bb + P2 + tl), st>>>(
      n, L, b, P2, fp.near, fp.Pm, s, fp.Lc + fp.node_off[L], op, g, y);
  VIE_CHECK_LAUNCH("k_fmm_leaf");
  return VIE_OK;
}

}  // namespace vie
