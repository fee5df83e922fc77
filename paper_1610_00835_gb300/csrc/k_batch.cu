// Batched operator apply over several 2D media of different sizes in one
// persistent launch (the operator of Section 3.2, M-iii, for each medium).
//
// Every grid's targets are cut into tiles of 128 cells and its unordered tile
// pairs (a <= b) form its items, exactly as in the symmetric single-grid
// kernel (k_pairs_sym.cu).  Items are grouped in batches of GROUPS items of
// one grid; a CTA of GROUPS x 128 threads takes batches from a global counter
// and gives one item to each of its groups.  When a batch belongs to another
// grid than the previous one, the CTA re-stages that grid's sigma_t lattice
// into shared memory; grids whose lattice does not fit read it from global
// memory through L1 instead.  The last CTA to finish resets the counter, so
// the launch can be replayed from a CUDA graph.  Per-grid partial sums
// [T][N] are reduced by the single-grid reduce kernel, one launch per grid.
// With the automatic kernel choice, every grid that the displacement kernel
// takes (k_pairs_disp.cu: 2 <= n <= 258) runs it instead, one launch of its
// own in the same graph, and only the others go to the persistent launch.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <string>
#include <vector>

#include "march.cuh"
#include "vie_internal.cuh"

namespace vie {

namespace {

using namespace march;

constexpr int kG = 128;  // targets per tile = threads per group

struct BatchGrid {
  int n, ldp;             // cells per side, lattice row stride (= n + 1)
  int T, n_items;         // tiles, items (tile pairs)
  int smem;               // 1: lattice staged in shared memory
  int pad;
  long N;
  long lat_off;           // floats, into the packed lattice buffer
  long lat_elems;
  long cell_off;          // cells, into packed src / y / diag
  long part_off;          // doubles, into the packed partial buffer
  long item_off;          // into the packed item list
  long batch_begin;       // first batch of this grid
  float tau_scale2, wcoef;
};

struct BatchArgs {
  const BatchGrid *grids;
  int count;
  long n_batches;
  const float *lattice;   // packed lattices (stride ldp, P rows)
  const float *src;       // packed s_k
  double *partial;        // packed [T][N] per grid
  const int2 *items;      // packed (a, b) per grid
  int *counter;           // [2]
};

__device__ __forceinline__ void gbar(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(kG) : "memory");
}

template <int GROUPS>
__global__ void __launch_bounds__(kG *GROUPS, 1) k_pairs_batch(BatchArgs a) {
  extern __shared__ float4 smem[];
  float4 *srcs_all = smem;                                            // [GROUPS][kG]
  float *col_all = reinterpret_cast<float *>(smem + GROUPS * kG);     // [GROUPS][4][kG]
  int *ctl = reinterpret_cast<int *>(col_all + GROUPS * 4 * kG);      // [4]
  float *lat = reinterpret_cast<float *>(ctl + 4);
  const int tid = threadIdx.x;
  const int grp = tid / kG, t = tid % kG, warp = t / 32, lane = t % 32;
  float4 *srcs = srcs_all + grp * kG;
  float *colw = col_all + grp * 4 * kG;
  int cur = -1;
  for (;;) {
    if (tid == 0) ctl[0] = (int)atomicAdd(a.counter, 1);
    __syncthreads();
    const long batch = ctl[0];
    if (batch >= a.n_batches) break;
    int gi = 0;
    while (gi + 1 < a.count && a.grids[gi + 1].batch_begin <= batch) ++gi;
    const BatchGrid G = a.grids[gi];
    if (gi != cur) {
      if (G.smem) {
        const float *src = a.lattice + G.lat_off;
        for (long i = tid; i < G.lat_elems; i += kG * GROUPS) lat[i] = src[i];
      }
      cur = gi;
      __syncthreads();
    }
    const long item = (batch - G.batch_begin) * GROUPS + grp;
    if (item < G.n_items) {
      const int2 ab = a.items[G.item_off + item];
      const int n = G.n;
      const long N = G.N;
      const long j_raw = (long)ab.x * kG + t;
      const bool jvalid = j_raw < N;
      const long j = jvalid ? j_raw : N - 1;
      const float jx = (float)(j % n), jy = (float)(j / n);
      const float *src = a.src + G.cell_off;
      const float sj = jvalid ? src[j] : 0.f;
      {
        const long k = (long)ab.y * kG + t;
        const bool kvalid = k < N;
        const long kc = kvalid ? k : N - 1;
        srcs[t] = make_float4((float)(kc % n), (float)(kc / n), 0.f, kvalid ? src[kc] : 0.f);
      }
      gbar(grp);
      const bool diag_item = ab.x == ab.y;
      Geo geo{};
      GeoG geog{};
      if (G.smem) {
        geo = make_geo((unsigned)__cvta_generic_to_shared(lat), 2, (unsigned)G.ldp, 0u);
      } else {
        geog.base = a.lattice + G.lat_off;
        geog.ldp = G.ldp;
        geog.bias = kTwo23Bits * (1u + (unsigned)G.ldp);
      }
      double dsum = 0.0;
#pragma unroll 1
      for (int c0 = 0; c0 < kG; c0 += 64) {
        float fsum = 0.f;
#pragma unroll 1
        for (int c = c0; c < c0 + 64; ++c) {
          const float4 q = srcs[c];
          const float dx = q.x - jx, dy = q.y - jy;
          const float r2 = fmaf(dy, dy, dx * dx);
          const float inv_r = rsqrtf(r2);
          const float r = r2 * inv_r;
          const float acc = G.smem ? march64<2, 0, 0>(geo, jx, jy, 0.f, dx, dy, 0.f)
                                   : march64_g(geog, jx, jy, dx, dy);
          float w = G.wcoef * exp2f(-G.tau_scale2 * acc * r) * inv_r;
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
      double *part = a.partial + G.part_off;
      if (jvalid) part[(long)ab.y * N + j] = dsum;
      if (!diag_item) {
        gbar(grp);
        const long k = (long)ab.y * kG + t;
        if (k < N)
          part[(long)ab.x * N + k] =
              (double)((colw[t] + colw[kG + t]) + (colw[2 * kG + t] + colw[3 * kG + t]));
      }
    }
    __syncthreads();  // every group done before the next batch may re-stage
  }
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(a.counter + 1, 1) == (int)gridDim.x - 1) {
      a.counter[0] = 0;
      a.counter[1] = 0;
      __threadfence();
    }
  }
}

// copy a padded (stride P) lattice into the packed buffer (stride ldp = P)
__global__ void k_pad_lattice(int n, const double *__restrict__ sig, float *__restrict__ out) {
  const int P = n + 1;
  const long total = (long)P * P;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long x = min(i % P, (long)n - 1), y = min(i / P, (long)n - 1);
    out[i] = (float)sig[y * n + x];
  }
}

size_t batch_smem(int groups, long max_lat) {
  return sizeof(float4) * groups * kG + sizeof(float) * groups * 4 * kG + 16 + sizeof(float) * max_lat;
}

const void *batch_kernel(int groups) {
  switch (groups) {
    case 2: return (const void *)k_pairs_batch<2>;
    case 4: return (const void *)k_pairs_batch<4>;
    default: return (const void *)k_pairs_batch<8>;
  }
}

}  // namespace

// ------------------------------------------------------------- host side

struct BatchPlanImpl {
  int groups = 8;
  int smem_policy = 0;   // 0: stage every lattice that fits, 1: only up to 128 KB
  std::vector<BatchGrid> host;
  BatchGrid *grids = nullptr;
  int2 *items = nullptr;
  long n_batches = 0;
  long max_smem_lat = 0;
  size_t smem = 0;
  int grid = 0;
};

vie_status batch_plan(BatchPlanImpl *bp, int count, const int *ns, const long *cell_off,
                      const long *lat_off, const long *part_off, const int *skip, int groups, int smem_policy,
                      int device) {
  DevProps prop;
  VIE_TRY(get_dev_props(device, &prop));
  bp->groups = groups;
  bp->smem_policy = smem_policy;
  bp->host.assign(count, BatchGrid{});
  const size_t fixed = batch_smem(groups, 0);
  const long lat_limit_policy = smem_policy == 1 ? 32768 : (1L << 40);
  const long lat_limit_smem = ((long)prop.sharedMemPerBlockOptin - (long)fixed) / 4;
  std::vector<int2> items;
  long nb = 0, max_lat = 0;
  for (int i = 0; i < count; ++i) {
    BatchGrid &G = bp->host[i];
    const int n = ns[i];
    G.n = n;
    G.ldp = n + 1;
    G.N = (long)n * n;
    G.T = (int)((G.N + kG - 1) / kG);
    G.n_items = G.T * (G.T + 1) / 2;
    G.lat_elems = (long)(n + 1) * (n + 1);
    G.smem = (G.lat_elems <= lat_limit_smem && G.lat_elems <= lat_limit_policy) ? 1 : 0;
    if (G.smem && !skip[i]) max_lat = std::max(max_lat, G.lat_elems);
    G.lat_off = lat_off[i];
    G.cell_off = cell_off[i];
    G.part_off = part_off[i];
    G.item_off = (long)items.size();
    G.batch_begin = nb;
    if (skip[i]) {
      G.n_items = 0;  // this grid runs the displacement kernel instead
      G.smem = 0;
    } else {
      nb += (G.n_items + groups - 1) / groups;
      for (int a = 0; a < G.T; ++a)
        for (int b = a; b < G.T; ++b) items.push_back(make_int2(a, b));
    }
    const double h = 1.0 / n;
    G.tau_scale2 = (float)(h / kS * 1.4426950408889634);
    G.wcoef = (float)(h / (2.0 * kPi));
  }
  bp->n_batches = nb;
  bp->max_smem_lat = max_lat;
  if (bp->grids) vie_free(bp->grids);
  if (bp->items) vie_free(bp->items);
  bp->grids = nullptr;
  bp->items = nullptr;
  VIE_CUDA(vie_malloc((void **)&bp->grids, sizeof(BatchGrid) * count));
  VIE_CUDA(cudaMemcpy(bp->grids, bp->host.data(), sizeof(BatchGrid) * count, cudaMemcpyHostToDevice));
  VIE_CUDA(vie_malloc((void **)&bp->items, sizeof(int2) * std::max<size_t>(1, items.size())));
  if (!items.empty())
    VIE_CUDA(cudaMemcpy(bp->items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice));
  bp->smem = batch_smem(groups, max_lat);
  const void *k = batch_kernel(groups);
  VIE_TRY(raise_smem_limit(k, (size_t)((int)bp->smem)));
  int bps = 0;
  VIE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, kG * groups, bp->smem));
  if (bps < 1) {
    set_error("batch: kernel does not fit on an SM");
    return VIE_ERR_UNSUPPORTED;
  }
  bp->grid = (int)std::min<long>((long)bps * prop.multiProcessorCount, nb);  // 0: nothing to launch
  return VIE_OK;
}

void batch_plan_free(BatchPlanImpl *bp) {
  if (bp->grids) vie_free(bp->grids);
  if (bp->items) vie_free(bp->items);
  bp->grids = nullptr;
  bp->items = nullptr;
}

vie_status batch_pad_lattice(int n, const double *sig, float *out, cudaStream_t st) {
  const long total = (long)(n + 1) * (n + 1);
  k_pad_lattice<<<(int)std::min((total + 255) / 256, 4096L), 256, 0, st>>>(n, sig, out);
  VIE_CHECK_LAUNCH("k_pad_lattice");
  return VIE_OK;
}

vie_status batch_launch(const BatchPlanImpl &bp, const float *lattice, const float *src,
                        double *partial, int *counter, cudaStream_t st) {
  if (bp.grid < 1) return VIE_OK;  // every grid runs the displacement kernel
  BatchArgs a;
  a.grids = bp.grids;
  a.count = (int)bp.host.size();
  a.n_batches = bp.n_batches;
  a.lattice = lattice;
  a.src = src;
  a.partial = partial;
  a.items = bp.items;
  a.counter = counter;
  void *args[] = {&a};
  VIE_CUDA(cudaLaunchKernel(batch_kernel(bp.groups), dim3(bp.grid), dim3(kG * bp.groups), args,
                            bp.smem, st));
  count_launch();
  return VIE_OK;
}

}  // namespace vie

// ------------------------------------------------------------- C ABI

using namespace vie;

struct vie_batch {
  int device = 0;
  int count = 0;
  std::vector<int> ns;
  std::vector<long> cell_off, lat_off, part_off;  // count + 1 entries each
  double *sig_t = nullptr, *sig_s = nullptr, *diag = nullptr;
  float *lattice = nullptr, *src = nullptr;
  double *partial = nullptr;
  int *counter = nullptr;
  BatchPlanImpl plan;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int key_op = -1, key_nrhs = 0;
  const void *key_g = nullptr;
  const void *key_y = nullptr;
  int graph_kernels = 0;
  double *stage_g = nullptr, *stage_y = nullptr;
  long stage_cap = 0;          // doubles in each staging buffer
  std::vector<DispPlan> disp;  // per grid: the displacement kernel, when it takes the grid
  std::vector<int> use_disp;
};

namespace {

void batch_free(vie_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (void *p : {(void *)b->sig_t, (void *)b->sig_s, (void *)b->diag, (void *)b->lattice,
                  (void *)b->src, (void *)b->partial, (void *)b->counter, (void *)b->stage_g,
                  (void *)b->stage_y})
    if (p) vie_free(p);
  batch_plan_free(&b->plan);
  for (auto &d : b->disp) disp_release(&d);
}

bool dev_ptr(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

vie_status bad(const char *m) {
  set_error(m);
  return VIE_ERR_INVALID_ARG;
}

vie_status replan(vie_batch *b, int groups, int policy) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->key_op = -1;
  return batch_plan(&b->plan, b->count, b->ns.data(), b->cell_off.data(), b->lat_off.data(),
                    b->part_off.data(), b->use_disp.data(), groups, policy, b->device);
}

// Queue one batched apply on stream st (also used under graph capture);
// *kernels = the launches queued.
vie_status enqueue_one(vie_batch *b, int op, const double *g, double *y, cudaStream_t st, int *kernels) {
  const long total = b->cell_off[b->count];
  vie_status s = launch_source_prep(total, op, b->sig_s, g, VIE_PREC_FP32, b->src, st);
  if (s != VIE_OK) return s;
  int k = 1;
  if ((s = batch_launch(b->plan, b->lattice, b->src, b->partial, b->counter, st)) != VIE_OK) return s;
  if (b->plan.grid > 0) ++k;
  for (int i = 0; i < b->count; ++i) {
    const long off = b->cell_off[i];
    const BatchGrid &G = b->plan.host[i];
    if (b->use_disp[i]) {
      const DispPlan &dp = b->disp[i];
      const double h = 1.0 / G.n;
      if ((s = disp_source(dp, G.N, op, b->sig_s + off, g + off, b->src + off, st)) != VIE_OK) return s;
      if ((s = disp_launch(dp, G.n, (float)(h / kS * 1.4426950408889634), (float)(h / (2.0 * kPi)), b->src + off,
                           st)) != VIE_OK)
        return s;
      if ((s = disp_reduce(dp, G.N, op, b->diag + off, b->sig_s + off, g + off, y + off, st)) != VIE_OK) return s;
      k += 3;
    } else {
      if ((s = launch_reduce(G.N, G.T, op, b->partial + b->part_off[i], b->diag + off, b->sig_s + off, g + off,
                             y + off, st)) != VIE_OK)
        return s;
      ++k;
    }
  }
  *kernels = k;
  return VIE_OK;
}

// nrhs sources one after the other: source r reads g + r total and writes
// y + r total (the scratch buffers are reused in stream order)
vie_status enqueue(vie_batch *b, int op, const double *g, double *y, int nrhs, cudaStream_t st, int *kernels) {
  const long total = b->cell_off[b->count];
  *kernels = 0;
  for (int r = 0; r < nrhs; ++r) {
    int k = 0;
    vie_status s = enqueue_one(b, op, g + (size_t)r * total, y + (size_t)r * total, st, &k);
    if (s != VIE_OK) return s;
    *kernels += k;
  }
  return VIE_OK;
}

}  // namespace

extern "C" {

vie_status vie_batch_create(vie_batch **out, int count, const vie_grid *grids,
                            const double *const *sigma_t, const double *const *sigma_s,
                            const vie_opts *o) {
  if (!out || !grids || !sigma_t || !sigma_s || count < 1 || count > 1024)
    return bad("vie_batch_create: bad arguments (1 <= count <= 1024)");
  *out = nullptr;
  vie_opts opts;
  vie_default_opts(&opts);
  if (o) opts = *o;
  if (opts.steps != 64 || opts.tau_mode != VIE_TAU_MARCH || opts.precision != VIE_PREC_FP32 ||
      opts.disc != VIE_DISC_MIII)
    return bad("vie_batch_create: the batch supports FP32 tiles with the S = 64 march and M-iii");
  if (opts.kernel != VIE_KERNEL_AUTO && opts.kernel != VIE_KERNEL_SYMMETRIC &&
      opts.kernel != VIE_KERNEL_DISPLACEMENT)
    return bad("vie_batch_create: kernel must be AUTO, SYMMETRIC or DISPLACEMENT");
  for (int i = 0; i < count; ++i) {
    if (grids[i].dim != 2 || grids[i].n < 1 || grids[i].n > 4096)
      return bad("vie_batch_create: 2D grids with 1 <= n <= 4096");
    const long N = (long)grids[i].n * grids[i].n;
    if (!sigma_t[i] || !sigma_s[i]) return bad("vie_batch_create: NULL coefficient array");
    for (long k = 0; k < N; ++k) {
      if (!isfinite(sigma_t[i][k]) || !isfinite(sigma_s[i][k])) {
        set_error("vie_batch_create: non-finite coefficient");
        return VIE_ERR_NONFINITE;
      }
      if (sigma_t[i][k] < 0 || sigma_s[i][k] < 0) return bad("vie_batch_create: negative coefficient");
    }
  }
  int prev = -1;
  cudaGetDevice(&prev);
  VIE_CUDA(cudaSetDevice(opts.device));
  vie_batch *b = new vie_batch();
  b->device = opts.device;
  b->count = count;
  b->cell_off.assign(count + 1, 0);
  b->lat_off.assign(count + 1, 0);
  b->part_off.assign(count + 1, 0);
  for (int i = 0; i < count; ++i) {
    const int n = grids[i].n;
    const long N = (long)n * n, T = (N + 127) / 128;
    b->ns.push_back(n);
    b->cell_off[i + 1] = b->cell_off[i] + N;
    b->lat_off[i + 1] = b->lat_off[i] + ((long)(n + 1) * (n + 1) + 3) / 4 * 4;  // 16-byte aligned
    b->part_off[i + 1] = b->part_off[i] + T * N;
  }
  const long cells = b->cell_off[count];
  vie_status s = VIE_OK;
  auto fail = [&](vie_status st) {
    batch_free(b);
    delete b;
    if (prev >= 0) cudaSetDevice(prev);
    return st;
  };
#define BTRY(call)                                            \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return fail(cuda_fail(_e, #call)); \
  } while (0)
  BTRY(vie_malloc(&b->sig_t, sizeof(double) * cells));
  BTRY(vie_malloc(&b->sig_s, sizeof(double) * cells));
  BTRY(vie_malloc(&b->diag, sizeof(double) * cells));
  BTRY(vie_malloc(&b->src, sizeof(float) * cells));
  BTRY(vie_malloc(&b->lattice, sizeof(float) * b->lat_off[count]));
  BTRY(vie_malloc(&b->partial, sizeof(double) * b->part_off[count]));
  BTRY(vie_malloc(&b->counter, 2 * sizeof(int)));
  BTRY(cudaMemset(b->counter, 0, 2 * sizeof(int)));
  BTRY(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  for (int i = 0; i < count; ++i) {
    const long N = (long)b->ns[i] * b->ns[i];
    BTRY(cudaMemcpy(b->sig_t + b->cell_off[i], sigma_t[i], sizeof(double) * N, cudaMemcpyHostToDevice));
    BTRY(cudaMemcpy(b->sig_s + b->cell_off[i], sigma_s[i], sizeof(double) * N, cudaMemcpyHostToDevice));
    if ((s = batch_pad_lattice(b->ns[i], b->sig_t + b->cell_off[i], b->lattice + b->lat_off[i], 0)) != VIE_OK)
      return fail(s);
    if ((s = launch_selfcell(2, b->ns[i], b->sig_t + b->cell_off[i], b->diag + b->cell_off[i], 0)) != VIE_OK)
      return fail(s);
  }
  b->disp.assign(count, DispPlan{});
  b->use_disp.assign(count, 0);
  if (opts.kernel != VIE_KERNEL_SYMMETRIC) {
    BTRY(cudaDeviceSynchronize());
    for (int i = 0; i < count; ++i) {
      if ((s = disp_prepare(&b->disp[i], b->ns[i], b->lattice + b->lat_off[i], opts.device, 0)) != VIE_OK)
        return fail(s);
      b->use_disp[i] = b->disp[i].usable;
    }
  }
  if ((s = replan(b, 8, 0)) != VIE_OK) return fail(s);
  BTRY(cudaDeviceSynchronize());
#undef BTRY
  if (prev >= 0) cudaSetDevice(prev);
  *out = b;
  return VIE_OK;
}

vie_status vie_batch_destroy(vie_batch *b) {
  if (!b) return VIE_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  batch_free(b);
  delete b;
  if (prev >= 0) cudaSetDevice(prev);
  return VIE_OK;
}

vie_status vie_batch_layout(vie_batch *b, long long *total_cells, long long *offsets) {
  if (!b) return bad("vie_batch_layout: NULL batch");
  if (total_cells) *total_cells = b->cell_off[b->count];
  if (offsets)
    for (int i = 0; i <= b->count; ++i) offsets[i] = b->cell_off[i];
  return VIE_OK;
}

vie_status vie_batch_apply(vie_batch *b, vie_op op, const double *g, double *y, int nrhs, void *stream) {
  if (!b || !g || !y) return bad("vie_batch_apply: NULL argument");
  if (op != VIE_OP_K_SIGMA_S && op != VIE_OP_I_MINUS_K && op != VIE_OP_A_RAW)
    return bad("vie_batch_apply: unknown op");
  if (nrhs < 1 || nrhs > 4096) return bad("vie_batch_apply: 1 <= nrhs <= 4096");
  int prev = -1;
  cudaGetDevice(&prev);
  VIE_CUDA(cudaSetDevice(b->device));
  cudaStream_t st = (cudaStream_t)stream;
  const long cells = b->cell_off[b->count] * (long)nrhs;
  const bool gd = dev_ptr(g), yd = dev_ptr(y);
  const double *gg = g;
  double *yy = y;
  if ((!gd || !yd) && b->stage_cap < cells) {
    // grow both staging buffers (a graph captured on the old ones is dropped)
    VIE_CUDA(cudaStreamSynchronize(st));
    if (b->stage_g) vie_free(b->stage_g);
    if (b->stage_y) vie_free(b->stage_y);
    b->stage_g = b->stage_y = nullptr;
    b->stage_cap = 0;
    VIE_CUDA(vie_malloc(&b->stage_g, sizeof(double) * cells));
    VIE_CUDA(vie_malloc(&b->stage_y, sizeof(double) * cells));
    b->stage_cap = cells;
    b->key_op = -1;
  }
  if (!gd) {
    VIE_CUDA(cudaMemcpyAsync(b->stage_g, g, sizeof(double) * cells, cudaMemcpyHostToDevice, st));
    gg = b->stage_g;
  }
  if (!yd) yy = b->stage_y;
  if (!b->exec || b->key_op != (int)op || b->key_g != gg || b->key_y != yy || b->key_nrhs != nrhs) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    VIE_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    int kernels = 0;
    vie_status s = enqueue(b, op, gg, yy, nrhs, b->cap, &kernels);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
    if (s != VIE_OK) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();  // the invalidated capture's error is reported through s
      return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    b->graph = graph;
    VIE_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
    b->key_op = op;
    b->key_g = gg;
    b->key_y = yy;
    b->key_nrhs = nrhs;
    b->graph_kernels = kernels;
  }
  VIE_CUDA(cudaGraphLaunch(b->exec, st));
  for (int i = 0; i < b->graph_kernels; ++i) count_launch();
  if (!yd) {
    VIE_CUDA(cudaMemcpyAsync(y, yy, sizeof(double) * cells, cudaMemcpyDeviceToHost, st));
    VIE_CUDA(cudaStreamSynchronize(st));
  }
  if (prev >= 0) cudaSetDevice(prev);
  return VIE_OK;
}

vie_status vie_batch_config(vie_batch *b, int *groups, int *smem_policy) {
  if (!b) return bad("vie_batch_config: NULL batch");
  if (groups) *groups = b->plan.groups;
  if (smem_policy) *smem_policy = b->plan.smem_policy;
  return VIE_OK;
}

vie_status vie_batch_autotune(vie_batch *b, const char *cache_path, void *stream) {
  if (!b) return bad("vie_batch_autotune: NULL batch");
  int prev = -1;
  cudaGetDevice(&prev);
  VIE_CUDA(cudaSetDevice(b->device));
  cudaDeviceProp prop;
  VIE_CUDA(cudaGetDeviceProperties(&prop, b->device));
  std::string key = std::string(prop.name) + "|";
  for (int n : b->ns) key += std::to_string(n) + ",";
  // cache lines: "<key> <groups> <policy>"
  if (cache_path) {
    FILE *fp = fopen(cache_path, "r");
    if (fp) {
      char line[8192];
      while (fgets(line, sizeof line, fp)) {
        std::string l(line);
        const size_t sp = l.rfind(' ', l.rfind(' ') - 1);
        if (sp == std::string::npos || l.substr(0, sp) != key) continue;
        int gr = 0, pol = 0;
        if (sscanf(l.c_str() + sp, "%d %d", &gr, &pol) == 2 && (gr == 2 || gr == 4 || gr == 8) &&
            (pol == 0 || pol == 1)) {
          fclose(fp);
          vie_status s = replan(b, gr, pol);
          if (prev >= 0) cudaSetDevice(prev);
          return s;
        }
      }
      fclose(fp);
    }
  }
  const long cells = b->cell_off[b->count];
  double *g = nullptr, *y = nullptr;
  VIE_CUDA(vie_malloc(&g, sizeof(double) * cells));
  VIE_CUDA(vie_malloc(&y, sizeof(double) * cells));
  VIE_CUDA(cudaMemset(g, 0, sizeof(double) * cells));
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  VIE_CUDA(cudaEventCreate(&e0));
  VIE_CUDA(cudaEventCreate(&e1));
  const int cand[][2] = {{8, 0}, {4, 0}, {2, 0}, {8, 1}};
  float best = 1e30f;
  int best_i = 0;
  vie_status s = VIE_OK;
  for (int c = 0; c < 4 && s == VIE_OK; ++c) {
    if ((s = replan(b, cand[c][0], cand[c][1])) != VIE_OK) break;
    if ((s = vie_batch_apply(b, VIE_OP_K_SIGMA_S, g, y, 1, st)) != VIE_OK) break;  // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < 2 && s == VIE_OK; ++r) s = vie_batch_apply(b, VIE_OP_K_SIGMA_S, g, y, 1, st);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      best_i = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  vie_free(g);
  vie_free(y);
  if (s == VIE_OK) s = replan(b, cand[best_i][0], cand[best_i][1]);
  if (s == VIE_OK && cache_path) {
    FILE *fp = fopen(cache_path, "a");
    if (fp) {
      fprintf(fp, "%s %d %d\n", key.c_str(), cand[best_i][0], cand[best_i][1]);
      fclose(fp);
    }
  }
  if (prev >= 0) cudaSetDevice(prev);
  return s;
}

}  // extern "C"
