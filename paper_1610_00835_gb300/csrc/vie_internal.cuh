// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/vie.h"

namespace vie {

constexpr double kPi = 3.14159265358979323846;
constexpr int kPairThreads = 256;  // targets per pair-kernel CTA

// Thread-local message behind vie_last_error().
void set_error(const std::string &msg);

// Bounds of the device-side waits of the tensor-core kernels, in clock
// cycles: `limit` for every wait, except the first producer/consumer wait of
// each CTA, which takes `first` (a shorter value lets a test make that wait
// run out); draining already issued copies and products after an abort
// always takes `limit`.  wait_limits(device) converts the process-wide
// setting of vie_set_wait_limits with the device's clock rate.
// Device memory of the library (vie_mem.cu): a caching allocator in front of
// cudaMalloc / cudaFree, same contract (vie_free synchronises the device, as
// cudaFree does, unless a DeviceIdle is alive on the calling thread).
cudaError_t vie_malloc(void **p, size_t bytes);
template <typename T>
inline cudaError_t vie_malloc(T **p, size_t bytes) {
  return vie_malloc(reinterpret_cast<void **>(p), bytes);
}
cudaError_t vie_free(void *p);
// the same for pinned host buffers (cudaMallocHost / cudaFreeHost)
cudaError_t vie_malloc_host(void **p, size_t bytes);
template <typename T>
inline cudaError_t vie_malloc_host(T **p, size_t bytes) {
  return vie_malloc_host(reinterpret_cast<void **>(p), bytes);
}
cudaError_t vie_free_host(void *p);
void vie_release_cached_memory();
// the caller has synchronised the device: frees need not wait for it again
struct DeviceIdle {
  DeviceIdle();
  ~DeviceIdle();
};

#ifdef __CUDACC__
// bf16 bits of v rounded to nearest even (finite v), in integer arithmetic (the
// FP32 -> BF16 conversion instruction shares GB300's narrow FP64 pipe)
__device__ __forceinline__ unsigned short bf16_bits_rn(float v) {
  const unsigned u = __float_as_uint(v);
  return (unsigned short)((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
}
#endif

struct WaitLimits {
  long long limit, first;
};
WaitLimits wait_limits(int device);

// The two device properties the launch planners read, queried once per device
// (cudaGetDeviceProperties is a slow driver round trip, too slow per apply).
struct DevProps {
  size_t sharedMemPerBlockOptin;
  int multiProcessorCount;
};
vie_status get_dev_props(int device, DevProps *out);

// Map a CUDA error to VIE_ERR_CUDA with a message naming the call site.
vie_status cuda_fail(cudaError_t e, const char *what);

// Count one kernel launch of this library (reported by vie_kernel_launches).
void count_launch();

#define VIE_CUDA(call)                                     \
  do {                                                     \
    cudaError_t _e = (call);                               \
    if (_e != cudaSuccess) return ::vie::cuda_fail(_e, #call); \
  } while (0)

#define VIE_TRY(call)                                      \
  do {                                                     \
    vie_status _s = (call);                                \
    if (_s != VIE_OK) return _s;                           \
  } while (0)

// Raise kernel k's dynamic shared-memory limit to at least `bytes`, never
// lower it: a kernel instance is shared by handles of different sizes.
vie_status raise_smem_limit(const void *k, size_t bytes);

#define VIE_CHECK_LAUNCH(what)                             \
  do {                                                     \
    cudaError_t _e = cudaGetLastError();                   \
    if (_e != cudaSuccess) return ::vie::cuda_fail(_e, what); \
    ::vie::count_launch();                                 \
  } while (0)

// Device-side description of one medium, used by the pair kernels.
struct Medium {
  int dim;
  int n;              // cells per side
  int P;              // n + 1, stride of the padded sigma_t lattice
  long N;             // n^dim
  const float *sig32; // padded FP32 sigma_t, P^dim, pad = copy of the edge
  const double *sig64;// padded FP64 sigma_t
  double sigma_c;     // constant sigma_t (closed-form tau)
};

// Launch plan of the FP32 pair kernel for one medium.
struct PairPlan {
  int smem_sigma;     // 1: sigma_t staged in shared memory
  int tiles;          // target tiles of kPairThreads
  int splits;         // source splits (cross-CTA partial sums)
  int chunk;          // sources per split
  int grid;           // CTAs launched
  size_t smem_bytes;  // dynamic shared memory per CTA
};

// ---- apply kernels (k_apply.cu)
vie_status plan_pairs(const Medium &m, int steps, int tau_closed, int precision, int device,
                      PairPlan *plan);
// src: per-source value s_k (FP32 for precision FP32, FP64 otherwise), [N]
// partial: [plan.splits][N] FP64
vie_status launch_pairs(const Medium &m, const PairPlan &plan, int steps, int tau_closed,
                        int precision, const void *src, double *partial, cudaStream_t st);
vie_status launch_source_prep(long N, int op, const double *sigma_s, const double *g,
                              int precision, void *src, cudaStream_t st);
vie_status launch_reduce(long N, int splits, int op, const double *partial, const double *diag,
                         const double *sigma_s, const double *g, double *y, cudaStream_t st);
vie_status launch_pad_sigma(int dim, int n, const double *sig, float *out32, double *out64,
                            cudaStream_t st);
vie_status launch_selfcell(int dim, int n, const double *sigma_t, double *diag,
                           cudaStream_t st);

// ---- symmetric pair kernel (k_pairs_sym.cu): FP32 tiles, S = 64, lattice
// in shared memory.  partial must hold [T][N] doubles.
struct SymPlan {
  int usable = 0;
  int global_lattice = 0;  // 1: 2D lattice read from global memory (too large to stage)
  int T = 0, n_items = 0, ldp = 0, plane = 0, grid = 0;
  size_t smem = 0;
  long lattice_elems = 0;
  int2 *items = nullptr;
  int *counter = nullptr;
  float *lattice = nullptr;
  const void *kernel = nullptr;
};
size_t sym_smem_bytes(int dim, int n, int *ldp, int *plane);
vie_status sym_prepare(SymPlan *sp, int dim, int n, long N, const float *sig_padded, int device,
                       cudaStream_t st);
void sym_release(SymPlan *sp);
// the symmetric plan on caller-owned buffers (lattice_mem: max_lattice floats,
// items for max_T target tiles); unusable (sp->usable = 0, nothing launched)
// when the grid needs more
vie_status sym_plan_external(SymPlan *sp, int dim, int n, long N, const float *sig_padded,
                             int device, int2 *items_mem, int *counter_mem, float *lattice_mem,
                             long max_lattice, int max_T, cudaStream_t st);
vie_status sym_launch(const SymPlan &sp, int dim, int n, long N, float tau_scale2, float wcoef,
                      const float *src, double *partial, cudaStream_t st);

// ---- displacement-major pair kernel (k_pairs_disp.cu): 2D, FP32, S = 64.
// partial must hold [grid][N] doubles.
struct DispPlan {
  int usable = 0;
  long n_units = 0, lat_elems = 0;
  int ldp = 0, grid = 0, n = 0;
  size_t smem = 0;
  float *src_t = nullptr;     // s transposed (FP32 [N])
  float *ss32 = nullptr;      // sigma_s in FP32 (for the expansion into K)
  void *yacc = nullptr;       // int64 [2 N]: fixed-point sums (x fastest, then y fastest), zero between applies
  void *geometry = nullptr;   // shared stencils and units of this n (owned by a cache)
  void *units = nullptr;
  void *stencil = nullptr;    // per-displacement chunk records (float4)
  size_t stencil_bytes = 0;
  int *counter = nullptr;
  void *lattice = nullptr;
  void *lattice_t = nullptr;  // lattice with y fastest (global-lattice kernels only)
  int global = 0;             // lattice read from global memory (grids past shared memory, n <= 258)
  unsigned *smax = nullptr;   // max |s| of the current apply (float bits)
  double *scale = nullptr;    // fixed-point scale of the current apply
  double rbound = 0.0;        // bound on every row sum of A
  double taps = 0.0;          // multiply-adds of the tau sums per apply: sum_D |W_D| pairs(D)
  const void *kernel = nullptr;
  // displacement-major assembled operator: every unordered pair's FP32 weight
  const void *kernel_store = nullptr, *kernel_stream = nullptr;
  size_t smem_store = 0, smem_stream = 0;
  int grid_store = 0, grid_stream = 0;
  long long stored = 0;       // weights stored: N (N - 1) / 2
  const long long *doff = nullptr;
  const float *wtab = nullptr;  // M-ii: per-D weight (h / 2 pi) x cell integral; null for M-iii
};
// 3D displacement-major kernel (k_pairs_disp3.cu), grids up to 32^3
struct DispPlan3 {
  int usable = 0, n = 0, grid = 0;
  size_t smem = 0;
  long n_units = 0, lat_elems = 0;
  double taps = 0.0, rbound = 0.0;
  void *geometry = nullptr;   // shared stencils and units of this n (owned by a cache)
  void *units = nullptr, *stencil = nullptr, *lattice = nullptr;
  int *counter = nullptr;
  unsigned *smax = nullptr;
  double *scale = nullptr;
  float *src_t = nullptr;
  unsigned long long *yacc = nullptr;
  const void *kernel = nullptr;
  // dense assembly from the stored pair weights (built on first use)
  const void *kernel_store = nullptr;
  int grid_store = 0, nq = 0;
  long items = 0;              // expansion items: (line displacement, target line) pairs
  long stored = 0;             // unordered pairs N (N - 1) / 2
  long long *doff = nullptr;   // per D of the half space: its first stored weight
  int *ioff = nullptr, *iqd = nullptr;  // expansion items per line displacement
};
size_t disp3_smem_bytes(int n);
vie_status disp3_prepare(DispPlan3 *dp, int n, const float *sig_padded, int device, cudaStream_t st);
void disp3_release(DispPlan3 *dp);
vie_status disp3_apply(const DispPlan3 &dp, int op, const double *sigma_s, const double *g, const double *diag,
                       float *src, float tau_scale2, float wcoef, double *y, cudaEvent_t mid0, cudaEvent_t mid1,
                       cudaStream_t st);
// K (row-major N x ldk, FP32 k32 or BF16 khi + klo) from the 3D displacement
// kernel's march: every unordered pair's weight stored once, then expanded;
// ldk = 0: A in the symmetric blocks of grid-line pairs instead (into k32)
vie_status disp3_assemble(DispPlan3 *dp, float tau_scale2, float wcoef, const double *sigma_s, const double *diag,
                          long ldk, float *k32, void *khi, void *klo, int device, cudaStream_t st);
// floats of the 3D symmetric blocks and of their row/column-sum partials
vie_status disp3_sym_sizes(DispPlan3 *dp, int device, long *block_floats, long *partial_floats);
// y = op(A s) from the 3D symmetric blocks (s: FP32 scratch of N floats)
vie_status symv3_apply(const DispPlan3 &dp, int op, const double *sigma_s, const double *g, const float *blocks,
                       float *s, float *partial, double *y, int device, cudaStream_t st);

size_t disp_smem_bytes(int n, int R);  // shared lattice bytes at stack depth R
bool disp_expand_fits(int n, int device);  // k_expand_pairs has room for the grid (n <= 169)
vie_status disp_source(const DispPlan &dp, long N, int op, const double *sigma_s, const double *g,
                       float *src, cudaStream_t st);
vie_status disp_reduce(const DispPlan &dp, long N, int op, const double *diag, const double *sigma_s,
                       const double *g, double *y, cudaStream_t st);
vie_status disp_prepare(DispPlan *dp, int n, const float *sig_padded, int device, cudaStream_t st);
// M-ii (Remark REM: NEW KERNEL): the per-D weight table of the plan and the
// diagonal value A_jj (the same for every cell); widens rbound to its row sums
vie_status disp_mii_prepare(DispPlan *dp, int n, double *diag_value, cudaStream_t st);
void disp_release(DispPlan *dp);
vie_status disp_launch(const DispPlan &dp, int n, float tau_scale2, float wcoef, const float *src,
                       cudaStream_t st);
vie_status disp_store(const DispPlan &dp, int n, float tau_scale2, float wcoef, float *wbuf, cudaStream_t st);
int symv_max_n();  // largest grid the symmetric-block product takes (160)
size_t symv_block_floats(int n);
size_t symv_partial_floats(int n);
vie_status symv_apply(int n, int op, const double *sigma_s, const double *g, const float *blocks, float *s,
                      float *partial, double *y, int device, cudaStream_t st);
vie_status disp_expand(const DispPlan &dp, int n, const float *wbuf, const double *sigma_s, const double *diag,
                       long ldk, float *k32, void *khi, void *klo, int device, cudaStream_t st);
vie_status disp_stream(const DispPlan &dp, int n, const float *wbuf, const float *src, cudaStream_t st);

// integral of 1/|z| over the unit square centred at (t1, t2), FP64 (the
// closed form of Remark REM: NEW KERNEL; k_pairs_disp.cu)
double unit_cell_integral(double t1, double t2);

// ---- FFT preconditioner (k_fftpre.cu): Section 4.4, Eqs. EQ: FFT, EQ:SOL FFT
struct FftPre {
  int on = 0, n = 0, m = 0, logm = 0;  // m: torus side, the power of two >= 2 n
  double mu = 0.0, mu_s = 0.0;         // mean sigma_t and sigma_s
  float *inv_lambda = nullptr;         // [m][m] 1 / (1 - mu_s F(W~)), FP32
  float2 *tw = nullptr;                // [m / 2] e^{-2 pi i k / m}
  float2 *buf = nullptr;               // [n][m] complex work lines
};
vie_status fft_prepare(FftPre *fp, int n, double mu, double mu_s, int mii, cudaStream_t st);
void fft_release(FftPre *fp);
// z = P F^{-1}(F(P^{-1} v) / lambda); v, z FP64 device [n * n]
vie_status fft_precondition(const FftPre &fp, const double *v, double *z, cudaStream_t st);

// ---- diffusion preconditioner (k_diffpre.cu): Section 4.4, Eq. EQ:DA
constexpr int kDiffMaxLevels = 16;
struct DiffLevel {
  int n = 0;
  double *c = nullptr;  // [6][n * n]: diagonal, the west, east, south, north couplings, 1 / diagonal
  double *f = nullptr;  // right-hand side of this level
  double *u = nullptr;  // its V-cycle iterate (level 0: the correction D^{-1}(sigma_s r))
};
struct DiffPre {
  int on = 0, n = 0, L = 0, graph_kernels = 0;
  const double *ss = nullptr;  // sigma_s on the device (the handle's)
  DiffLevel lv[kDiffMaxLevels];
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};
// sigma_t, sigma_s: host FP64 [n * n] (sigma_t > 0); sigma_s_dev stays the caller's
vie_status diffusion_prepare(DiffPre *dp, int n, const double *sigma_t, const double *sigma_s,
                             const double *sigma_s_dev, cudaStream_t st);
void diffusion_release(DiffPre *dp);
// z = v + D^{-1}(sigma_s v) by one V-cycle; v, z FP64 device [n * n]
vie_status diffusion_precondition(const DiffPre &dp, const double *v, double *z, cudaStream_t st);

// ---- interpolation-based FMM operator (k_fmm.cu): Section 3.3, 2D
struct FmmPlan {
  int on = 0, n = 0, p = 0, L = 0, b = 0;
  long node_off[32] = {};      // per level: first node value of W and Lc
  long m2l_off[32] = {};       // per level: first float of its M2L blocks
  long near_floats = 0, m2l_floats = 0;
  float *near = nullptr;       // [leaf][9][b^2][b^2] (source-major) near blocks
  float *m2l = nullptr;        // per level [box][27][p^2][p^2] (source-major)
  float *W = nullptr, *Lc = nullptr;  // multipole and local node values, per level
  float *Pm = nullptr;         // [p^2][b^2] leaf interpolation
  float *Cq = nullptr;         // [4][p^2][p^2] child-to-parent interpolation
  float *z = nullptr;          // [p] Chebyshev points
};
void fmm_leaf_levels(int n, int *L, int *b);
vie_status fmm_prepare(FmmPlan *fp, int n, int p, const float *sig32, const double *diag, int steps, int closed,
                       double sigma_c, cudaStream_t st);
void fmm_release(FmmPlan *fp);
// y = A s (op A_RAW, K_SIGMA_S: s already multiplied by sigma_s) or g - A s (I_MINUS_K)
vie_status fmm_apply(const FmmPlan &fp, int op, const float *s, const double *g, double *y, cudaStream_t st);

// ---- R GMRES solves in lockstep (k_krylov.cu).  Per right-hand side r:
// basis vector i at V + r ldv_r + i N, Hessenberg H + r (m + 1) m
// (column-major), rotations cs/sn + r m, residual vector gv + r (m + 1), the
// triangular solution yv + r m, the dot columns hcol/htmp + r (m + 1), dot
// partials part + r blocks (m + 1), block ticket ticket[r] (0 between
// launches), scalars scal + 8 r (slot 2: ||w||^2, 3: the Givens residual
// estimate), bnorm[r] = ||phi_r||, act[r] != 0 while r takes part.
struct KBatch {
  double *H, *cs, *sn, *gv, *yv, *hcol, *htmp, *part, *scal, *bnorm;
  int *ticket, *act;
  long N;
  int m, R, blocks;
};
vie_status launch_bdots(const KBatch &b, const double *V, long ldv_r, int nv, const double *w, long ldw_r,
                        double *out1, double *out2, cudaStream_t st);
vie_status launch_bnorm2_givens(const KBatch &b, const double *w, long ldw_r, int k, cudaStream_t st);
vie_status launch_bnorm2(const KBatch &b, const double *w, long ldw_r, int slot, cudaStream_t st);
vie_status launch_borth_update(const KBatch &b, const double *V, long ldv_r, int nv, const double *h, double *w,
                               long ldw_r, cudaStream_t st);
vie_status launch_bscale(const KBatch &b, const double *x, long ldx_r, int slot, int use_sqrt, double *y,
                         long ldy_r, cudaStream_t st);
vie_status launch_baxpby(const KBatch &b, double a, const double *x, long ldx_r, double c, const double *y,
                         long ldy_r, double *z, long ldz_r, cudaStream_t st);
vie_status launch_bupdate(const KBatch &b, const double *B, long ldb_r, const int *kk, double *x, long ldx_r,
                          cudaStream_t st);

// ---- assembled operator (k_assemble.cu, k_gemm_tc.cu)
long assembled_ldk(long N);
vie_status launch_assemble(const SymPlan &sp, int dim, int n, long N, const double *sigma_s,
                           const double *diag, float *k32, void *khi, void *klo, int device,
                           cudaStream_t st);
vie_status launch_gemv(const void *k, const void *klo, int bf16, long ldk, long N, const double *g,
                       float *g32, int op, double *y, cudaStream_t st);
vie_status launch_divide(long N, const double *a, const double *b, double *out, cudaStream_t st);
vie_status launch_divide_cols(long N, int R, const double *a, long lda, const double *b, double *out, long ldo,
                              cudaStream_t st);
size_t gemm_workspace_bytes(long N, long ldk, int nrhs, int *splits_out, int sms);
// A BF16 TMA descriptor: rank dims innermost first, byte strides of dims
// 1..rank-1, box, 64- or 128-byte swizzle, zero fill outside the tensor.
vie_status encode_bf16_map(CUtensorMap *m, int rank, const void *base, const unsigned long long *dims,
                           const unsigned long long *strides, const unsigned *box, int swizzle_bytes);
// Y = K G (op K_SIGMA_S) or G - K G (I_MINUS_K) for nrhs <= kGemmMaxRhs
// columns, column r of G at g + r ldg and of Y at y + r ldy (FP64), on the
// tensor cores.
constexpr int kGemmMaxRhs = 128;
vie_status launch_gemm_bf16x3(const void *khi, const void *klo, long ldk, long N, const double *g, long ldg,
                              int nrhs, int op, double *y, long ldy, void *workspace, int *err,
                              cudaStream_t st);

// ---- learned preconditioner (k_unet.cu)
struct UnetImpl;
UnetImpl *unet_impl(vie_unet *u);
int unet_levels(vie_unet *u);
// the network's device error word (set by a tensor-core convolution whose
// bounded wait gave up), and its synchronous check-and-clear
int *unet_error_word(UnetImpl *u);
vie_status unet_take_error(UnetImpl *u, cudaStream_t st);
// z = base + rms(v) Net(...) with base = v when null (one vector, or R at a time)
vie_status unet_precondition_batch(UnetImpl *u, const double *sigma_t, const double *sigma_s, double inv_ref,
                                   const double *v, long ldv, const double *scal, int slot, int R, int n,
                                   float *xbuf, const double *base, long ldb, double *z, long ldz, cudaStream_t st);
vie_status unet_precondition(UnetImpl *u, const double *sigma_t, const double *sigma_s, double inv_ref,
                             const double *v, const double *vnorm2, int n, float *xbuf, const double *base,
                             double *z, cudaStream_t st);

// ---- Krylov kernels (k_krylov.cu)
int dot_blocks(long N);
vie_status launch_dots(const double *V, int nv, long ldv, const double *w, long N, double *part,
                       int blocks, cudaStream_t st);
vie_status launch_dots_finish(const double *part, int blocks, int nv, double *out, int accumulate,
                              cudaStream_t st);
vie_status launch_orth_update(const double *V, int nv, long ldv, const double *h, double *w,
                              long N, cudaStream_t st);
vie_status launch_dots_last(const double *V, int nv, long ldv, const double *w, long N, double *part,
                            int blocks, int *ticket, double *out1, double *out2, cudaStream_t st);
vie_status launch_norm2_givens(const double *w, long N, double *part, int blocks, int *ticket, double *norm2,
                               double *H, int m, int k, const double *hcol, double *cs, double *sn, double *gv,
                               double bnorm, double *est, cudaStream_t st);
vie_status launch_scale(const double *x, const double *norm2, int use_sqrt, double *y, long N,
                        cudaStream_t st);
vie_status launch_axpby(double a, const double *x, double b, const double *y, double *z, long N,
                        cudaStream_t st);
vie_status launch_givens(double *H, int m, int k, const double *hcol, const double *hk1sq,
                         double *cs, double *sn, double *gv, double bnorm, double *est,
                         cudaStream_t st);
vie_status launch_backsolve(const double *H, int m, int k, const double *gv, double *y,
                            cudaStream_t st);
vie_status launch_lincomb_add(const double *V, int nv, long ldv, const double *y, double *x,
                              long N, cudaStream_t st);

// ---- sweep kernels (k_sweep.cu)
vie_status launch_make_q(int dim, int n, const double *sigma_s, const double *U, const double *f,
                         float *qpad, cudaStream_t st);
vie_status launch_sweep(int dim, int n, const float *sigpad, const float *qpad, const float *dirs,
                        int M, float *Phi, cudaStream_t st);

}  // namespace vie
