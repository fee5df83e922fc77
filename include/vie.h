/*
 * vie.h -- C ABI of the GB300 (sm_103a) volume-integral-equation library.
 *
 * The library implements the hot path of the two-step method of Ren, Zhang
 * & Zhong for the radiative transfer equation in isotropic media
 * (arXiv 1610.00835):
 *
 *   * the operator of Section 2, Eqs. EQ:Operator K and EQ:Kernel,
 *       (K g)(x) = int K(x,y) g(y) dy,
 *       K(x,y)   = sigma_s(y) exp(-tau(x,y)) / (|S^{d-1}| |x-y|^{d-1}),
 *     with tau(x,y) the line integral of sigma_t along the segment x -> y,
 *     discretised by piecewise-constant collocation on a uniform grid
 *     (Section 3.1) with approach M-iii of Section 3.2 (off-diagonal entries
 *     |T_k| K(x_j, x_k), the self cell integrated explicitly);
 *   * GMRES for (I - K) U = phi, phi = K(sigma_s^{-1} f) (Eq. EQ:ERT Intgrl
 *     FMM; Algorithm 1, S.2);
 *   * the scattering-free sweep that recovers Phi(x, v) from U
 *     (Algorithm 1, S.3; Eq. EQ:ERT Intgrl).
 *
 * Conventions shared by every entry point:
 *   - Domain (0,1)^d, d = 2 or 3, n cells per side, h = 1/n, N = n^d cells,
 *     cell centres x_j = (i + 1/2) h, linear index j = ix + n*iy (+ n^2*iz),
 *     x fastest (Section 3.1, uniform grid).
 *   - sigma_t is interpolated between cell centres bilinearly (2D) or
 *     trilinearly (3D), clamped to the hull of the centres.
 *   - tau is the S-step midpoint march
 *       tau = (r/S) sum_{i=0}^{S-1} sigma_t~(x + (i+1/2)/S (y - x)),
 *     or sigma_t r for homogeneous media (Eq. EQ:Kernel Cons).
 *   - A_jk = h^d exp(-tau_jk) / (|S^{d-1}| r_jk^{d-1}) for j != k and the
 *     self-cell integral d_j = int_{T_j} e^{-sigma_t,j |z|} / (|S^{d-1}|
 *     |z|^{d-1}) dz for j == k; K_jk = A_jk sigma_s,k.  |S^1| = 2 pi,
 *     |S^2| = 4 pi.  With VIE_DISC_MII (2D): approach M-ii of Section 3.2
 *     with the kernel of Remark REM: NEW KERNEL instead,
 *     A_jk = exp(-tau_jk) / (2 pi) int_{T_k} |x_j - z|^{-1} dz for every j
 *     and k (tau_jj = 0), the cell integral in closed form.
 *   - Every call returns a vie_status; on failure vie_last_error() gives a
 *     message (thread-local).  No C++ exception crosses this boundary.
 *   - Vectors (g, y, f, U, Phi) may be host or device pointers; the library
 *     detects which.  Device pointers stay owned by the caller and work is
 *     queued on the caller's stream (asynchronous unless stated).  Host
 *     pointers are copied through library-owned device buffers and the call
 *     returns after the copy back (synchronous).
 *   - The handle owns all device memory it allocates; vie_destroy frees it.
 *     A handle is not thread-safe: one call at a time per handle.
 */
#ifndef VIE_H
#define VIE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VIE_OK = 0,
  VIE_ERR_INVALID_ARG = 1,  /* bad size, pointer, option or coefficient   */
  VIE_ERR_CUDA = 2,         /* a CUDA runtime call failed                 */
  VIE_ERR_OOM = 3,          /* device allocation failed                   */
  VIE_ERR_NOT_CONVERGED = 4,/* GMRES hit maxit; U and the report are valid */
  VIE_ERR_TIMEOUT = 5,      /* a device-side bounded wait gave up         */
  VIE_ERR_NONFINITE = 6,    /* NaN or Inf in an input or a residual       */
  VIE_ERR_UNSUPPORTED = 7   /* option combination not built               */
} vie_status;

/* Uniform grid on the unit square (dim 2) or cube (dim 3), n cells per side.
 * Section 3.1 (uniform grid, centroid collocation points). */
typedef struct {
  int dim; /* 2 or 3                       */
  int n;   /* cells per side, 1 <= n <= 4096 (2D), 1 <= n <= 256 (3D) */
} vie_grid;

enum { VIE_TAU_MARCH = 0, VIE_TAU_CLOSED = 1 };
enum { VIE_PREC_FP32 = 0, VIE_PREC_FP64 = 1 };
/* Discretisation of Section 3.2: M-iii (collocation, the default), or M-ii
 * (the cell integral of |x_j - z|^{1-d} exact, Remark REM: NEW KERNEL; error
 * O(h^2 (1 + log h)) against O(h), Eq. EQ: ERROR).  M-ii is built for 2D
 * grids with FP32 tiles, the S = 64 march and the displacement kernel
 * (n <= 258); other combinations return VIE_ERR_UNSUPPORTED at create. */
enum { VIE_DISC_MIII = 0, VIE_DISC_MII = 1 };

typedef struct {
  int steps;     /* S, midpoint-march steps for tau (>= 1; 64 by default)   */
  int tau_mode;  /* VIE_TAU_MARCH, or VIE_TAU_CLOSED (needs constant sigma_t) */
  int precision; /* VIE_PREC_FP32: FP32 kernel tiles, FP64 sums across tiles;
                    VIE_PREC_FP64: every pair in FP64                        */
  int device;    /* CUDA device ordinal                                     */
  int kernel;    /* pair kernel for FP32 tiles: VIE_KERNEL_AUTO picks the
                    fastest that applies; the others force one (a forced
                    kernel that does not apply falls back to AUTO)         */
  int disc;      /* VIE_DISC_MIII (default) or VIE_DISC_MII                  */
} vie_opts;

enum {
  VIE_KERNEL_AUTO = 0,
  VIE_KERNEL_SYMMETRIC = 1,     /* tile pairs, each unordered pair once       */
  VIE_KERNEL_DISPLACEMENT = 2,  /* 2D, S = 64: warps share one displacement   */
  VIE_KERNEL_GENERAL = 3        /* every ordered pair; any S                  */
};

/* Default options: S = 64, march, FP32 tiles, device 0, automatic kernel,
 * M-iii. */
void vie_default_opts(vie_opts *o);

typedef struct vie_handle vie_handle;

/* Create an operator for one medium (Section 3.1-3.2).
 *   g        : grid.
 *   sigma_t  : host FP64 [N], total attenuation mu at the cell centres, >= 0.
 *   sigma_s  : host FP64 [N], scattering coefficient mu_s, >= 0.
 *   o        : options (NULL: defaults).
 * Both arrays are copied; the caller keeps ownership.  The self-cell
 * diagonal d_j is computed on the device here (FP64 Gauss-Legendre).
 * Errors: INVALID_ARG (sizes, negative coefficient, non-constant sigma_t
 * with VIE_TAU_CLOSED, unknown disc), UNSUPPORTED (VIE_DISC_MII outside its
 * combination), NONFINITE, OOM, CUDA. */
vie_status vie_create(vie_handle **out, const vie_grid *g, const double *sigma_t,
                      const double *sigma_s, const vie_opts *o);

/* Free every device buffer of the handle (after synchronising its device).
 * NULL is accepted. */
vie_status vie_destroy(vie_handle *h);

typedef enum {
  VIE_OP_K_SIGMA_S = 0, /* y = K g,        K_jk = A_jk sigma_s,k           */
  VIE_OP_I_MINUS_K = 1, /* y = g - K g     (Eq. EQ: LINEAR SYSTEM)          */
  VIE_OP_A_RAW = 2      /* y = A g         (phi = A f, Eq. EQ:ERT Intgrl FMM) */
} vie_op;

/* Apply the discrete operator (Section 3.2, Eq. EQ: DISCRETIZED; Section 3.3:
 * "the main computational cost ... the evaluations of K U").
 *   g, y   : FP64 [nrhs][N] (RHS r at offset r*N), host or device; g and y
 *            must not overlap.
 *   nrhs   : >= 1.
 *   stream : cudaStream_t (NULL: legacy default stream).
 * With host pointers the call reports VIE_ERR_TIMEOUT if a tensor-core
 * product gave up on a bounded wait (see vie_check_device for device pointers).
 * Errors: INVALID_ARG, CUDA, TIMEOUT. */
vie_status vie_apply(vie_handle *h, vie_op op, const double *g, double *y, int nrhs,
                     void *stream);

/* Operator storage modes for vie_assemble. */
enum {
  VIE_OPERATOR_OTF = 0,          /* entries generated on the fly (default)        */
  VIE_OPERATOR_FP32 = 1,         /* K assembled in HBM, FP32                      */
  VIE_OPERATOR_BF16X3 = 2,       /* K assembled as BF16 hi + lo; products with
                                    several right-hand sides on the tensor cores,
                                    G split exactly into BF16 hi + mid + lo, the
                                    five products above 2^-24 kept, FP32
                                    accumulate (split-precision correction)     */
  VIE_OPERATOR_PAIRS32 = 3,      /* A_jk of every unordered pair once, FP32,
                                    displacement-major (2D handles that use the
                                    displacement kernel): applies stream it */
  VIE_OPERATOR_SYM32 = 4,        /* A (symmetric) in FP32 blocks, one per pair of
                                    grid rows yj <= yk (2D) or grid lines (3D):
                                    applies read each block once, y = A (sigma_s g) */
  VIE_OPERATOR_FMM = 5           /* the interpolation-based FMM of Section 3.3
                                    with cached near-field and M2L blocks
                                    (vie_assemble_fmm; Chebyshev order 6 here) */
};

/* VIE_OPERATOR_SYM32: A_jk = A_kj (Section 2, Eq. EQ:Kernel; M-iii of
 * Section 3.2) with the self cell d_j on the diagonal, FP32, stored once per
 * unordered pair of grid rows: for yj <= yk the n x n block of targets on row yj
 * and sources on row yk (n (n + 1) / 2 blocks, 541 MB at 128^2).  An apply forms
 * s = sigma_s g (or g for VIE_OP_A_RAW) in FP32, takes from every block its row
 * sums (for row yj) and column sums (for row yk) in FP32, and adds each
 * target's n block sums in a fixed order in FP64: deterministic, half the bytes
 * of the dense K per apply.  Same handles as VIE_OPERATOR_PAIRS32 (2D, n <= 160).
 * 3D handles on the 3D displacement kernel (n <= 32): one n x n block per
 * unordered pair of grid lines (y, z), targets on the first line (x the row)
 * and sources on the second (x the column), 2.16 GB at 32^3; each target adds
 * its ~n^2 row or column sums as an FP32 hi + lo pair (error-free additions) in a
 * fixed order. */

/* VIE_OPERATOR_PAIRS32: the weights A_jk = A_kj (Section 2, Eq. EQ:Kernel with
 * the M-iii collocation of Section 3.2) of the N (N - 1) / 2 unordered pairs,
 * each stored once in FP32 (537 MB at 128^2), grouped by displacement D = k - j:
 * for each D of the half plane (dy > 0, or dy = 0 and dx > 0) the rectangle of
 * targets j with j + D in the grid.  Every apply (any vie_op, nrhs applies for
 * nrhs right-hand sides) reads them once and accumulates exactly as the
 * on-the-fly displacement kernel does, so its results are bitwise equal to
 * the on-the-fly applies of the same handle.  Only for handles whose
 * vie_get_kernel is VIE_KERNEL_DISPLACEMENT (else VIE_ERR_UNSUPPORTED).
 *
 * Assemble K = [K_jk omega_k] (Section 3.2, Eq. EQ: LINEAR SYSTEM) into device
 * memory and use it for later VIE_OP_K_SIGMA_S / VIE_OP_I_MINUS_K applies and
 * solves; the paper caches its kernel evaluations for reuse across GMRES
 * iterations in the same way (Section 4.2).  Entries are the on-the-fly FP32
 * values (S = 64 march, self cell on the diagonal); storage is N x LDK with
 * LDK = N rounded up to 64, 4 bytes per entry in both modes (1.07 GB at
 * 128^2, 17.2 GB at 256^2).  VIE_OP_A_RAW uses phi = K (sigma_s^{-1} f)
 * (Eq. EQ:ERT Intgrl FMM) when sigma_s > 0 everywhere, else the on-the-fly
 * path.  One RHS
 * uses a bandwidth-bound CUDA-core product; vie_apply with nrhs >= 2 in
 * VIE_OPERATOR_BF16X3 mode uses one tensor-core product per 128 RHS.
 * VIE_OPERATOR_OTF frees the matrix.  Needs FP32 precision, the march and
 * S = 64 (else VIE_ERR_UNSUPPORTED).  Asynchronous on `stream`.
 * Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA. */
vie_status vie_assemble(vie_handle *h, int mode, void *stream);

/* VIE_OPERATOR_FMM with Chebyshev order `order` per axis (2..12; the paper
 * uses 4, 6 and 9).  Section 3.3, Eqs. EQ: CHEB, EQ:Kernel Approx, EQ:
 * SUMMATION, EQ: M2L, EQ: L2L (Fong-Darve), 2D: the grid as a quadtree with
 * leaves of b x b cells, n = 2^L b, b >= 8 and L >= 2 (L as large as the
 * factors of two allow); the near field (a leaf and its 3 x 3 neighbourhood)
 * from the M-iii entries A_jk (self cell on the diagonal), the far field from
 * the kernel h^2 e^{-tau} / (2 pi r) at the order^2 first-kind Chebyshev
 * nodes of each box: P2M, M2M, M2L over the 27-box interaction lists from
 * level 2 down, L2L, L2P.  Every near entry and every M2L kernel value is
 * computed once here on the device (FP32, the handle's tau: the S-step march
 * with sample points clamped to the hull of the cell centres, or the closed
 * form) and stored: 4 b^4 9 4^L + 4 * 27 order^4 sum_{l=2..L} 4^l bytes
 * (0.09 GB at 128^2, 1.4 GB at 512^2 with order 6).  Applies (any vie_op; phi
 * = A f directly) are 2 L launches that read the cached blocks once.
 * The far field is an approximation: relative error ~1e-6 (order 6) on
 * homogeneous media, 1e-5 .. 1e-4 on heterogeneous ones (tau of a bilinear
 * sigma_t is only piecewise smooth).  Needs a 2D grid, FP32 tiles and M-iii.
 * Errors: INVALID_ARG (order), UNSUPPORTED (grid without a far field, 3D,
 * FP64, M-ii), OOM, CUDA. */
vie_status vie_assemble_fmm(vie_handle *h, int order, void *stream);

typedef struct {
  double rtol;  /* stop when ||phi - (I-K)U||_2 / ||phi||_2 <= rtol (FP64)   */
  int restart;  /* m, Krylov dimension per cycle (1..256; 64 by default)    */
  int maxit;    /* total Arnoldi steps allowed (default 1000)               */
  int zero_x0;  /* 1: ignore U on entry and start from U = 0               */
  int rhs_is_phi; /* 1: f already holds phi; 0: phi = A f is formed here     */
  int time_apply; /* 1: record CUDA events around every operator apply      */
  int nrhs;       /* sources solved together on this medium (1..4096; 1 by
                     default); f and U are then [nrhs][N] and rep an array of
                     nrhs reports (see vie_solve_gmres)                      */
} vie_gmres_opts;

void vie_default_gmres_opts(vie_gmres_opts *o);

typedef struct {
  int iters;           /* Arnoldi steps taken                                 */
  int restarts;        /* completed restart cycles                            */
  int converged;       /* 1 if relres <= rtol                                 */
  int n_apply;         /* operator applications (including phi and residuals) */
  double relres;       /* final true relative residual, FP64                  */
  double relres_est;   /* last Givens residual estimate                       */
  double t_total_ms;   /* host wall time of the call                          */
  double t_apply_ms;   /* summed CUDA-event time of the applies (time_apply)  */
  double t_apply_kernel_ms; /* of that, the pair kernel alone (time_apply)     */
  int precond_iters;   /* Arnoldi steps taken with the learned preconditioner  */
  int fell_back;       /* 1 if the preconditioned iteration stalled and plain
                          GMRES finished the solve                            */
} vie_report;

/* Solve (I - K) U = phi by restarted GMRES(m) in FP64 (Algorithm 1, S.2;
 * Section 5: GMRES).  Arnoldi with classical Gram-Schmidt applied twice,
 * Givens rotations and the triangular solve run on the device in FP64; the
 * operator is applied with the handle's precision; convergence is judged
 * on the FP64 true residual.
 *   f      : FP64 [nrhs][N] sources f (or phi if rhs_is_phi), host or device.
 *   U      : FP64 [nrhs][N] initial guesses on entry (unless zero_x0),
 *            solutions on exit.
 *   rep    : NULL, or nrhs reports (one per source).
 * With nrhs > 1 the nrhs solves run in lockstep: every Arnoldi step applies
 * the operator to the nrhs current directions at once -- with
 * VIE_OPERATOR_BF16X3 as one tensor-core product, up to 128 columns per
 * product -- and a learned preconditioner runs one forward pass over all of
 * them; CGS2, the Givens steps and the updates of all solves are one launch
 * each.  Each solve keeps its own restart cycles, residual estimate, stall
 * fallback and FP64 true residual, and leaves the lockstep when it
 * converges (its report counts its own steps).
 * The call synchronises the stream once per Arnoldi step (residual test; one
 * copy of all nrhs estimates).  Returns NOT_CONVERGED (U and rep valid) when
 * maxit is reached (for any source). */
vie_status vie_solve_gmres(vie_handle *h, const double *f, double *U,
                           const vie_gmres_opts *o, vie_report *rep, void *stream);

/* Step two (Algorithm 1, S.3): Q = sigma_s U + f, then for every direction
 * v_m and cell x_j the backward characteristic of Eq. EQ:ERT Intgrl,
 *   Phi(x_j, v_m) = int_0^L exp(-int_0^l sigma_t(x_j - l' v_m) dl') Q(x_j - l v_m) dl,
 * L the distance to the boundary along -v_m.  The ray is cut into
 * ceil(2 n L - 1e-6) equal steps (each <= h/2, decided in FP64); on each
 * step sigma_t and Q (interpolated like sigma_t) are frozen at the step
 * midpoint and the step is integrated exactly.
 *   U, f : FP64 [N], host or device.
 *   dirs : FP32 [M][dim] unit vectors, host or device.
 *   Phi  : FP32 [M][N], host or device.
 * Errors: INVALID_ARG, CUDA. */
vie_status ert_sweep(vie_handle *h, const double *U, const double *f, const float *dirs,
                     int M, float *Phi, void *stream);

/* One operator apply that allocates no device memory, for callers that cannot
 * call cudaMalloc (a host that owns all device memory through its own pool or
 * fixed budget, or a latency-critical loop that cannot take an allocation's
 * implicit synchronisation).  The paper has no counterpart: this is a
 * deployment variant of vie_apply.
 *   dim, n           : grid as in vie_grid; n^dim <= 16384 (2D n <= 128,
 *                      3D n <= 25), else VIE_ERR_INVALID_ARG.
 *   sigma_t, sigma_s : device FP64 [N] coefficients (caller-owned).
 *   op, g, y         : as vie_apply with nrhs = 1; g and y device FP64 [N].
 * Computes what vie_apply computes for a handle made with the default options
 * (S = 64 march, FP32 tiles), self-cell diagonal included, with every
 * intermediate in one fixed device array of about 17 MB that the library
 * image holds on every GPU that loads it until the process exits.  The first
 * call with a device current looks up that array's address on the device
 * and copies the self-cell quadrature rule there (synchronously); make it
 * before any stream capture.  Calls share the array and it keeps the last
 * call's contents (the work counter is cleared on every call); calls whose
 * work overlaps on the same GPU race, so serialise them.  Asynchronous on
 * `stream`.  Errors: INVALID_ARG (sizes, non-device pointers), UNSUPPORTED
 * (the device's shared memory cannot hold the grid's lattice for the
 * symmetric kernel; nothing is launched), CUDA. */
vie_status vie_apply_noalloc(int dim, int n, const double *sigma_t, const double *sigma_s,
                             vie_op op, const double *g, double *y, void *stream);

/* ---- Batches of media (many uneven 2D grids in one launch). */
typedef struct vie_batch vie_batch;

/* Create a batch of `count` 2D media (grids[i].dim == 2), each with its own
 * n and host FP64 coefficients sigma_t[i], sigma_s[i] (copied).  Options must
 * be FP32 tiles with the S = 64 march and M-iii.  o->kernel selects how the
 * grids run: VIE_KERNEL_SYMMETRIC puts every grid's tile pairs into one
 * persistent launch; VIE_KERNEL_AUTO (and DISPLACEMENT) give each grid that
 * the displacement kernel takes (2 <= n <= 258) a launch of that kernel and
 * put only the others into the persistent launch; all of them are replayed
 * from one CUDA graph.  Vectors of the batch are packed: medium i occupies
 * cells [offsets[i], offsets[i+1]) (vie_batch_layout).
 * Errors: INVALID_ARG, NONFINITE, OOM, CUDA. */
vie_status vie_batch_create(vie_batch **out, int count, const vie_grid *grids,
                            const double *const *sigma_t, const double *const *sigma_s,
                            const vie_opts *o);
vie_status vie_batch_destroy(vie_batch *b);

/* Total cells and the count + 1 packed offsets of the media. */
vie_status vie_batch_layout(vie_batch *b, long long *total_cells, long long *offsets);

/* Apply the operator of every medium (as vie_apply) to nrhs packed FP64
 * vectors g, writing the packed y: layout [nrhs][total_cells], source r of
 * medium i at r * total_cells + offsets[i].  Each source is one pass of the
 * launches vie_batch_create chose (the displacement kernel per grid, one
 * persistent kernel over the remaining media's tile pairs with dynamic
 * scheduling across media); all nrhs passes are replayed from one CUDA graph,
 * captured on the first call for a given (op, g, y, nrhs) and re-captured when
 * they change.  The pairs are marched again for every source: for many sources
 * on one medium, vie_assemble and vie_apply with nrhs amortise the march.
 * Host pointers are staged and the call then synchronises.
 *   nrhs : 1 <= nrhs <= 4096.
 * Errors: INVALID_ARG, CUDA, OOM. */
vie_status vie_batch_apply(vie_batch *b, vie_op op, const double *g, double *y, int nrhs, void *stream);

/* Time the launch configurations (CTA groups 8/4/2; shared-memory staging of
 * every lattice that fits, or only up to 128 KB) on this batch and keep the
 * fastest.  With cache_path, a line "<device>|<n_1>,...,<n_k>, <groups>
 * <policy>" is read from (a hit skips the timing) or appended to that file.
 * Errors: INVALID_ARG, CUDA. */
vie_status vie_batch_autotune(vie_batch *b, const char *cache_path, void *stream);

/* Current configuration: CTA groups and lattice staging policy. */
vie_status vie_batch_config(vie_batch *b, int *groups, int *smem_policy);

/* ---- Learned right preconditioner (no paper counterpart; it takes the place
 * of the paper's FFT and diffusion preconditioners, Section 4.4).
 * A U-Net with `levels` levels and `channels` channels maps the input
 * (sigma_t / s_ref, sigma_s / s_ref, b / rms(b)) on an n x n grid to o, and
 * the preconditioner is M(b) = b + rms(b) o: the network supplies the smooth
 * part of (I - K)^{-1} b.  Weights are FP32 (training) with a BF16 copy for
 * inference (tensor cores); accumulation is FP32.  Parameter layout: for every convolution
 * in the order encoder (level 0 first, two each), decoder (deepest first, two
 * each), head: weights [Co][Ci][k][k] then bias [Co]. */
typedef struct vie_unet vie_unet;
vie_status vie_unet_create(vie_unet **out, int levels, int channels, unsigned long long seed, int device);
vie_status vie_unet_destroy(vie_unet *u);
vie_status vie_unet_num_params(vie_unet *u, long long *n);
vie_status vie_unet_get_params(vie_unet *u, float *host_params);
vie_status vie_unet_set_params(vie_unet *u, const float *host_params);
/* o = Net(x): x device FP32 [B][3][n][n], o device FP32 [B][n][n]; n divisible
 * by 2^(levels-1).  use_bf16 = 0: FP32 weights and activations on the CUDA
 * cores, asynchronous.  use_bf16 = 1 (what the preconditioner uses): BF16
 * weights; with 16 or 32 channels every 3x3 convolution runs on the tensor
 * cores (tcgen05, an implicit GEMM whose shifted input tiles the TMA loads)
 * with its inputs rounded to BF16 and FP32 accumulation, other widths on the
 * CUDA cores with FP32 activations; the call synchronises the stream and
 * returns VIE_ERR_TIMEOUT if a convolution gave up on a bounded wait. */
vie_status vie_unet_forward(vie_unet *u, const float *x, float *o, int B, int n, int use_bf16, void *stream);
/* Diagnostics (no paper counterpart): copy the input and the output of
 * convolution `layer` (parameter order: encoder, decoder, head) as the most
 * recent vie_unet_forward computed them, FP32 [B][ci][H][H] and
 * [B][co][H][H] (H = n / 2^level), into `in` and `out` (host or device;
 * `in` may be NULL, and layer 0's input, the caller's x, is not copied).
 * Synchronous.  Errors: INVALID_ARG (no forward yet, layer out of range). */
vie_status vie_unet_layer_io(vie_unet *u, int layer, float *in, float *out, void *stream);

/* Mean squared error of Net(x) against t (device FP32 [B][n][n]) and, if
 * grads_host is not NULL, its gradient with respect to every parameter
 * (host FP32 [num_params]). Synchronous. */
vie_status vie_unet_loss_grad(vie_unet *u, const float *x, const float *t, int B, int n, float *grads_host,
                              double *loss, void *stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on the batch; returns the loss
 * mean_b w_b mean_p (o - t)^2, w_b = weights[b] (device FP32 [B]) or 1 if
 * weights is NULL. */
vie_status vie_unet_train_step(vie_unet *u, const float *x, const float *t, const float *weights, int B,
                               int n, float lr, double *loss, void *stream);
/* Checkpoint: the parameters and the Adam state (step count, first and
 * second moments), so that vie_unet_train_step resumes exactly where a saved
 * run stopped.  vie_unet_load also reads parameter-only files of the earlier
 * format (the optimizer state then starts from zero).  The file must match
 * the network's levels and channels, else INVALID_ARG. */
vie_status vie_unet_save(vie_unet *u, const char *path);
vie_status vie_unet_load(vie_unet *u, const char *path);
/* Adam steps taken so far (restored by vie_unet_load). */
vie_status vie_unet_train_state(vie_unet *u, long long *step);
/* Use `u` as the right preconditioner of vie_solve_gmres on this handle
 * (flexible GMRES); NULL restores plain GMRES.  2D handles only, n divisible
 * by 2^(levels-1); s_ref scales the coefficient channels (> 0).  If the
 * preconditioned residual stalls (two consecutive Arnoldi steps each
 * reducing it by less than 20 %) or the network output is not finite, the
 * solve continues with plain GMRES from the current iterate and reports
 * fell_back = 1.  The network must outlive its use by the handle. */
vie_status vie_set_preconditioner(vie_handle *h, vie_unet *u, double s_ref);

/* The learned network as a correction of the diffusion preconditioner (below):
 *   M(v) = D(v) + rms(v) Net(sigma_t / s_ref, sigma_s / s_ref, v / rms(v)),
 * D the diffusion preconditioner's z = v + D^{-1}(sigma_s v); the network is
 * trained on the part of (I - K)^{-1} v that D misses (train_unet.py --base
 * diffusion).  Builds the diffusion hierarchy (synchronous), replaces any other
 * preconditioner; NULL u removes both.  Same conditions and stall fallback as
 * vie_set_preconditioner and vie_set_diffusion_preconditioner.
 * Errors: INVALID_ARG, OOM, CUDA. */
vie_status vie_set_preconditioner_on_diffusion(vie_handle *h, vie_unet *u, double s_ref, void *stream);

/* The FFT preconditioner of Section 4.4 (Eqs. EQ: FFT and EQ:SOL FFT) as the
 * right preconditioner of vie_solve_gmres (flexible GMRES, with the same
 * stall fallback as above); enable = 0 removes it.  It replaces sigma_t and
 * sigma_s by their means over the grid, extends the resulting convolution
 * periodically to an m x m torus (m the power of two >= 2 n), extends the
 * vector by zero, and inverts the periodic operator by FFT:
 *   z = P F^{-1}( F(P^{-1} v) / F(delta - mean(sigma_s) W~) ),
 * W~ the homogeneous medium's A (of the handle's discretisation) as a
 * function of the displacement.  The symbol is computed once here on the
 * host in FP64 (synchronous); applies run three FP32 FFT launches on the
 * device.  It replaces any other preconditioner set on the handle (learned
 * or diffusion), and setting one of those replaces it.  2D handles, n <= 2048.
 * Errors: INVALID_ARG (3D; mean sigma_s >= mean sigma_t leaves the periodic
 * operator singular), UNSUPPORTED (n > 2048), OOM, CUDA. */
vie_status vie_set_fft_preconditioner(vie_handle *h, int enable, void *stream);

/* z = M v with the FFT preconditioner alone (v, z FP64 [N], host or device,
 * not overlapping).  Errors: INVALID_ARG (none set), CUDA. */
vie_status vie_fft_precondition(vie_handle *h, const double *v, double *z, void *stream);

/* The diffusion preconditioner of Section 4.4 (Eq. EQ:DA) as the right
 * preconditioner of vie_solve_gmres (flexible GMRES, same stall fallback);
 * enable = 0 removes it.  D is the second-order finite-volume form of
 *   -div(1/(d mu) grad U) + mu_a U,  U + (2/(d mu)) dU/dn = 0 on the boundary,
 * mu = sigma_t, mu_a = sigma_t - sigma_s per cell (harmonic-mean face
 * coefficients; the Robin condition eliminated at boundary faces), and the
 * preconditioner is the diffusion-synthetic form on U,
 *   z = v + D^{-1}(sigma_s v),
 * D^{-1} one geometric-multigrid V-cycle from zero (levels n, n/2, ... while
 * even and above 8; red-black Gauss-Seidel 2 + 2; mean restriction; bilinear
 * prolongation; 200 sweeps on the coarsest grid), FP64, replayed from a CUDA
 * graph.  It works where the diffusion approximation holds and the cells are
 * optically thin (sigma_t h well below 1); on thick cells the correction can
 * overshoot and the stall fallback takes over.  It replaces any other
 * preconditioner set on the handle.  2D handles; sigma_t > 0 in every cell.
 * Errors: INVALID_ARG (3D, sigma_t = 0 somewhere), OOM, CUDA. */
vie_status vie_set_diffusion_preconditioner(vie_handle *h, int enable, void *stream);

/* z = M v with the diffusion preconditioner alone (v, z FP64 [N], host or
 * device, not overlapping).  Errors: INVALID_ARG (none set), CUDA. */
vie_status vie_diffusion_precondition(vie_handle *h, const double *v, double *z, void *stream);

/* ---- Failure detection of the tensor-core kernels (no paper counterpart).
 * Every wait of the kernels that issue tcgen05.mma (the multi-RHS product of
 * VIE_OPERATOR_BF16X3 and the BF16 convolutions of the learned
 * preconditioner) on an mbarrier is bounded.  A CTA whose wait runs out stops
 * issuing work, waits (bounded by the full limit) for the copies and
 * products it already issued, frees its tensor memory, writes NaN into its
 * outputs and sets the error word of its handle or network.  Synchronous
 * calls report that as VIE_ERR_TIMEOUT: vie_solve_gmres (checked at every
 * Arnoldi step), vie_apply with host pointers, vie_unet_forward with
 * use_bf16 (which synchronises its stream) and vie_check_device; the word is
 * cleared when reported, so the next call runs normally.
 *
 * vie_set_wait_limits sets the bounds for later launches, process-wide, in
 * milliseconds (converted with the device's clock rate): limit_ms for every
 * wait (default 1000), first_wait_ms for the first producer/consumer wait of
 * each CTA (negative: the same as limit_ms; 0: that wait gives up at once,
 * which lets a test exercise the failure path without a fault).
 * Errors: INVALID_ARG (0 < limit_ms <= 60000 and first_wait_ms <= limit_ms
 * required). */
vie_status vie_set_wait_limits(double limit_ms, double first_wait_ms);

/* Synchronise `stream` and return VIE_ERR_TIMEOUT if a tensor-core kernel of
 * this handle (or of its learned preconditioner) gave up on a bounded wait
 * since the last report; asynchronous vie_apply calls report this way. */
vie_status vie_check_device(vie_handle *h, void *stream);

/* Device memory.  The library keeps the device buffers that vie_destroy,
 * vie_unet_destroy, vie_batch_destroy and workspace growth free, per device
 * and size class (512-byte steps up to 1 MiB, 2 MiB steps above; at most
 * 4 GiB in all), and hands them to later requests of the same class: a
 * handle created per solve then costs no cudaMalloc after the first.  Its
 * pinned host buffers (the solvers' read-back scalars) are kept likewise.  A
 * buffer enters the cache only after the device has finished with it.  An
 * allocation that fails releases the cache and tries again.
 * vie_release_memory synchronises the current device and returns every
 * cached buffer, device and pinned host, to CUDA (buffers still owned by live
 * objects stay).
 * Errors: none. */
vie_status vie_release_memory(void);

/* The pair kernel this handle's on-the-fly applies use (VIE_KERNEL_*). */
vie_status vie_get_kernel(vie_handle *h, int *kernel);

/* Multiply-adds that one on-the-fly apply spends on the optical depths, by
 * the method's own count (a diagnostic for rooflines; no counterpart in the
 * paper).  Displacement kernel: sum over displacements D of the cells of the
 * stencil W_D (the per-cell sum of the S midpoint samples' bilinear weights,
 * Section 3.2 M-iii) times the pairs with that displacement.  Other kernels:
 * 3 S per unordered pair (three linear blends per bilinear sample; 7 per
 * trilinear sample in 3D). */
vie_status vie_get_kernel_work(vie_handle *h, double *fma_per_apply);

/* Read back the self-cell diagonal d_j (FP64 [N], host or device). */
vie_status vie_get_diagonal(vie_handle *h, double *d, void *stream);

/* Message of the last failed call on this thread ("" if none). */
const char *vie_last_error(void);

/* Library version string. */
const char *vie_version(void);

/* Number of CUDA kernels this library has launched in this process (all
 * handles, all devices); a diagnostic for benchmarks. */
unsigned long long vie_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* VIE_H */
