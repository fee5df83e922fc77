/*
 * vie_oracle.c -- plain FP64 CPU oracle for the volume-integral-equation
 * (VIE) path of Ren, Zhang & Zhong, "A fast algorithm for radiative transport
 * in isotropic media" (arXiv 1610.00835).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA library; it is written
 * to be read against the paper, not to be fast (OpenMP over target rows is
 * the only concession).
 *
 * What it computes (Section 2, Eqs. EQ:Operator K, EQ:Kernel; Section 3.2,
 * Eqs. EQ: DISCRETIZED, EQ: KIJ, approach M-iii):
 *
 *   grid      : n cells per side on (0,1)^d, h = 1/n, centres x_j=(i+1/2)h,
 *               j = ix + n*iy (+ n*n*iz).                       (Section 3.1)
 *   sigma~    : bilinear (2D) / trilinear (3D) interpolation of the cell
 *               values on the lattice of cell centres, clamped to the hull
 *               of the centres (clamp-to-edge).
 *   tau(x,y)  : line integral of sigma_t along the segment x -> y
 *               (Section 2, definition of E(x,y)); evaluated either
 *               TAU_MARCH: (r/S) sum_{i=0}^{S-1} sigma~(x + (i+1/2)/S (y-x)),
 *               TAU_CLOSED: sigma_t r (homogeneous media, Eq. EQ:Kernel Cons),
 *               TAU_EXACT: exact integral of the piecewise-polynomial
 *               sigma~ (cross-check only).
 *   A_jk      : j != k:  h^d exp(-tau_jk) / (|S^{d-1}| r^{d-1})   (M-iii)
 *               j == k:  d_j = int_{T_j} exp(-sigma_t,j |z|)/(|S^{d-1}||z|^{d-1}) dz
 *               (self cell computed explicitly, sigma frozen at the centre)
 *               |S^1| = 2 pi, |S^2| = 4 pi.
 *               With the flag OR_DISC_MII in `mode` (2D only), approach
 *               M-ii with the kernel of Remark REM: NEW KERNEL instead:
 *               A_jk = exp(-tau_jk) / (2 pi) int_{T_k} |x_j - z|^{-1} dz for
 *               every j and k (tau_jj = 0), the cell integral in the
 *               closed form of that remark.
 *   K_jk      : A_jk sigma_s,k       (the matrix [K_jk omega_k] of
 *               Eq. EQ: LINEAR SYSTEM; omega_k = h^d is inside A).
 *   phi       : A f  (Eq. EQ:ERT Intgrl FMM: phi = K(mu_s^{-1} f); the
 *               sigma_s inside K cancels the mu_s^{-1}).
 *   U         : solution of (I - K) U = phi (Algorithm 1, S.2), by GMRES.
 *   sweep     : Algorithm 1, S.3 / Eq. EQ:ERT Intgrl: backward long
 *               characteristic from x_j in direction -v to the boundary,
 *               step-characteristic integration of exp(-tau) Q.
 *   DO solve  : source iteration of the full transport equation Eq. EQ:ERT
 *               (scattering with the angular mean) on a direction set;
 *               a brute-force check of the integral reformulation.
 *
 * Parity status: every function here is pinned by the not-gpu tests (closed
 * forms, limits, invariants, brute force) except the discrete-ordinates
 * source iteration, which agrees with the VIE only to discretisation level.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

enum { OR_TAU_MARCH = 0, OR_TAU_CLOSED = 1, OR_TAU_EXACT = 2 };
/* `mode` = tau mode | OR_DISC_MII (discretisation M-ii instead of M-iii) */
enum { OR_TAU_MASK = 15, OR_DISC_MII = 16 };
enum { OR_OP_K_SIGMA_S = 0, OR_OP_I_MINUS_K = 1, OR_OP_A_RAW = 2 };

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

/* ---------------------------------------------------------------- sigma~ */

/* Interpolate the cell values `v` (n per side) at physical point p.
 * Lattice coordinate u = p/h - 1/2 puts cell centres on the integers;
 * u is clamped to [0, n-1] (clamp-to-edge outside the hull of centres). */
double or_interp(int dim, int n, const double *v, const double *p) {
  if (n == 1) return v[0];
  int i0[3];
  double a[3];
  for (int d = 0; d < dim; ++d) {
    double u = p[d] * n - 0.5;
    if (u < 0.0) u = 0.0;
    if (u > n - 1) u = n - 1;
    int i = (int)floor(u);
    if (i > n - 2) i = n - 2;
    i0[d] = i;
    a[d] = u - i;
  }
  if (dim == 2) {
    const double *r0 = v + (long)i0[1] * n + i0[0];
    const double *r1 = r0 + n;
    double lo = (1.0 - a[0]) * r0[0] + a[0] * r0[1];
    double hi = (1.0 - a[0]) * r1[0] + a[0] * r1[1];
    return (1.0 - a[1]) * lo + a[1] * hi;
  }
  double out = 0.0;
  for (int cz = 0; cz < 2; ++cz)
    for (int cy = 0; cy < 2; ++cy)
      for (int cx = 0; cx < 2; ++cx) {
        double w = (cx ? a[0] : 1.0 - a[0]) * (cy ? a[1] : 1.0 - a[1]) *
                   (cz ? a[2] : 1.0 - a[2]);
        long idx = ((long)(i0[2] + cz) * n + (i0[1] + cy)) * n + (i0[0] + cx);
        out += w * v[idx];
      }
  return out;
}

static double dist(int dim, const double *x, const double *y) {
  double s = 0.0;
  for (int d = 0; d < dim; ++d) s += (y[d] - x[d]) * (y[d] - x[d]);
  return sqrt(s);
}

/* ------------------------------------------------------------------- tau */

/* S-step midpoint march of sigma~ along the segment x -> y. */
double or_tau_march(int dim, int n, const double *sig, const double *x,
                    const double *y, int S) {
  double r = dist(dim, x, y);
  double acc = 0.0, p[3];
  for (int i = 0; i < S; ++i) {
    double t = (i + 0.5) / S;
    for (int d = 0; d < dim; ++d) p[d] = x[d] + t * (y[d] - x[d]);
    acc += or_interp(dim, n, sig, p);
  }
  return r * acc / S;
}

static int cmp_double(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return (x > y) - (x < y);
}

/* Exact line integral of sigma~ along x -> y.  Between consecutive crossings
 * of lattice planes u_d = integer the interpolant is a polynomial of degree
 * <= dim in the arc parameter, so Simpson's rule on each piece is exact for
 * dim <= 3 (Simpson integrates cubics exactly). */
double or_tau_exact(int dim, int n, const double *sig, const double *x,
                    const double *y) {
  double r = dist(dim, x, y);
  if (r == 0.0) return 0.0;
  int cap = 2 + dim * (2 * n + 4);
  double *ts = (double *)malloc(sizeof(double) * cap);
  int m = 0;
  ts[m++] = 0.0;
  ts[m++] = 1.0;
  for (int d = 0; d < dim; ++d) {
    double u0 = x[d] * n - 0.5, u1 = y[d] * n - 0.5;
    if (u1 == u0) continue;
    for (int k = 0; k <= n - 1; ++k) {
      double t = (k - u0) / (u1 - u0);
      if (t > 0.0 && t < 1.0) ts[m++] = t;
    }
  }
  qsort(ts, m, sizeof(double), cmp_double);
  double acc = 0.0, p[3];
  for (int s = 0; s + 1 < m; ++s) {
    double ta = ts[s], tb = ts[s + 1];
    if (tb <= ta) continue;
    double tm = 0.5 * (ta + tb), f[3];
    double tt[3] = {ta, tm, tb};
    for (int q = 0; q < 3; ++q) {
      for (int d = 0; d < dim; ++d) p[d] = x[d] + tt[q] * (y[d] - x[d]);
      f[q] = or_interp(dim, n, sig, p);
    }
    acc += (tb - ta) / 6.0 * (f[0] + 4.0 * f[1] + f[2]);
  }
  free(ts);
  return r * acc;
}

/* ------------------------------------------------------------- self cell */

/* (1 - exp(-s R)) / s, with its limit R at s = 0 (radial integral of
 * exp(-s rho) from 0 to R). */
static double radial(double s, double R) {
  if (s == 0.0) return R;
  return -expm1(-s * R) / s;
}

typedef double (*fn1)(double, void *);

static double simpson_rec(fn1 f, void *ctx, double a, double b, double fa,
                          double fm, double fb, double whole, double tol,
                          int depth) {
  double m = 0.5 * (a + b);
  double lm = 0.5 * (a + m), rm = 0.5 * (m + b);
  double flm = f(lm, ctx), frm = f(rm, ctx);
  double left = (m - a) / 6.0 * (fa + 4.0 * flm + fm);
  double right = (b - m) / 6.0 * (fm + 4.0 * frm + fb);
  double diff = left + right - whole;
  if (depth <= 0 || fabs(diff) <= 15.0 * tol)
    return left + right + diff / 15.0;
  return simpson_rec(f, ctx, a, m, fa, flm, fm, left, 0.5 * tol, depth - 1) +
         simpson_rec(f, ctx, m, b, fm, frm, fb, right, 0.5 * tol, depth - 1);
}

/* Adaptive Simpson quadrature of f on [a, b] to absolute tolerance tol. */
double or_adaptive_simpson(fn1 f, void *ctx, double a, double b, double tol) {
  double fa = f(a, ctx), fb = f(b, ctx), fm = f(0.5 * (a + b), ctx);
  double whole = (b - a) / 6.0 * (fa + 4.0 * fm + fb);
  return simpson_rec(f, ctx, a, b, fa, fm, fb, whole, tol, 48);
}

struct sc_ctx { double sigma, a, phi, tol; };

/* 2D: polar coordinates about the centre of the square [-a,a]^2; by the
 * eight-fold symmetry theta in [0, pi/4] and the ray leaves the square at
 * R = a sec(theta).  d = (1/2pi) * 8 * int (1 - e^{-sigma R})/sigma dtheta. */
static double sc2_integrand(double th, void *c) {
  struct sc_ctx *q = (struct sc_ctx *)c;
  return radial(q->sigma, q->a / cos(th));
}

/* 3D: spherical coordinates about the centre of the cube [-a,a]^3.  The
 * directions through one face x = a are parametrised by the face point
 * (a, s cos(phi), s sin(phi)); rho = sqrt(a^2 + s^2), solid angle
 * a s ds dphi / rho^3 = a drho dphi / rho^2 (s ds = rho drho).  Six faces,
 * eight symmetric triangles per face, phi in [0, pi/4], s in [0, a sec phi]. */
static double sc3_inner(double rho, void *c) {
  struct sc_ctx *q = (struct sc_ctx *)c;
  return q->a * radial(q->sigma, rho) / (rho * rho);
}

static double sc3_outer(double phi, void *c) {
  struct sc_ctx *q = (struct sc_ctx *)c;
  double sec = 1.0 / cos(phi);
  double rmax = q->a * sqrt(1.0 + sec * sec);
  return or_adaptive_simpson(sc3_inner, q, q->a, rmax, q->tol);
}

/* Self-cell value d = int_{cell} exp(-sigma |z|) / (|S^{d-1}| |z|^{d-1}) dz
 * for a cell of side h centred at the origin (M-iii, self term computed
 * explicitly with sigma frozen at the collocation point). */
double or_selfcell(int dim, double h, double sigma) {
  struct sc_ctx q;
  q.sigma = sigma;
  q.a = 0.5 * h;
  if (dim == 2) {
    q.tol = 1e-15 * h;
    double I = or_adaptive_simpson(sc2_integrand, &q, 0.0, OR_PI / 4.0, q.tol);
    return 8.0 * I / (2.0 * OR_PI);
  }
  q.tol = 1e-15 * h;
  double I = or_adaptive_simpson(sc3_outer, &q, 0.0, OR_PI / 4.0, q.tol);
  return 6.0 * 8.0 * I / (4.0 * OR_PI);
}

/* ---------------------------------------------------------------- kernel */

static void centre(int dim, int n, long j, double *x) {
  double h = 1.0 / n;
  long ix = j % n, rest = j / n;
  x[0] = (ix + 0.5) * h;
  if (dim == 2) {
    x[1] = (rest + 0.5) * h;
  } else {
    x[1] = (rest % n + 0.5) * h;
    x[2] = (rest / n + 0.5) * h;
  }
}

static double sphere_area(int dim) { return dim == 2 ? 2.0 * OR_PI : 4.0 * OR_PI; }

static double tau_of(int dim, int n, const double *st, int mode, int S,
                     const double *x, const double *y) {
  mode &= OR_TAU_MASK;
  if (mode == OR_TAU_CLOSED) return st[0] * dist(dim, x, y);
  if (mode == OR_TAU_EXACT) return or_tau_exact(dim, n, st, x, y);
  return or_tau_march(dim, n, st, x, y, S);
}

/* F(r, s) of Remark REM: NEW KERNEL (Section 3.2): an antiderivative of
 * 1/sqrt(r^2 + s^2) in r and in s, odd in each argument.  It vanishes where
 * r = 0 or s = 0 (the sign factors), which also covers the r log r terms. */
static double paper_F(double r, double s) {
  if (r == 0.0 || s == 0.0) return 0.0;
  double ar = fabs(r), as = fabs(s), rho = sqrt(r * r + s * s);
  double v = ar * log(as + rho) + as * log(ar + rho) - ar * log(ar) - as * log(as);
  return ((r > 0) == (s > 0)) ? v : -v;
}

/* int over the square of side h centred at t = (t1, t2) of |z|^{-1} dz: the
 * four-corner sum of F in the remark (2D). */
double or_cell_integral2(double t1, double t2, double h) {
  double acc = 0.0;
  for (int i = -1; i <= 1; i += 2)
    for (int jj = -1; jj <= 1; jj += 2)
      acc += i * jj * paper_F(t1 + i * 0.5 * h, t2 + jj * 0.5 * h);
  return acc;
}

/* A_jk.  M-iii: off-diagonal weight h^d e^{-tau}/(|S| r^{d-1}), the diagonal
 * the self-cell value d_j.  M-ii (2D): e^{-tau} / (2 pi) times the cell
 * integral of |x_j - z|^{-1} over T_k, the same formula on the diagonal. */
double or_entry(int dim, int n, const double *st, int mode, int S, long j,
                long k) {
  double h = 1.0 / n;
  double x[3], y[3];
  if (mode & OR_DISC_MII) {
    if (dim != 2) return NAN;
    centre(dim, n, j, x);
    centre(dim, n, k, y);
    double tau = j == k ? 0.0 : tau_of(dim, n, st, mode, S, x, y);
    return exp(-tau) * or_cell_integral2(y[0] - x[0], y[1] - x[1], h) / sphere_area(dim);
  }
  if (j == k) return or_selfcell(dim, h, st[j]);
  centre(dim, n, j, x);
  centre(dim, n, k, y);
  double r = dist(dim, x, y);
  double tau = tau_of(dim, n, st, mode, S, x, y);
  double hd = dim == 2 ? h * h : h * h * h;
  double rd = dim == 2 ? r : r * r;
  return hd * exp(-tau) / (sphere_area(dim) * rd);
}

static long npow(int n, int dim) { return dim == 2 ? (long)n * n : (long)n * n * n; }

/* Diagonal d_j for every cell. */
void or_selfcells(int dim, int n, const double *st, double *d) {
  long N = npow(n, dim);
  double h = 1.0 / n;
#pragma omp parallel for schedule(dynamic, 16)
  for (long j = 0; j < N; ++j) d[j] = or_selfcell(dim, h, st[j]);
}

/* Diagonal A_jj of the discretisation `mode` for every cell. */
static void diagonal(int dim, int n, const double *st, int mode, double *d) {
  if (!(mode & OR_DISC_MII)) {
    or_selfcells(dim, n, st, d);
    return;
  }
  long N = npow(n, dim);
  for (long j = 0; j < N; ++j) d[j] = or_entry(dim, n, st, mode, 64, j, j);
}

/* Dense A (N x N, row-major, A[j*N + k]). */
void or_assemble(int dim, int n, const double *st, int mode, int S, double *A) {
  long N = npow(n, dim);
  double *d = (double *)malloc(sizeof(double) * N);
  diagonal(dim, n, st, mode, d);
#pragma omp parallel for schedule(dynamic, 4)
  for (long j = 0; j < N; ++j)
    for (long k = 0; k < N; ++k)
      A[j * N + k] = (j == k) ? d[j] : or_entry(dim, n, st, mode, S, j, k);
  free(d);
}

/* Matrix-free apply on target rows `rows` (all rows if rows == NULL):
 *   op K_SIGMA_S : y_j = sum_k A_jk sigma_s,k g_k
 *   op I_MINUS_K : y_j = g_j - sum_k A_jk sigma_s,k g_k
 *   op A_RAW     : y_j = sum_k A_jk g_k          (phi = A f)
 * `diag` may hold precomputed d_j (NULL: computed here per row); M-ii
 * ignores it and takes every entry, the diagonal included, from or_entry. */
void or_apply(int dim, int n, const double *st, const double *ss, int mode,
              int S, int op, const double *diag, const double *g,
              const long *rows, long nrows, double *y) {
  long N = npow(n, dim);
  if (rows == NULL) nrows = N;
  double h = 1.0 / n;
#pragma omp parallel for schedule(dynamic, 1)
  for (long r = 0; r < nrows; ++r) {
    long j = rows ? rows[r] : r;
    double acc = 0.0;
    for (long k = 0; k < N; ++k) {
      double a = (k == j && !(mode & OR_DISC_MII))
                     ? (diag ? diag[j] : or_selfcell(dim, h, st[j]))
                     : or_entry(dim, n, st, mode, S, j, k);
      double s = (op == OR_OP_A_RAW) ? 1.0 : ss[k];
      acc += a * s * g[k];
    }
    y[r] = (op == OR_OP_I_MINUS_K) ? g[j] - acc : acc;
  }
}

/* Dense y = M x (N x N row-major). */
void or_matvec(long N, const double *M, const double *x, double *y) {
#pragma omp parallel for
  for (long j = 0; j < N; ++j) {
    double acc = 0.0;
    for (long k = 0; k < N; ++k) acc += M[j * N + k] * x[k];
    y[j] = acc;
  }
}

/* ----------------------------------------------------------------- GMRES */

static double dot(long N, const double *a, const double *b) {
  double s = 0.0;
  for (long i = 0; i < N; ++i) s += a[i] * b[i];
  return s;
}

struct op_ctx {
  int dim, n, mode, S;
  const double *st, *ss, *diag, *dense; /* dense: N x N matrix of (I - K) */
};

static void op_apply(const struct op_ctx *c, const double *x, double *y) {
  long N = npow(c->n, c->dim);
  if (c->dense) {
    or_matvec(N, c->dense, x, y);
  } else {
    or_apply(c->dim, c->n, c->st, c->ss, c->mode, c->S, OR_OP_I_MINUS_K,
             c->diag, x, NULL, N, y);
  }
}

/* Restarted GMRES(m) for (I - K) U = phi (Algorithm 1, S.2), textbook form:
 * Arnoldi with modified Gram-Schmidt, Givens rotations on the Hessenberg
 * matrix, stop when the true relative residual ||phi - (I-K)U|| / ||phi||
 * <= rtol (checked at every restart and on the estimate inside a cycle).
 * `dense`, if not NULL, is the N x N matrix (I - K) used instead of the
 * matrix-free apply.  U holds the initial guess on entry.  Returns 0 when
 * converged, 1 otherwise; *iters counts Arnoldi steps. */
int or_gmres(int dim, int n, const double *st, const double *ss, int mode,
             int S, const double *dense, const double *phi, double *U,
             double rtol, int m, int maxit, int *iters, double *relres) {
  long N = npow(n, dim);
  struct op_ctx c = {dim, n, mode, S, st, ss, NULL, dense};
  double *diag = NULL;
  if (!dense) {
    diag = (double *)malloc(sizeof(double) * N);
    diagonal(dim, n, st, mode, diag);
    c.diag = diag;
  }
  double *V = (double *)malloc(sizeof(double) * N * (m + 1));
  double *H = (double *)calloc((size_t)(m + 1) * m, sizeof(double));
  double *cs = (double *)malloc(sizeof(double) * m);
  double *sn = (double *)malloc(sizeof(double) * m);
  double *gv = (double *)malloc(sizeof(double) * (m + 1));
  double *yv = (double *)malloc(sizeof(double) * m);
  double *w = (double *)malloc(sizeof(double) * N);
  double bnorm = sqrt(dot(N, phi, phi));
  if (bnorm == 0.0) bnorm = 1.0;
  int it = 0, converged = 0;
  double rel = 1.0;
  while (it < maxit) {
    op_apply(&c, U, w);
    for (long i = 0; i < N; ++i) w[i] = phi[i] - w[i];
    double beta = sqrt(dot(N, w, w));
    rel = beta / bnorm;
    if (rel <= rtol) { converged = 1; break; }
    for (long i = 0; i < N; ++i) V[i] = w[i] / beta;
    memset(gv, 0, sizeof(double) * (m + 1));
    gv[0] = beta;
    int k;
    for (k = 0; k < m && it < maxit; ++k) {
      ++it;
      double *vk1 = V + (long)(k + 1) * N;
      op_apply(&c, V + (long)k * N, vk1);
      for (int i = 0; i <= k; ++i) {
        double hik = dot(N, V + (long)i * N, vk1);
        H[i * m + k] = hik;
        for (long q = 0; q < N; ++q) vk1[q] -= hik * V[(long)i * N + q];
      }
      double hk1 = sqrt(dot(N, vk1, vk1));
      H[(k + 1) * m + k] = hk1;
      if (hk1 != 0.0)
        for (long q = 0; q < N; ++q) vk1[q] /= hk1;
      for (int i = 0; i < k; ++i) {
        double a = H[i * m + k], b = H[(i + 1) * m + k];
        H[i * m + k] = cs[i] * a + sn[i] * b;
        H[(i + 1) * m + k] = -sn[i] * a + cs[i] * b;
      }
      double a = H[k * m + k], b = H[(k + 1) * m + k];
      double den = sqrt(a * a + b * b);
      cs[k] = den == 0.0 ? 1.0 : a / den;
      sn[k] = den == 0.0 ? 0.0 : b / den;
      H[k * m + k] = den;
      H[(k + 1) * m + k] = 0.0;
      gv[k + 1] = -sn[k] * gv[k];
      gv[k] = cs[k] * gv[k];
      if (fabs(gv[k + 1]) / bnorm <= rtol || hk1 == 0.0) { ++k; break; }
    }
    for (int i = k - 1; i >= 0; --i) {
      double s = gv[i];
      for (int q = i + 1; q < k; ++q) s -= H[i * m + q] * yv[q];
      yv[i] = s / H[i * m + i];
    }
    for (int i = 0; i < k; ++i)
      for (long q = 0; q < N; ++q) U[q] += yv[i] * V[(long)i * N + q];
  }
  if (!converged) {
    op_apply(&c, U, w);
    for (long i = 0; i < N; ++i) w[i] = phi[i] - w[i];
    rel = sqrt(dot(N, w, w)) / bnorm;
    converged = rel <= rtol;
  }
  *iters = it;
  *relres = rel;
  free(V); free(H); free(cs); free(sn); free(gv); free(yv); free(w); free(diag);
  return converged ? 0 : 1;
}

/* ----------------------------------------------------------------- sweep */

/* Distance from x to the boundary of (0,1)^d travelling in direction -v
 * (the tau(x,v) of Eq. EQ:ERT Intgrl). */
double or_exit_length(int dim, const double *x, const double *v) {
  double L = INFINITY;
  for (int d = 0; d < dim; ++d) {
    if (v[d] > 0.0) L = fmin(L, x[d] / v[d]);
    else if (v[d] < 0.0) L = fmin(L, (1.0 - x[d]) / (-v[d]));
  }
  return L;
}

/* Number of march steps for a ray of length L on an n-grid: steps of at
 * most h/2 (at least one step). */
long or_sweep_steps(int n, double L) {
  long m = (long)ceil(L * 2.0 * n - 1e-6);
  return m < 1 ? 1 : m;
}

/* Scattering-free transport solve (Algorithm 1, S.3 (ii)) along the backward
 * characteristic, Eq. EQ:ERT Intgrl with q = Q:
 *   Phi(x,v) = int_0^{L} exp(-int_0^l sigma_t(x - l'v) dl') Q(x - l v) dl.
 * The ray is cut into equal steps of length Delta <= h/2; on each step sigma~
 * and Q~ are frozen at the step midpoint and the step is integrated exactly:
 *   Phi += e^{-tau_acc} Q~ (1 - e^{-sigma~ Delta}) / sigma~,  tau_acc += sigma~ Delta.
 * dirs: [M][dim] unit vectors; Phi: [M][N]. */
void or_sweep(int dim, int n, const double *st, const double *Q,
              const double *dirs, int M, double *Phi) {
  long N = npow(n, dim);
#pragma omp parallel for collapse(2) schedule(dynamic, 64)
  for (int m = 0; m < M; ++m)
    for (long j = 0; j < N; ++j) {
      const double *v = dirs + (long)m * dim;
      double x[3], p[3];
      centre(dim, n, j, x);
      double L = or_exit_length(dim, x, v);
      long ns = or_sweep_steps(n, L);
      double dl = L / ns, tau = 0.0, acc = 0.0;
      for (long s = 0; s < ns; ++s) {
        double l = (s + 0.5) * dl;
        for (int d = 0; d < dim; ++d) p[d] = x[d] - l * v[d];
        double sg = or_interp(dim, n, st, p);
        double q = or_interp(dim, n, Q, p);
        acc += exp(-tau) * q * radial(sg, dl);
        tau += sg * dl;
      }
      Phi[(long)m * N + j] = acc;
    }
}

/* Discrete-ordinates source iteration for the full transport equation
 * Eq. EQ:ERT with scattering through the angular mean (equal weights over
 * the M directions):  Q = sigma_s U + f,  Phi = sweep(Q),  U = mean_m Phi.
 * Stops when ||U_new - U|| <= tol ||U_new||.  Returns iterations used. */
int or_do_solve(int dim, int n, const double *st, const double *ss,
                const double *f, const double *dirs, int M, double tol,
                int maxit, double *U) {
  long N = npow(n, dim);
  double *Q = (double *)malloc(sizeof(double) * N);
  double *Phi = (double *)malloc(sizeof(double) * N * M);
  for (long j = 0; j < N; ++j) U[j] = 0.0;
  int it;
  for (it = 1; it <= maxit; ++it) {
    for (long j = 0; j < N; ++j) Q[j] = ss[j] * U[j] + f[j];
    or_sweep(dim, n, st, Q, dirs, M, Phi);
    double dn = 0.0, un = 0.0;
    for (long j = 0; j < N; ++j) {
      double s = 0.0;
      for (int m = 0; m < M; ++m) s += Phi[(long)m * N + j];
      s /= M;
      dn += (s - U[j]) * (s - U[j]);
      un += s * s;
      U[j] = s;
    }
    if (sqrt(dn) <= tol * sqrt(un)) break;
  }
  free(Q);
  free(Phi);
  return it;
}
