"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test names what pins it: a closed form, a limit, an invariant or a brute
force.  None of them re-types the oracle's own formula.
"""
import math

import numpy as np
import pytest

import oracle as O
import vie_synth as V


# --------------------------------------------------------------- self cell

def paper_F(r, s):
    """F(r, s) of Remark REM: NEW KERNEL (Section 3.2), the closed form of the
    cell integral of |x - z|^{-1} in 2D."""
    def xlogx(u):
        return 0.0 if u == 0.0 else u * math.log(u)
    rho = math.hypot(r, s)
    val = 0.0
    if r != 0.0:
        val += abs(r) * math.log(abs(s) + rho)
    if s != 0.0:
        val += abs(s) * math.log(abs(r) + rho)
    val -= xlogx(abs(r)) + xlogx(abs(s))
    return math.copysign(1.0, r) * math.copysign(1.0, s) * val if r and s else 0.0


def paper_cell_integral(t1, t2, h):
    return sum(i * j * paper_F(t1 + i * h / 2, t2 + j * h / 2) for i in (-1, 1) for j in (-1, 1))


@pytest.mark.parametrize("h", [1 / 32, 0.1, 0.37])
def test_selfcell_2d_zero_sigma_matches_paper_F(h):
    # sigma -> 0: d = (1/2pi) int_T |z|^{-1} dz, the paper's closed form at t = 0.
    want = paper_cell_integral(0.0, 0.0, h) / (2 * math.pi)
    assert O.selfcell(2, h, 0.0) == pytest.approx(want, rel=1e-12)


def test_paper_F_against_offcentre_brute_force():
    # Sanity of the F transcription itself: off-centre cell, midpoint brute force.
    h, t1, t2 = 0.1, 0.3, 0.1
    K = 2000
    u = (np.arange(K) + 0.5) / K * h - h / 2
    zx, zy = np.meshgrid(t1 + u, t2 + u)
    bf = np.sum(1.0 / np.hypot(zx, zy)) * (h / K) ** 2
    assert paper_cell_integral(t1, t2, h) == pytest.approx(bf, rel=1e-6)


@pytest.mark.parametrize("h", [1 / 32, 0.2])
def test_selfcell_2d_odd_and_even_parts(h):
    # d(sigma) = (1/2pi) int_T e^{-sigma rho}/rho dA.  Odd part in sigma:
    # -(1/2pi)(sigma |T| + (sigma^3/6) int_T rho^2 dA) + O(sigma^5), with
    # |T| = h^2 and int_T rho^2 dA = h^4/6.  The even part's sigma^2
    # coefficient is (1/4pi) int_T rho dA = (1/4pi)(4a^3/3)(sqrt2 + ln(1+sqrt2)).
    s = 2e-3 / h
    dp, dm, d0 = O.selfcell(2, h, s), O.selfcell(2, h, -s), O.selfcell(2, h, 0.0)
    odd = (dp - dm) / (2 * s)
    assert odd == pytest.approx(-(h * h + s * s * h ** 4 / 36) / (2 * math.pi), rel=1e-9)
    a = h / 2
    even = ((dp + dm) / 2 - d0) / s ** 2
    want = (4 * a ** 3 / 3) * (math.sqrt(2) + math.log(1 + math.sqrt(2))) / (4 * math.pi)
    assert even == pytest.approx(want, rel=1e-5)


def test_selfcell_3d_even_part_is_cell_volume():
    # d(sigma) = (1/4pi) int_T e^{-sigma rho}/rho^2 dV; sigma^2 coefficient of
    # the even part is (1/4pi)(1/2)|T| = h^3/(8 pi).
    h = 0.05
    s = 2e-3 / h
    dp, dm, d0 = O.selfcell(3, h, s), O.selfcell(3, h, -s), O.selfcell(3, h, 0.0)
    even = ((dp + dm) / 2 - d0) / s ** 2
    assert even == pytest.approx(h ** 3 / (8 * math.pi), rel=1e-5)


def _midpoint_cell(dim, h, sigma, K):
    u = (np.arange(K) + 0.5) / K * h - h / 2
    grids = np.meshgrid(*([u] * dim), indexing="ij")
    rho = np.sqrt(sum(g * g for g in grids))
    area = 2 * math.pi if dim == 2 else 4 * math.pi
    return np.sum(np.exp(-sigma * rho) / (area * rho ** (dim - 1))) * (h / K) ** dim


@pytest.mark.parametrize("dim,sigma", [(2, 0.0), (2, 7.5), (3, 0.0), (3, 3.0), (3, 40.0)])
def test_selfcell_brute_force_midpoint(dim, sigma):
    # Brute force: midpoint sums M(K) on K^d sub-cells (K even, so the singular
    # point is a sub-cell vertex).  The error expands in 1/K and 1/K^2, so two
    # Richardson levels over K/4, K/2, K remove both leading terms.
    h = 0.1
    K = 512 if dim == 2 else 128
    m = [_midpoint_cell(dim, h, sigma, K // q) for q in (4, 2, 1)]
    r1 = [2 * m[1] - m[0], 2 * m[2] - m[1]]
    extrap = (4 * r1[1] - r1[0]) / 3
    assert O.selfcell(dim, h, sigma) == pytest.approx(extrap, rel=1e-6)


# ------------------------------------------------------------------- tau

def _cubic_coeffs_along(dim, factors, x, y):
    """Coefficients of prod_d (a_d + b_d p_d(t)), p(t) = x + t (y - x), in t."""
    poly = np.array([1.0])
    for d in range(dim):
        a, b = factors[d]
        lin = np.array([a + b * x[d], b * (y[d] - x[d])])  # c0 + c1 t
        poly = np.convolve(poly, lin)
    return np.pad(poly, (0, 4 - poly.size))


@pytest.mark.parametrize("dim", [2, 3])
def test_tau_linear_field_is_midpoint_value(dim):
    # For linear sigma_t, multilinear interpolation and the midpoint march are
    # both exact: tau = r sigma_t((x + y) / 2).
    n = 9 if dim == 3 else 17
    beta = [0.7, -1.3, 0.4][:dim]
    st = V.linear_field(dim, n, 2.0, beta)
    xs = V.cell_centres(dim, n)
    rng = np.random.default_rng(1)
    for _ in range(40):
        j, k = rng.integers(0, n ** dim, 2)
        x, y = xs[j], xs[k]
        r = np.linalg.norm(y - x)
        want = r * (2.0 + np.dot(beta, (x + y) / 2))
        assert O.tau_march(dim, st, x, y, 64) == pytest.approx(want, rel=1e-13, abs=1e-15)
        assert O.tau_exact(dim, st, x, y) == pytest.approx(want, rel=1e-13, abs=1e-15)


@pytest.mark.parametrize("dim,S", [(2, 64), (2, 7), (3, 64), (3, 5)])
def test_tau_product_field_closed_form(dim, S):
    # sigma = prod_d (a_d + b_d x_d) is reproduced exactly by multilinear
    # interpolation; along the segment it is a polynomial q(t) of degree dim.
    # Exact integral: r int_0^1 q.  S-step midpoint rule: r (int q - c2/(12 S^2)
    # - c3/(8 S^2)) (composite midpoint errors of t^2 and t^3).
    n = 11 if dim == 3 else 23
    factors = [(1.0, 0.8), (1.5, -0.9), (0.7, 1.1)][:dim]
    xs = V.cell_centres(dim, n)
    st = np.ones(n ** dim)
    for d in range(dim):
        st = st * (factors[d][0] + factors[d][1] * xs[:, d])
    rng = np.random.default_rng(7)
    for _ in range(30):
        j, k = rng.integers(0, n ** dim, 2)
        x, y = xs[j], xs[k]
        r = np.linalg.norm(y - x)
        c = _cubic_coeffs_along(dim, factors, x, y)
        integral = c[0] + c[1] / 2 + c[2] / 3 + c[3] / 4
        march = integral - c[2] / (12 * S * S) - c[3] / (8 * S * S)
        assert O.tau_exact(dim, st, x, y) == pytest.approx(r * integral, rel=1e-12, abs=1e-14)
        assert O.tau_march(dim, st, x, y, S) == pytest.approx(r * march, rel=1e-12, abs=1e-14)


def test_tau_march_converges_to_exact_on_bump_medium():
    m = V.heterogeneous_2d(n=24)
    xs = V.cell_centres(2, 24)
    x, y = xs[3 + 24 * 5], xs[20 + 24 * 17]
    ex = O.tau_exact(2, m.sigma_t, x, y)
    errs = [abs(O.tau_march(2, m.sigma_t, x, y, S) - ex) for S in (64, 256, 1024, 4096)]
    assert errs[-1] < 1e-6 * ex
    assert errs[0] > errs[-1]


def test_interp_clamps_outside_hull():
    n = 8
    st = V.linear_field(2, n, 1.0, [1.0, 2.0])
    # outside the hull of centres the value is that of the nearest hull point
    assert O.interp(2, st, [0.0, 0.5]) == pytest.approx(O.interp(2, st, [0.5 / n, 0.5]))
    assert O.interp(2, st, [0.3, 1.0]) == pytest.approx(O.interp(2, st, [0.3, 1 - 0.5 / n]))


# ---------------------------------------------------------------- kernel

@pytest.mark.parametrize("dim", [2, 3])
def test_reciprocity(dim):
    # A_jk = A_kj: the midpoint sample set is symmetric under x <-> y.
    m = V.heterogeneous_2d(n=16) if dim == 2 else V.heterogeneous_3d(n=8)
    rng = np.random.default_rng(3)
    for _ in range(50):
        j, k = rng.integers(0, m.N, 2)
        a, b = O.entry(dim, m.sigma_t, j, k), O.entry(dim, m.sigma_t, k, j)
        assert a == pytest.approx(b, rel=1e-13)
        assert a > 0


def test_homogeneous_entry_closed_form():
    # Eq. EQ:Kernel Cons: constant sigma gives h^2 e^{-sigma r}/(2 pi r).
    n = 16
    st = np.full(n * n, 1.1)
    xs = V.cell_centres(2, n)
    for j, k in [(0, 1), (5, 200), (17, 255)]:
        r = np.linalg.norm(xs[j] - xs[k])
        want = math.exp(-1.1 * r) / (2 * math.pi * r) / n ** 2
        assert O.entry(2, st, j, k, mode=O.TAU_MARCH) == pytest.approx(want, rel=1e-13)
        assert O.entry(2, st, j, k, mode=O.TAU_CLOSED) == pytest.approx(want, rel=1e-14)


@pytest.mark.parametrize("dim,sizes", [(2, (41, 81, 161))])
def test_row_sum_disk_closed_form(dim, sizes):
    # int_{|y|<R} e^{-sigma|y|}/(|S^{d-1}| |y|^{d-1}) dy = (1 - e^{-sigma R})/sigma
    # in 2D and 3D.  The M-iii row sum over the cells of a disk (ball) plus the
    # self cell converges to it at O(h).
    sigma, R = 1.1, 0.25
    want = (1 - math.exp(-sigma * R)) / sigma
    errs = []
    for n in sizes:
        st = np.full(n ** dim, sigma)
        xs = V.cell_centres(dim, n)
        c = n ** dim // 2  # n odd: the centre cell sits at (1/2, ..., 1/2)
        g = (np.linalg.norm(xs - xs[c], axis=1) < R).astype(float)
        got = O.apply(dim, st, st, g, op=O.OP_A_RAW, mode=O.TAU_CLOSED, rows=[c])[0]
        errs.append(abs(got - want) / want)
    assert errs[-1] < errs[0]
    assert errs[-1] < 2.5 / sizes[-1]


@pytest.mark.parametrize("dim,sizes", [(2, (41, 81, 161)), (3, (21, 41))])
def test_row_sum_gaussian_weight_closed_form(dim, sizes):
    # With a Gaussian weight g(y) = exp(-|y|^2/(2w^2)) about an interior centre,
    # int e^{-sigma rho} g / (|S^{d-1}| rho^{d-1}) dy = int_0^inf e^{-sigma rho -
    # rho^2/(2w^2)} drho = w sqrt(pi/2) e^{sigma^2 w^2/2} erfc(sigma w/sqrt2) in
    # both 2D and 3D.  M-iii plus the self cell converges to it at the first
    # order that Eq. EQ: ERROR states for M-iii.
    sigma, w = 1.1, 0.08
    want = w * math.sqrt(math.pi / 2) * math.exp(sigma ** 2 * w ** 2 / 2) * math.erfc(
        sigma * w / math.sqrt(2))
    errs = []
    for n in sizes:
        st = np.full(n ** dim, sigma)
        xs = V.cell_centres(dim, n)
        c = n ** dim // 2
        g = np.exp(-np.sum((xs - xs[c]) ** 2, axis=1) / (2 * w * w))
        got = O.apply(dim, st, st, g, op=O.OP_A_RAW, mode=O.TAU_CLOSED, rows=[c])[0]
        errs.append(abs(got - want) / want)
    order = math.log(errs[-2] / errs[-1]) / math.log(sizes[-1] / sizes[-2])
    assert 0.75 < order < 1.3
    assert errs[-1] < 1.5 / sizes[-1]


# ------------------------------------------------- M-ii (Remark REM: NEW KERNEL)

@pytest.mark.parametrize("h", [1 / 64, 0.1, 0.5])
def test_mii_cell_integral_centre_closed_form(h):
    # int_{[-a,a]^2} |z|^{-1} dz = 8 a ln(1 + sqrt 2) (polar integral over the
    # eight triangles of the square), a = h / 2
    assert O.cell_integral2(0.0, 0.0, h) == pytest.approx(4 * h * math.log(1 + math.sqrt(2)), rel=1e-13)


def _gauss_legendre_cell(t1, t2, h, sub=8, q=16):
    # composite tensor Gauss-Legendre quadrature of |z|^{-1} over the square of
    # side h centred at (t1, t2) (smooth there: the square avoids the origin)
    x, wq = np.polynomial.legendre.leggauss(q)
    edges = np.linspace(-h / 2, h / 2, sub + 1)
    pts, wts = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        pts.append((a + b) / 2 + (b - a) / 2 * x)
        wts.append((b - a) / 2 * wq)
    p, w = np.concatenate(pts), np.concatenate(wts)
    zx, zy = np.meshgrid(t1 + p, t2 + p, indexing="ij")
    return float(np.sum(np.outer(w, w) / np.hypot(zx, zy)))


@pytest.mark.parametrize("t", [(1, 0), (0, -1), (1, 1), (-2, 1), (5, -3), (0, 7)])
def test_mii_cell_integral_against_quadrature(t):
    h = 0.1
    t1, t2 = t[0] * h, t[1] * h
    assert O.cell_integral2(t1, t2, h) == pytest.approx(_gauss_legendre_cell(t1, t2, h), rel=1e-11)


def test_mii_cell_integral_far_field_expansion():
    # the cell average of 1/|t + z| is 1/|t| + (h^2/24) Laplacian(1/|t|) + O(|t|^-5),
    # and in 2D Laplacian(1/r) = 1/r^3: after the two leading terms the rest
    # falls like |t|^-5
    h = 0.01
    rest = []
    for m in (10, 20, 40):
        t1, t2 = 0.6 * m * h, 0.8 * m * h
        r = m * h
        rest.append(O.cell_integral2(t1, t2, h) - h * h * (1 / r + h * h / (24 * r ** 3)))
    assert rest[0] / rest[1] == pytest.approx(32, rel=0.15)
    assert rest[1] / rest[2] == pytest.approx(32, rel=0.15)


def test_mii_reciprocity_and_diagonal():
    # A_jk = A_kj (the cell integral is even in t, tau symmetric); the diagonal
    # is the cell integral at t = 0 over 2 pi, i.e. the self cell without
    # attenuation
    n = 7
    st = V.bump_medium(2, n, 3, 0.9, seed=71).sigma_t
    A = O.assemble(2, st, mode=O.TAU_MARCH | O.DISC_MII)
    np.testing.assert_allclose(A, A.T, rtol=1e-13, atol=0)
    np.testing.assert_allclose(np.diag(A), O.selfcell(2, 1 / n, 0.0), rtol=1e-13)


def test_mii_row_sum_gaussian_weight_second_order():
    # The Gaussian-weight closed form of the M-iii test above: M-ii converges
    # at the h^2 (1 + log h) rate that Eq. EQ: ERROR states for it
    sigma, w = 1.1, 0.08
    want = w * math.sqrt(math.pi / 2) * math.exp(sigma ** 2 * w ** 2 / 2) * math.erfc(
        sigma * w / math.sqrt(2))
    sizes = (41, 81, 161)
    errs = []
    for n in sizes:
        st = np.full(n * n, sigma)
        xs = V.cell_centres(2, n)
        c = n * n // 2
        g = np.exp(-np.sum((xs - xs[c]) ** 2, axis=1) / (2 * w * w))
        got = O.apply(2, st, st, g, op=O.OP_A_RAW, mode=O.TAU_CLOSED | O.DISC_MII, rows=[c])[0]
        errs.append(abs(got - want) / want)
    order = math.log(errs[-2] / errs[-1]) / math.log(sizes[-1] / sizes[-2])
    assert 1.6 < order < 2.3
    assert errs[-1] < 7 / sizes[-1] ** 2 < errs[0]


def test_mii_gmres_matches_lu():
    n = 9
    m = V.bump_medium(2, n, 3, 0.9, seed=72)
    mode = O.TAU_MARCH | O.DISC_MII
    phi = O.apply(2, m.sigma_t, m.sigma_s, m.f, op=O.OP_A_RAW, mode=mode)
    U, it, rr, ok = O.gmres(2, m.sigma_t, m.sigma_s, phi, rtol=1e-12, mode=mode)
    assert ok
    np.testing.assert_allclose(U, O.lu_solve(2, m.sigma_t, m.sigma_s, phi, mode=mode), rtol=1e-9, atol=0)


def test_sigma_s_zero_is_pure_absorption():
    # sigma_s = 0: K = 0 and U = phi; GMRES stops at once.
    m = V.heterogeneous_2d(n=12)
    ss = np.zeros(m.N)
    phi = O.apply(2, m.sigma_t, ss, m.f, op=O.OP_A_RAW)
    U, it, rr, ok = O.gmres(2, m.sigma_t, ss, phi, rtol=1e-12)
    assert ok and it <= 1
    np.testing.assert_allclose(U, phi, rtol=1e-13)


def test_lu_equals_gmres_and_positivity():
    m = V.heterogeneous_2d(n=16)
    phi = O.apply(2, m.sigma_t, m.sigma_s, m.f, op=O.OP_A_RAW)
    U_lu = O.lu_solve(2, m.sigma_t, m.sigma_s, phi)
    U, it, rr, ok = O.gmres(2, m.sigma_t, m.sigma_s, phi, rtol=1e-12)
    assert ok and rr <= 1e-12
    np.testing.assert_allclose(U, U_lu, rtol=1e-10, atol=1e-14 * np.abs(U_lu).max())
    assert np.all(phi >= 0) and np.all(U >= phi)


def test_neumann_series_contracts():
    # ||K||_inf <= max sigma_s/sigma_t < 1 (Eq. EQ:ERT Intgrl FMM is uniquely
    # solvable); the Neumann series converges to the LU solution.
    m = V.heterogeneous_2d(n=12)
    K = O.k_matrix(2, m.sigma_t, m.sigma_s)
    assert np.abs(K).sum(axis=1).max() < np.max(m.sigma_s / m.sigma_t)
    phi = O.apply(2, m.sigma_t, m.sigma_s, m.f, op=O.OP_A_RAW)
    U, term = phi.copy(), phi.copy()
    for _ in range(400):
        term = K @ term
        U += term
    np.testing.assert_allclose(U, O.lu_solve(2, m.sigma_t, m.sigma_s, phi), rtol=1e-9)


def test_dense_and_matrix_free_apply_agree():
    m = V.heterogeneous_3d(n=6)
    g = np.random.default_rng(0).standard_normal(m.N)
    K = O.k_matrix(3, m.sigma_t, m.sigma_s)
    y = O.apply(3, m.sigma_t, m.sigma_s, g)
    np.testing.assert_allclose(y, K @ g, rtol=1e-12)
    rows = [0, 7, 100, m.N - 1]
    np.testing.assert_allclose(O.apply(3, m.sigma_t, m.sigma_s, g, op=O.OP_I_MINUS_K, rows=rows),
                               (g - K @ g)[rows], rtol=1e-12)


# ----------------------------------------------------------------- sweep

def test_exit_length():
    assert O.exit_length(2, [0.3, 0.6], [1.0, 0.0]) == pytest.approx(0.3)
    assert O.exit_length(2, [0.3, 0.6], [0.0, -1.0]) == pytest.approx(0.4)
    v = np.array([1.0, 1.0]) / math.sqrt(2)
    assert O.exit_length(2, [0.3, 0.6], v) == pytest.approx(0.3 * math.sqrt(2))
    assert O.exit_length(3, [0.5, 0.5, 0.9], [0, 0, -1.0]) == pytest.approx(0.1)


@pytest.mark.parametrize("dim", [2, 3])
def test_sweep_constant_medium_exact(dim):
    # constant sigma and Q: Phi = Q (1 - e^{-sigma L}) / sigma exactly.
    n = 10 if dim == 2 else 6
    st = np.full(n ** dim, 1.7)
    Q = np.full(n ** dim, 0.3)
    dirs = V.directions(dim, 24)
    Phi = O.sweep(dim, st, Q, dirs)
    xs = V.cell_centres(dim, n)
    for m in range(0, 24, 5):
        for j in range(0, n ** dim, 7):
            L = O.exit_length(dim, xs[j], dirs[m])
            assert Phi[m, j] == pytest.approx(0.3 * (1 - math.exp(-1.7 * L)) / 1.7, rel=1e-12)


def test_sweep_vacuum_linear_source():
    # sigma = 0 and a linear cell field Q: the interpolant is Q(clamp(p)) with
    # the clamp to the hull of centres [h/2, 1-h/2]^2, linear except for the
    # kink where the ray crosses into the boundary strip.  Phi is the integral
    # of it along the ray; the h/2-step midpoint rule is exact on every step
    # but the (at most two) kinked ones, error <= |beta|_1 Delta^2.
    n = 12
    h = 1.0 / n
    beta = np.array([0.5, -0.25])
    st = np.zeros(n * n)
    Q = V.linear_field(2, n, 1.0, beta)
    dirs = V.directions(2, 16)
    Phi = O.sweep(2, st, Q, dirs)
    xs = V.cell_centres(2, n)
    for m in range(16):
        for j in range(0, n * n, 11):
            L = O.exit_length(2, xs[j], dirs[m])
            l = (np.arange(200000) + 0.5) / 200000 * L
            p = np.clip(xs[j][None, :] - l[:, None] * dirs[m][None, :], h / 2, 1 - h / 2)
            fine = np.sum(1.0 + p @ beta) * (L / l.size)
            delta = L / O.sweep_steps(n, L)
            assert abs(Phi[m, j] - fine) <= 2 * np.abs(beta).sum() * delta ** 2 + 1e-9


def test_sweep_mean_matches_phi_without_scattering():
    # sigma_s = 0: the angular mean of the sweep of f (Algorithm 1, S.1 (i)-(ii))
    # is phi = A f up to discretisation; the gap shrinks with h.
    gaps = []
    for n in (12, 24):
        m = V.heterogeneous_2d(n=n)
        phi = O.apply(2, m.sigma_t, m.sigma_s, m.f, op=O.OP_A_RAW)
        mean = O.sweep(2, m.sigma_t, m.f, V.directions(2, 720)).mean(axis=0)
        gaps.append(np.linalg.norm(mean - phi) / np.linalg.norm(phi))
    assert gaps[1] < gaps[0] and gaps[1] < 0.05


@pytest.mark.slow
def test_discrete_ordinates_brute_force_matches_vie():
    # Full transport equation by source iteration vs the integral equation:
    # agreement to discretisation level, improving with h.
    gaps = []
    for n in (8, 16):
        st = np.full(n * n, 2.0)
        ss = np.full(n * n, 1.5)
        f = V.gaussian_source(2, n, width=0.15)
        U_do, it = O.do_solve(2, st, ss, f, V.directions(2, 720), tol=1e-10)
        phi = O.apply(2, st, ss, f, op=O.OP_A_RAW)
        U_vie = O.lu_solve(2, st, ss, phi)
        gaps.append(np.linalg.norm(U_do - U_vie) / np.linalg.norm(U_vie))
    assert gaps[1] < gaps[0] and gaps[1] < 0.08


def test_gmres_dense_branch_equals_matrix_free_and_lu():
    # or_gmres with the dense (I - K) (its `dense` argument) against the
    # matrix-free branch and numpy's LU: one Krylov iteration, two operators
    m = V.heterogeneous_2d(n=12)
    phi = O.apply(2, m.sigma_t, m.sigma_s, m.f, op=O.OP_A_RAW)
    IK = np.eye(m.N) - O.k_matrix(2, m.sigma_t, m.sigma_s)
    Ud, itd, rrd, okd = O.gmres(2, m.sigma_t, m.sigma_s, phi, rtol=1e-12, dense=IK)
    Um, itm, rrm, okm = O.gmres(2, m.sigma_t, m.sigma_s, phi, rtol=1e-12)
    assert okd and okm and rrd <= 1e-12 and itd == itm
    U_lu = np.linalg.solve(IK, phi)
    assert np.linalg.norm(Ud - U_lu) <= 1e-11 * np.linalg.norm(U_lu)
    assert np.linalg.norm(Ud - Um) <= 1e-11 * np.linalg.norm(U_lu)
    # a different dense operator gives its own solution (the argument is used)
    Ud2, _, _, ok2 = O.gmres(2, m.sigma_t, m.sigma_s, phi, rtol=1e-12, dense=2.0 * IK)
    assert ok2 and np.linalg.norm(Ud2 - 0.5 * U_lu) <= 1e-11 * np.linalg.norm(U_lu)
