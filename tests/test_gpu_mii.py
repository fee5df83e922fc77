"""Approach M-ii (Section 3.2, Remark REM: NEW KERNEL) on the GPU against the
FP64 oracle's M-ii, element by element, through the C ABI."""
import math

import numpy as np
import pytest

import oracle as O
import vie_synth as V

torch = pytest.importorskip("torch")
import paper_1610_00835_gb300 as P  # noqa: E402
from gpu_util import dev, host, rel_l2  # noqa: E402

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5   # relative L2 bar for FP32 kernel tiles
MII = O.TAU_MARCH | O.DISC_MII
OPS = (P.VIE_OP_K_SIGMA_S, P.VIE_OP_I_MINUS_K, P.VIE_OP_A_RAW)


def gpu_apply(h, op, g, nrhs=1):
    y = torch.empty(nrhs * h.N, dtype=torch.float64, device="cuda:0")
    P.vie_apply(h, op, dev(g), y, nrhs)
    return host(y)


def mii_handle(m, n, **kw):
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s, disc=P.VIE_DISC_MII, **kw)
    assert P.vie_get_kernel(h) == P.VIE_KERNEL_DISPLACEMENT
    return h


@pytest.mark.parametrize("n", [2, 3, 9, 24, 37, 64])
def test_mii_apply_all_rows(n):
    # several warp units per displacement plus ragged edges; n = 2, 3 degenerate
    m = V.bump_medium(2, n, 4, 0.9, seed=4700 + n)
    h = mii_handle(m, n)
    g = m.f + 0.05 * np.random.default_rng(n).standard_normal(m.N)
    for op in OPS:
        want = O.apply(2, m.sigma_t, m.sigma_s, g, op=op, mode=MII)
        assert rel_l2(gpu_apply(h, op, g), want) < FP32_TOL


@pytest.mark.parametrize("n", [128, 233, 256])
def test_mii_apply_full_size_sampled_rows(n):
    m = V.bump_medium(2, n, 4, 0.9, seed=4800 + n)
    h = mii_handle(m, n)
    g = m.f + 0.05 * np.random.default_rng(n).standard_normal(m.N)
    got = gpu_apply(h, P.VIE_OP_K_SIGMA_S, g)
    rows = np.unique(np.concatenate([np.random.default_rng(n + 1).choice(m.N, 12, replace=False),
                                     [0, n - 1, m.N - n, m.N - 1, m.N // 2]]))
    want = O.apply(2, m.sigma_t, m.sigma_s, g, mode=MII, rows=rows)
    assert rel_l2(got[rows], want) < FP32_TOL
    again = gpu_apply(h, P.VIE_OP_K_SIGMA_S, g)
    np.testing.assert_array_equal(again, got)   # exact fixed-point sums


def test_mii_diagonal_is_the_cell_integral_at_zero():
    # A_jj = (1/2pi) int_T |z|^{-1} dz = (1/2pi) 4 h ln(1 + sqrt 2) for every cell
    n = 40
    m = V.bump_medium(2, n, 4, 0.9, seed=4901)
    h = mii_handle(m, n)
    d = np.empty(m.N)
    P.vie_get_diagonal(h, d)
    want = 4 / n * math.log(1 + math.sqrt(2)) / (2 * math.pi)
    np.testing.assert_allclose(d, want, rtol=1e-14, atol=0)


def test_mii_gmres_matches_oracle_lu():
    n = 24
    m = V.bump_medium(2, n, 4, 0.9, seed=4902)
    h = mii_handle(m, n)
    U = torch.empty(m.N, dtype=torch.float64, device="cuda:0")
    # 1e-8, as for M-iii: the FP32 rounding of the sources puts the residual
    # an FP32-tile operator can reach near 1e-9
    rep = P.vie_solve_gmres(h, dev(m.f), U, rtol=1e-8)
    assert rep["converged"]
    phi = O.apply(2, m.sigma_t, m.sigma_s, m.f, op=O.OP_A_RAW, mode=MII)
    U_lu = O.lu_solve(2, m.sigma_t, m.sigma_s, phi, mode=MII)
    assert rel_l2(host(U), U_lu) < FP32_TOL


@pytest.mark.parametrize("n", [37, 128])
def test_mii_assembled_operators(n):
    # the pair weights are the on-the-fly kernel's (bitwise equal applies); the
    # symmetric blocks and dense K carry the same weights and the M-ii diagonal
    m = V.bump_medium(2, n, 4, 0.9, seed=4903 + n)
    h = mii_handle(m, n)
    g = m.f + 0.05 * np.random.default_rng(n).standard_normal(m.N)
    otf = [gpu_apply(h, op, g) for op in OPS]
    P.vie_assemble(h, P.VIE_OPERATOR_PAIRS32)
    for op, want in zip(OPS, otf):
        np.testing.assert_array_equal(gpu_apply(h, op, g), want)
    rows = np.unique(np.concatenate([np.random.default_rng(n + 2).choice(m.N, 10, replace=False), [0]]))
    want = O.apply(2, m.sigma_t, m.sigma_s, g, mode=MII, rows=rows)
    for mode in (P.VIE_OPERATOR_SYM32, P.VIE_OPERATOR_FP32, P.VIE_OPERATOR_BF16X3):
        P.vie_assemble(h, mode)
        got = gpu_apply(h, P.VIE_OP_K_SIGMA_S, g)
        assert rel_l2(got[rows], want) < FP32_TOL
        assert rel_l2(got, otf[0]) < 2e-6


def test_mii_beats_miii_on_the_gaussian_weight_closed_form():
    # homogeneous sigma (the march of a constant field is exact): the row sum of
    # A against a Gaussian about the centre cell has the closed form
    # w sqrt(pi/2) e^{sigma^2 w^2/2} erfc(sigma w/sqrt 2); M-ii's error is
    # O(h^2 (1 + log h)), M-iii's O(h) (Eq. EQ: ERROR)
    n, sigma, w = 161, 1.1, 0.08
    want = w * math.sqrt(math.pi / 2) * math.exp(sigma ** 2 * w ** 2 / 2) * math.erfc(
        sigma * w / math.sqrt(2))
    st = np.full(n * n, sigma)
    xs = V.cell_centres(2, n)
    c = n * n // 2
    g = np.exp(-np.sum((xs - xs[c]) ** 2, axis=1) / (2 * w * w))
    err = {}
    for disc in (P.VIE_DISC_MIII, P.VIE_DISC_MII):
        h = P.vie_create(2, n, st, st, disc=disc)
        assert P.vie_get_kernel(h) == P.VIE_KERNEL_DISPLACEMENT
        err[disc] = abs(gpu_apply(h, P.VIE_OP_A_RAW, g)[c] - want) / want
    assert err[P.VIE_DISC_MII] < err[P.VIE_DISC_MIII] / 8
    assert err[P.VIE_DISC_MII] < 7 / n ** 2


@pytest.mark.parametrize("case", ["3d", "fp64", "symmetric", "n259", "n1", "closed_tau"])
def test_mii_outside_its_combination_is_unsupported(case):
    kw = {"disc": P.VIE_DISC_MII}
    if case == "3d":
        m = V.heterogeneous_3d(n=5)
        args = (3, 5, m.sigma_t, m.sigma_s)
    else:
        n = {"n259": 259, "n1": 1}.get(case, 16)
        m = V.bump_medium(2, n, 2, 0.9, seed=4904)
        args = (2, n, m.sigma_t, m.sigma_s)
        if case == "fp64":
            kw["precision"] = P.VIE_PREC_FP64
        elif case == "symmetric":
            kw["kernel"] = P.VIE_KERNEL_SYMMETRIC
        elif case == "closed_tau":
            args = (2, n, np.full(n * n, 1.3), np.full(n * n, 1.0))
            kw["tau_mode"] = P.VIE_TAU_CLOSED
    with pytest.raises(P.VieError) as e:
        P.vie_create(*args, **kw)
    assert e.value.status == P.vie.VIE_ERR_UNSUPPORTED
