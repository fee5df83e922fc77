"""Pins of the oracle's FFT preconditioner (Section 4.4, Eqs. EQ: FFT and
EQ:SOL FFT) against its definition: the torus kernel is the homogeneous
medium's matrix A, and the DFT inversion equals a dense solve of the periodic
operator."""
import numpy as np
import pytest

import oracle as O
import vie_synth as V
from oracle import fft_precond as F


@pytest.mark.parametrize("mii", [False, True])
def test_torus_kernel_is_the_homogeneous_matrix(mii):
    # W~ at every displacement inside the grid equals A_jk of the homogeneous
    # medium (closed-form tau) from the pinned oracle entry
    n, mu = 6, 3.7
    st = np.full(n * n, mu)
    m = F.grid_size(n)
    W = F.kernel_on_torus(n, mu, m, mii)
    mode = O.TAU_CLOSED | (O.DISC_MII if mii else 0)
    j = 2 + n * 3
    for k in range(n * n):
        dx, dy = k % n - j % n, k // n - j // n
        assert W[dy % m, dx % m] == pytest.approx(O.entry(2, st, j, k, mode=mode), rel=1e-13)


@pytest.mark.parametrize("n,mii", [(3, False), (4, False), (5, False), (4, True), (5, True)])
def test_dft_inversion_equals_dense_periodic_solve(n, mii):
    # the periodic operator C = I - mu_s W~ (circulant on the m x m torus) as a
    # dense matrix, solved with LAPACK for the zero-extended b, then restricted
    mu, mu_s = 2.3, 2.0
    m = F.grid_size(n)
    W = F.kernel_on_torus(n, mu, m, mii)
    C = np.eye(m * m)
    for p in range(m * m):
        px, py = p % m, p // m
        for q in range(m * m):
            qx, qy = q % m, q // m
            C[p, q] -= mu_s * W[(qy - py) % m, (qx - px) % m]
    b = np.random.default_rng(n).standard_normal(n * n)
    B = np.zeros((m, m))
    B[:n, :n] = b.reshape(n, n)
    want = np.linalg.solve(C, B.ravel()).reshape(m, m)[:n, :n].ravel()
    np.testing.assert_allclose(F.precondition(b, n, mu, mu_s, mii), want, rtol=1e-11, atol=1e-13)


def test_symbol_is_real_and_positive():
    # W~ is even (W(-D) = W(D)) so its DFT is real; mu_s sum W < mu_s / mu <= 1
    # keeps every eigenvalue of the periodic operator positive
    lam = F.symbol(16, 4.0, 3.9)
    assert np.max(np.abs(lam.imag)) < 1e-12 * np.max(np.abs(lam.real))
    assert np.min(lam.real) > 0


@pytest.mark.parametrize("mu,tol", [(20.2, 1e-3), (10.2, 2e-2)])
def test_homogeneous_medium_is_nearly_inverted(mu, tol):
    # on a homogeneous medium the preconditioner differs from (I - K)^{-1} only
    # through the boundary, which a source far from it hardly reaches
    n = 32 if mu > 15 else 48
    st, ss = np.full(n * n, mu), np.full(n * n, mu - 0.2)
    xs = V.cell_centres(2, n)
    x = np.exp(-np.sum((xs - 0.5) ** 2, axis=1) / (2 * 0.05 ** 2))
    y = O.apply(2, st, ss, x, op=O.OP_I_MINUS_K, mode=O.TAU_CLOSED)
    z = F.precondition_medium(y, st, ss, n)
    assert np.linalg.norm(z - x) / np.linalg.norm(x) < tol
