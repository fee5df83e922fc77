"""Pins of the oracle's diffusion preconditioner (Section 4.4, Eq. EQ:DA):
the finite-volume operator against a manufactured solution of the Robin
problem, the V-cycle against the sparse direct solve, and the
diffusion-synthetic correction against the transport operator in the regime
where the diffusion approximation holds."""
import math

import numpy as np

import oracle as O
import vie_synth as V
from oracle import diffusion as Dm


def test_operator_is_symmetric_positive_definite():
    n = 8
    m = V.bump_medium(2, n, 3, 0.9, seed=61)
    D = Dm.operator(*Dm.coefficients(m.sigma_t, m.sigma_s, n)).toarray()
    np.testing.assert_allclose(D, D.T, rtol=1e-14, atol=0)
    assert np.min(np.linalg.eigvalsh(D)) > 0


def test_manufactured_robin_solution_second_order():
    # U = g(x) g(y), g(t) = 1 + t (1 - t) / l, satisfies U + l dU/dn = 0 on the
    # whole boundary (constant mu, l = 2 / (d mu)); f = -kappa Lap U + mu_a U
    mu, mus = 3.0, 2.7
    ell, kap = 2.0 / (2 * mu), 1.0 / (2 * mu)
    errs = []
    for n in (16, 32, 64):
        x = (np.arange(n) + 0.5) / n
        g = 1 + x * (1 - x) / ell
        X, Y = np.meshgrid(g, g)
        U = X * Y
        f = -kap * (-2 / ell) * (X + Y) + (mu - mus) * U
        Uh = Dm.solve(np.full(n * n, mu), np.full(n * n, mus), f.ravel(), n)
        errs.append(np.max(np.abs(Uh - U.ravel())) / np.max(U))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 1.9
    assert errs[-1] < 1e-4


def test_vcycles_converge_to_the_direct_solve():
    n = 64
    m = V.bump_medium(2, n, 4, 0.9, seed=62)
    mu, mu_a = Dm.coefficients(m.sigma_t, m.sigma_s, n)
    levels = Dm.hierarchy(mu, mu_a)
    assert [lv[1] for lv in levels] == [64, 32, 16, 8]
    f = np.random.default_rng(1).standard_normal(n * n)
    exact = Dm.solve(m.sigma_t, m.sigma_s, f, n)
    u = np.zeros(n * n)
    errs = []
    for _ in range(8):
        u += Dm.vcycle(levels, f - levels[0][0] @ u)
        errs.append(np.linalg.norm(u - exact) / np.linalg.norm(exact))
    assert max(errs[i + 1] / errs[i] for i in range(len(errs) - 1)) < 0.15
    assert errs[-1] < 1e-8


def test_diffusion_correction_in_the_diffusive_regime():
    # optically thin cells (mu h = 0.08), strong scattering: K barely reduces a
    # smooth residual, the preconditioned operator (I - K) M nearly keeps it
    n = 64
    st, ss = np.full(n * n, 5.0), np.full(n * n, 4.9)
    xs = V.cell_centres(2, n)
    r = np.exp(-np.sum((xs - 0.5) ** 2, axis=1) / (2 * 0.2 ** 2))
    Kr = r - O.apply(2, st, ss, r, op=O.OP_I_MINUS_K, mode=O.TAU_CLOSED)
    z = Dm.precondition(r, st, ss, n)
    y = O.apply(2, st, ss, z, op=O.OP_I_MINUS_K, mode=O.TAU_CLOSED)
    assert np.linalg.norm(Kr) / np.linalg.norm(r) > 0.7
    assert np.linalg.norm(y - r) / np.linalg.norm(r) < 0.3
