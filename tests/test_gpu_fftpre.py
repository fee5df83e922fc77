"""The FFT preconditioner (Section 4.4, Eqs. EQ: FFT and EQ:SOL FFT) on the GPU
against the oracle's numpy reference, and inside flexible GMRES."""
import numpy as np
import pytest

import oracle as O
import vie_synth as V
from oracle import fft_precond as F

torch = pytest.importorskip("torch")
import paper_1610_00835_gb300 as P  # noqa: E402
from gpu_util import dev, host, rel_l2  # noqa: E402

pytestmark = pytest.mark.gpu


def _precondition(h, v):
    z = torch.empty(h.N, dtype=torch.float64, device="cuda:0")
    P.vie_fft_precondition(h, dev(v), z)
    return host(z)


@pytest.mark.parametrize("n", [1, 4, 9, 24, 37, 64, 128, 200])
def test_fft_precondition_matches_oracle(n):
    # n = 1 (a 2 x 2 torus) up to a 512 x 512 torus; ragged n between powers of two
    m = V.bump_medium(2, n, 4, 0.9, seed=5100 + n)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    P.vie_set_fft_preconditioner(h)
    xs = V.cell_centres(2, n)
    smooth = np.exp(-np.sum((xs - 0.45) ** 2, axis=1) / (2 * 0.1 ** 2))
    noise = np.random.default_rng(n).standard_normal(m.N)
    for v, tol in ((smooth, 2e-5), (noise, 1e-4)):
        want = F.precondition_medium(v, m.sigma_t, m.sigma_s, n)
        assert rel_l2(_precondition(h, v), want) < tol
    # host pointers give the same bits
    z_host = np.empty(m.N)
    P.vie_fft_precondition(h, noise, z_host)
    np.testing.assert_array_equal(z_host, _precondition(h, noise))


def test_fft_precondition_mii_matches_oracle():
    n = 37
    m = V.bump_medium(2, n, 4, 0.9, seed=5200)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s, disc=P.VIE_DISC_MII)
    P.vie_set_fft_preconditioner(h)
    v = np.random.default_rng(3).standard_normal(m.N)
    want = F.precondition_medium(v, m.sigma_t, m.sigma_s, n, mii=True)
    assert rel_l2(_precondition(h, v), want) < 1e-4


@pytest.mark.parametrize("mu_s", [10.0, 40.0])
def test_fft_fgmres_on_constant_coefficients(mu_s):
    # the setting of the paper's Experiment VI at a smaller grid: mu_a = 0.2,
    # constant mu_s, a source away from the boundary, tolerance 1e-10 (FP64
    # pairs with the closed-form tau, so that the operator is linear to 1e-16)
    n = 64
    st, ss = np.full(n * n, mu_s + 0.2), np.full(n * n, mu_s)
    xs = V.cell_centres(2, n)
    f = np.exp(-np.sum((xs - 0.5) ** 2, axis=1) / (2 * 0.1 ** 2))
    h = P.vie_create(2, n, st, ss, tau_mode=P.VIE_TAU_CLOSED, precision=P.VIE_PREC_FP64)
    U0 = torch.empty(n * n, dtype=torch.float64, device="cuda:0")
    plain = P.vie_solve_gmres(h, dev(f), U0, rtol=1e-10)
    P.vie_set_fft_preconditioner(h)
    U1 = torch.empty_like(U0)
    pre = P.vie_solve_gmres(h, dev(f), U1, rtol=1e-10)
    assert pre["converged"] and not pre["fell_back"] and pre["precond_iters"] > 0
    assert pre["iters"] * 2 <= plain["iters"]
    phi = O.apply(2, st, ss, f, op=O.OP_A_RAW, mode=O.TAU_CLOSED)
    U_lu = O.lu_solve(2, st, ss, phi, mode=O.TAU_CLOSED)
    assert rel_l2(host(U0), U_lu) < 1e-8
    assert rel_l2(host(U1), U_lu) < 1e-8
    P.vie_set_fft_preconditioner(h, False)
    again = P.vie_solve_gmres(h, dev(f), U1, rtol=1e-10)
    assert again["precond_iters"] == 0 and again["iters"] == plain["iters"]


def test_fft_and_learned_preconditioners_replace_each_other():
    n = 32
    m = V.bump_medium(2, n, 4, 0.9, seed=5300)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    net = P.vie_unet_create(2, 32, seed=1)
    P.vie_set_preconditioner(h, net)
    P.vie_set_fft_preconditioner(h)           # replaces the network
    U = torch.empty(m.N, dtype=torch.float64, device="cuda:0")
    rep = P.vie_solve_gmres(h, dev(m.f), U, rtol=1e-8)
    assert rep["converged"] and rep["precond_iters"] > 0
    z = _precondition(h, m.f)
    assert rel_l2(z, F.precondition_medium(m.f, m.sigma_t, m.sigma_s, n)) < 2e-5
    P.vie_set_preconditioner(h, net)          # replaces the FFT preconditioner
    with pytest.raises(P.VieError) as e:
        _precondition(h, m.f)
    assert e.value.status == P.vie.VIE_ERR_INVALID_ARG
    P.vie_set_preconditioner(h, None)
    P.vie_unet_destroy(net)


def test_fft_preconditioner_invalid_uses():
    m3 = V.heterogeneous_3d(n=5)
    h3 = P.vie_create(3, 5, m3.sigma_t, m3.sigma_s)
    with pytest.raises(P.VieError) as e:
        P.vie_set_fft_preconditioner(h3)
    assert e.value.status == P.vie.VIE_ERR_INVALID_ARG
    n = 16
    st = np.full(n * n, 1.0)
    h = P.vie_create(2, n, st, 5.0 * st)     # mean sigma_s far above sigma_t
    with pytest.raises(P.VieError) as e:
        P.vie_set_fft_preconditioner(h)
    assert e.value.status == P.vie.VIE_ERR_INVALID_ARG
    with pytest.raises(P.VieError) as e:
        _precondition(h, np.ones(n * n))
    assert e.value.status == P.vie.VIE_ERR_INVALID_ARG
