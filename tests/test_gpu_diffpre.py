"""The diffusion preconditioner (Section 4.4, Eq. EQ:DA) on the GPU against
the oracle's numpy/scipy reference, and inside flexible GMRES."""
import numpy as np
import pytest

import oracle as O
import vie_synth as V
from oracle import diffusion as Dm

torch = pytest.importorskip("torch")
import paper_1610_00835_gb300 as P  # noqa: E402
from gpu_util import dev, host, rel_l2  # noqa: E402

pytestmark = pytest.mark.gpu


def _precondition(h, v):
    z = torch.empty(h.N, dtype=torch.float64, device="cuda:0")
    P.vie_diffusion_precondition(h, dev(v), z)
    return host(z)


@pytest.mark.parametrize("n", [1, 5, 8, 16, 24, 64, 128, 133, 200, 300])
def test_diffusion_precondition_matches_oracle(n):
    # one level (n <= 8 or odd: the coarse solve only), up to five levels
    # (128 -> 8); 200 stops at the odd 25; up to 256 the single-CTA kernel,
    # 300 (300 -> 150 -> 75) the graph of per-phase launches
    m = V.bump_medium(2, n, 4, 0.9, seed=5400 + n)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    P.vie_set_diffusion_preconditioner(h)
    xs = V.cell_centres(2, n)
    smooth = np.exp(-np.sum((xs - 0.45) ** 2, axis=1) / (2 * 0.15 ** 2))
    noise = np.random.default_rng(n).standard_normal(m.N)
    for v in (smooth, noise):
        want = Dm.precondition(v, m.sigma_t, m.sigma_s, n)
        assert rel_l2(_precondition(h, v), want) < 1e-12
    z_host = np.empty(m.N)
    P.vie_diffusion_precondition(h, noise, z_host)
    np.testing.assert_array_equal(z_host, _precondition(h, noise))


def test_diffusion_fgmres_in_the_diffusive_regime():
    # the paper's Experiment V at h = 1/128: mu_a = 0.2, mu_s = 40 (sigma_t h =
    # 0.31), FP64 pairs with the closed-form tau to 1e-10
    n = 128
    st, ss = np.full(n * n, 40.2), np.full(n * n, 40.0)
    xs = V.cell_centres(2, n)
    f = np.exp(-np.sum((xs - 0.5) ** 2, axis=1) / (2 * 0.1 ** 2))
    h = P.vie_create(2, n, st, ss, tau_mode=P.VIE_TAU_CLOSED, precision=P.VIE_PREC_FP64)
    U0 = torch.empty(n * n, dtype=torch.float64, device="cuda:0")
    plain = P.vie_solve_gmres(h, dev(f), U0, rtol=1e-10)
    P.vie_set_diffusion_preconditioner(h)
    U1 = torch.empty_like(U0)
    pre = P.vie_solve_gmres(h, dev(f), U1, rtol=1e-10)
    assert pre["converged"] and not pre["fell_back"] and pre["precond_iters"] > 0
    assert pre["iters"] * 2 <= plain["iters"]
    assert rel_l2(host(U1), host(U0)) < 1e-8


def test_preconditioners_replace_each_other():
    n = 32
    m = V.bump_medium(2, n, 4, 0.9, seed=5500)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    P.vie_set_fft_preconditioner(h)
    P.vie_set_diffusion_preconditioner(h)     # replaces the FFT preconditioner
    with pytest.raises(P.VieError):
        P.vie_fft_precondition(h, m.f, np.empty(m.N))
    U = torch.empty(m.N, dtype=torch.float64, device="cuda:0")
    rep = P.vie_solve_gmres(h, dev(m.f), U, rtol=1e-6)
    assert rep["converged"] and rep["precond_iters"] > 0
    P.vie_set_fft_preconditioner(h)           # and back
    with pytest.raises(P.VieError) as e:
        _precondition(h, m.f)
    assert e.value.status == P.vie.VIE_ERR_INVALID_ARG
    P.vie_set_fft_preconditioner(h, False)
    rep = P.vie_solve_gmres(h, dev(m.f), U, rtol=1e-6)
    assert rep["precond_iters"] == 0


def test_diffusion_preconditioner_invalid_uses():
    m3 = V.heterogeneous_3d(n=5)
    h3 = P.vie_create(3, 5, m3.sigma_t, m3.sigma_s)
    with pytest.raises(P.VieError) as e:
        P.vie_set_diffusion_preconditioner(h3)
    assert e.value.status == P.vie.VIE_ERR_INVALID_ARG
    n = 12
    st = np.full(n * n, 2.0)
    st[5] = 0.0                                # a void cell: kappa = 1 / (2 sigma_t) undefined
    h = P.vie_create(2, n, st, 0.5 * st)
    with pytest.raises(P.VieError) as e:
        P.vie_set_diffusion_preconditioner(h)
    assert e.value.status == P.vie.VIE_ERR_INVALID_ARG
    with pytest.raises(P.VieError) as e:
        _precondition(h, np.ones(n * n))
    assert e.value.status == P.vie.VIE_ERR_INVALID_ARG
