"""Parity of the step-two sweep (Algorithm 1, S.3) with the oracle."""
import numpy as np
import pytest

import oracle as O
import vie_synth as V

torch = pytest.importorskip("torch")
import paper_1610_00835_gb300 as P  # noqa: E402
from gpu_util import dev, host, rel_l2  # noqa: E402

pytestmark = pytest.mark.gpu


def run_sweep(h, U, f, dirs32):
    Phi = torch.empty(dirs32.shape[0] * h.N, dtype=torch.float32, device="cuda:0")
    P.ert_sweep(h, dev(U), dev(f), dev(dirs32, torch.float32), Phi)
    return host(Phi).reshape(dirs32.shape[0], h.N)


@pytest.mark.parametrize("dim,n,M", [(2, 1, 4), (2, 3, 8), (2, 16, 32), (2, 29, 7), (3, 2, 6),
                                     (3, 8, 16)])
def test_sweep_matches_oracle(dim, n, M):
    m = V.heterogeneous_2d(n=n) if dim == 2 else V.heterogeneous_3d(n=n)
    h = P.vie_create(dim, n, m.sigma_t, m.sigma_s)
    U = np.abs(np.random.default_rng(n).standard_normal(m.N))
    dirs32 = V.directions(dim, M).astype(np.float32)
    got = run_sweep(h, U, m.f, dirs32)
    Q = m.sigma_s * U + m.f
    want = O.sweep(dim, m.sigma_t, Q, dirs32.astype(np.float64))
    assert rel_l2(got, want) < 1e-5


def test_axis_aligned_directions_step_count():
    # exact axis directions put L * 2n on integers: both sides must agree
    n = 12
    m = V.heterogeneous_2d(n=n)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    dirs32 = np.array([[1, 0], [0, 1], [-1, 0], [0, -1]], dtype=np.float32)
    got = run_sweep(h, np.ones(m.N), m.f, dirs32)
    want = O.sweep(2, m.sigma_t, m.sigma_s + m.f, dirs32.astype(np.float64))
    assert rel_l2(got, want) < 1e-5


def test_config3_sweep_sampled_rays():
    m = V.heterogeneous_3d()
    h = P.vie_create(3, m.n, m.sigma_t, m.sigma_s)
    U = torch.empty(m.N, dtype=torch.float64, device="cuda:0")
    P.vie_solve_gmres(h, dev(m.f), U, rtol=1e-6)
    dirs32 = V.fibonacci_directions(128).astype(np.float32)
    got = run_sweep(h, host(U), m.f, dirs32)
    # oracle on a sample: 8 directions, all cells
    sel = np.arange(0, 128, 16)
    Q = m.sigma_s * host(U) + m.f
    want = O.sweep(3, m.sigma_t, Q, dirs32[sel].astype(np.float64))
    assert rel_l2(got[sel], want) < 1e-5
    # the angular mean of Phi recovers U up to discretisation (Algorithm 1 consistency)
    assert rel_l2(got.mean(axis=0), host(U)) < 0.1
