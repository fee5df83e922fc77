"""What the trained network gains: FGMRES with the learned preconditioner against
plain GMRES, both with the assembled operator, on held-out 256^2 media of the
strongly scattering family the network was trained on (at 128^2)."""
import os

import numpy as np
import pytest

import vie_synth as V

torch = pytest.importorskip("torch")
import paper_1610_00835_gb300 as P  # noqa: E402
from gpu_util import host, rel_l2  # noqa: E402

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "paper_1610_00835_gb300", "data", "unet_l4_c32.bin")


@pytest.mark.parametrize("seed", [9004, 9005])
def test_trained_network_halves_iterations_on_hard_media(seed):
    net = P.vie_unet_create(4, 32)
    P.vie_unet_load(net, WEIGHTS)
    m = V.diffusive_training_medium(256, seed)
    h = P.vie_create(2, 256, m.sigma_t, m.sigma_s)
    P.vie_assemble(h, P.VIE_OPERATOR_BF16X3)
    f = torch.as_tensor(m.f, dtype=torch.float64, device="cuda:0")
    U0 = torch.empty_like(f)
    plain = P.vie_solve_gmres(h, f, U0, rtol=1e-6, restart=128)
    P.vie_set_preconditioner(h, net, 5.0)
    U1 = torch.empty_like(f)
    learned = P.vie_solve_gmres(h, f, U1, rtol=1e-6, restart=128)
    assert plain["converged"] and learned["converged"] and not learned["fell_back"]
    assert learned["iters"] <= 0.75 * plain["iters"], (plain["iters"], learned["iters"])
    assert rel_l2(host(U1), host(U0)) < 1e-5


@pytest.mark.parametrize("seed", [9004, 9006])
def test_learned_solution_at_256_matches_oracle_on_sampled_rows(seed):
    # the learned FGMRES solution at 256^2 (65536 unknowns) is judged by the FP64
    # oracle itself: its residual phi_j - (U_j - (K U)_j) on sampled rows is at
    # the level of the 1e-6 tolerance, whatever the preconditioner did.
    import oracle as O
    net = P.vie_unet_create(4, 32)
    P.vie_unet_load(net, WEIGHTS)
    m = V.diffusive_training_medium(256, seed)
    h = P.vie_create(2, 256, m.sigma_t, m.sigma_s)
    P.vie_assemble(h, P.VIE_OPERATOR_BF16X3)
    P.vie_set_preconditioner(h, net, 5.0)
    f = torch.as_tensor(m.f, dtype=torch.float64, device="cuda:0")
    U = torch.empty_like(f)
    rep = P.vie_solve_gmres(h, f, U, rtol=1e-6, restart=128)
    assert rep["converged"] and rep["relres"] <= 1e-6 and rep["precond_iters"] >= 1
    u = host(U)
    rows = np.unique(np.random.default_rng(seed).choice(m.N, 32, replace=False))
    phi = O.apply(2, m.sigma_t, m.sigma_s, m.f, op=O.OP_A_RAW, rows=rows)
    lhs = O.apply(2, m.sigma_t, m.sigma_s, u, op=O.OP_I_MINUS_K, rows=rows)
    assert np.linalg.norm(phi - lhs) <= 1e-5 * np.linalg.norm(phi)
    P.vie_destroy(h)
