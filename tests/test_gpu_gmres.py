"""GMRES on the GPU (FP64 Krylov) against the oracle's solution."""
import numpy as np
import pytest

import oracle as O
import vie_synth as V

torch = pytest.importorskip("torch")
import paper_1610_00835_gb300 as P  # noqa: E402
from gpu_util import dev, host, rel_l2  # noqa: E402

pytestmark = pytest.mark.gpu


def test_config1_fp64_gmres_to_1e10():
    m = V.homogeneous_medium(2, 32, 1.1, 1.0)
    h = P.vie_create(2, 32, m.sigma_t, m.sigma_s, tau_mode=P.VIE_TAU_CLOSED,
                     precision=P.VIE_PREC_FP64)
    U = torch.empty(m.N, dtype=torch.float64, device="cuda:0")
    rep = P.vie_solve_gmres(h, dev(m.f), U, rtol=1e-10)
    assert rep["converged"] and rep["relres"] <= 1e-10
    phi = O.apply(2, m.sigma_t, m.sigma_s, m.f, op=O.OP_A_RAW, mode=O.TAU_CLOSED)
    U_lu = O.lu_solve(2, m.sigma_t, m.sigma_s, phi, mode=O.TAU_CLOSED)
    assert rel_l2(host(U), U_lu) < 1e-9


@pytest.mark.parametrize("restart", [64, 5])
def test_fp32_tiles_gmres_matches_lu(restart):
    n = 32
    m = V.heterogeneous_2d(n=n)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    U = np.zeros(m.N)
    rep = P.vie_solve_gmres(h, m.f, U, rtol=1e-8, restart=restart)   # host pointers
    assert rep["converged"] and rep["relres"] <= 1e-8
    if restart == 5:
        assert rep["restarts"] >= 2
    phi = O.apply(2, m.sigma_t, m.sigma_s, m.f, op=O.OP_A_RAW)
    U_lu = O.lu_solve(2, m.sigma_t, m.sigma_s, phi)
    assert rel_l2(U, U_lu) < 1e-5


def test_3d_gmres_matches_lu():
    n = 9
    m = V.heterogeneous_3d(n=n)
    h = P.vie_create(3, n, m.sigma_t, m.sigma_s)
    U = torch.empty(m.N, dtype=torch.float64, device="cuda:0")
    rep = P.vie_solve_gmres(h, dev(m.f), U, rtol=1e-8)
    assert rep["converged"]
    phi = O.apply(3, m.sigma_t, m.sigma_s, m.f, op=O.OP_A_RAW)
    assert rel_l2(host(U), O.lu_solve(3, m.sigma_t, m.sigma_s, phi)) < 1e-5


def test_sigma_s_zero_returns_phi():
    n = 20
    m = V.heterogeneous_2d(n=n)
    ss = np.zeros(m.N)
    h = P.vie_create(2, n, m.sigma_t, ss)
    U = np.zeros(m.N)
    rep = P.vie_solve_gmres(h, m.f, U, rtol=1e-12)
    assert rep["iters"] <= 1
    phi = O.apply(2, m.sigma_t, ss, m.f, op=O.OP_A_RAW)
    assert rel_l2(U, phi) < 1e-5


def test_not_converged_reports():
    m = V.heterogeneous_2d(n=16)
    h = P.vie_create(2, 16, m.sigma_t, m.sigma_s)
    U = np.zeros(m.N)
    rep = P.vie_solve_gmres(h, m.f, U, rtol=1e-14, maxit=2, raise_on_nonconvergence=False)
    assert rep["converged"] == 0 and rep["iters"] == 2 and rep["relres"] > 1e-14
    with pytest.raises(P.VieError):
        P.vie_solve_gmres(h, m.f, U, rtol=1e-14, maxit=2)


def test_zero_source():
    m = V.heterogeneous_2d(n=10)
    h = P.vie_create(2, 10, m.sigma_t, m.sigma_s)
    U = np.ones(m.N)
    rep = P.vie_solve_gmres(h, np.zeros(m.N), U)
    assert rep["converged"] and np.all(U == 0)


def test_config2_full_size_solve_sampled_residual():
    # Property at full size: the oracle's own residual of the GPU solution on
    # sampled rows, r_j = phi_j - (U_j - (K U)_j), is at the 1e-6 level.
    m = V.heterogeneous_2d()
    h = P.vie_create(2, m.n, m.sigma_t, m.sigma_s)
    U = torch.empty(m.N, dtype=torch.float64, device="cuda:0")
    rep = P.vie_solve_gmres(h, dev(m.f), U, rtol=1e-6)
    assert rep["converged"] and rep["relres"] <= 1e-6
    u = host(U)
    rows = np.unique(np.random.default_rng(5).choice(m.N, 24, replace=False))
    phi = O.apply(2, m.sigma_t, m.sigma_s, m.f, op=O.OP_A_RAW, rows=rows)
    lhs = O.apply(2, m.sigma_t, m.sigma_s, u, op=O.OP_I_MINUS_K, rows=rows)
    assert np.max(np.abs(phi - lhs)) <= 2e-5 * np.max(np.abs(phi))


def test_bench_medium_solution_matches_oracle_solution():
    # the benchmark's solve (128^2, seed 2000) against the FP64 oracle's U
    # stored by tests/golden/make_bench_solution.py: plain on-the-fly GMRES and
    # the assembled BF16 hi/lo operator
    import os
    U_or = np.load(os.path.join(os.path.dirname(__file__), "golden", "bench_U_2d_128.npy"))
    m = V.heterogeneous_2d(n=128, seed=V.seed_for(2, 0))
    h = P.vie_create(2, 128, m.sigma_t, m.sigma_s)
    U = torch.empty(m.N, dtype=torch.float64, device="cuda:0")
    rep = P.vie_solve_gmres(h, dev(m.f), U, rtol=1e-8)
    assert rep["converged"]
    assert rel_l2(host(U), U_or) < 1e-5
    for mode in (P.VIE_OPERATOR_BF16X3, P.VIE_OPERATOR_PAIRS32, P.VIE_OPERATOR_SYM32):
        P.vie_assemble(h, mode)
        rep = P.vie_solve_gmres(h, dev(m.f), U, rtol=1e-8)
        assert rep["converged"]
        assert rel_l2(host(U), U_or) < 1e-5


def _sampled_rows(N, count, seed):
    return np.unique(np.random.default_rng(seed).choice(N, count, replace=False))


def _check_sampled_residual(dim, m, h, f_dev, U, rows, rtol):
    """The oracle's own residual r_j = phi_j - (U_j - (K U)_j) of the GPU
    solution on sampled rows, at the level rtol implies, and the GPU's
    operator on those rows equal to the oracle's (Algorithm 1, S.2)."""
    u = host(U)
    phi = O.apply(dim, m.sigma_t, m.sigma_s, m.f, op=O.OP_A_RAW, rows=rows)
    lhs = O.apply(dim, m.sigma_t, m.sigma_s, u, op=O.OP_I_MINUS_K, rows=rows)
    r_or = phi - lhs
    # sampled rows carry the global 2-norm level within a small factor
    assert np.linalg.norm(r_or) <= 10 * rtol * np.linalg.norm(phi), \
        (np.linalg.norm(r_or) / np.linalg.norm(phi))
    # the GPU's own (I - K) U and A f on the same rows: FP32 tiles against FP64
    y = torch.empty_like(U)
    P.vie_apply(h, P.VIE_OP_I_MINUS_K, U, y)
    ph = torch.empty_like(U)
    P.vie_apply(h, P.VIE_OP_A_RAW, f_dev, ph)
    scale = np.abs(u).max()
    assert np.max(np.abs(host(y)[rows] - lhs)) <= 2e-6 * scale
    assert np.max(np.abs(host(ph)[rows] - phi)) <= 2e-6 * np.abs(phi).max()


def test_config3_full_size_solve_sampled_oracle_residual():
    # 32^3 heterogeneous medium (6 bumps, sigma_s = 0.8 sigma_t), S = 64
    # trilinear march, FP32 tiles, FP64 GMRES to 1e-6: the solution that the
    # step-two sweep consumes, checked by the FP64 oracle on sampled rows.
    m = V.heterogeneous_3d()
    assert m.n == 32
    h = P.vie_create(3, m.n, m.sigma_t, m.sigma_s)
    f = dev(m.f)
    U = torch.empty(m.N, dtype=torch.float64, device="cuda:0")
    rep = P.vie_solve_gmres(h, f, U, rtol=1e-6)
    assert rep["converged"] and rep["relres"] <= 1e-6
    _check_sampled_residual(3, m, h, f, U, _sampled_rows(m.N, 32, 33), 1e-6)
    P.vie_destroy(h)
