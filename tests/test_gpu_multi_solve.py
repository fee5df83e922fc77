"""Several sources on one medium solved together (vie_gmres_opts.nrhs > 1):
lockstep GMRES / FGMRES whose operator applies go through one multi-RHS
product per Arnoldi step (Algorithm 1, S.2 for each source)."""
import numpy as np
import pytest

import oracle as O
import vie_synth as V

torch = pytest.importorskip("torch")
import paper_1610_00835_gb300 as P  # noqa: E402
from gpu_util import dev, host, rel_l2  # noqa: E402

pytestmark = pytest.mark.gpu


def _sources(m, R, seed):
    return V.bump_sources(2, m.n, R, seed=seed)


def _lu(m, F):
    K = O.k_matrix(2, m.sigma_t, m.sigma_s)
    A = K / np.where(m.sigma_s > 0, m.sigma_s, 1.0)[None, :]
    IK = np.eye(m.N) - K
    return np.stack([np.linalg.solve(IK, A @ f) for f in F])


def test_lockstep_on_the_fly_equals_single_solves_bitwise():
    # with the on-the-fly operator every column is applied by the single
    # apply, and the batched Krylov kernels do the single kernels' arithmetic
    # in the same order: each lockstep solution equals its own single solve
    n, R = 24, 4
    m = V.heterogeneous_2d(n=n)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    F = _sources(m, R, seed=71)
    U = torch.empty(R * m.N, dtype=torch.float64, device="cuda:0")
    reps = P.vie_solve_gmres(h, dev(F.ravel()), U, rtol=1e-9, restart=8, nrhs=R)
    assert len(reps) == R and all(r["converged"] for r in reps)
    got = host(U).reshape(R, m.N)
    for r in range(R):
        u1 = torch.empty(m.N, dtype=torch.float64, device="cuda:0")
        one = P.vie_solve_gmres(h, dev(F[r]), u1, rtol=1e-9, restart=8)
        np.testing.assert_array_equal(got[r], host(u1))
        assert one["iters"] == reps[r]["iters"] and one["restarts"] == reps[r]["restarts"]


@pytest.mark.parametrize("R", [2, 5, 17])
def test_lockstep_tensor_core_operator_matches_lu(R):
    n = 20
    m = V.heterogeneous_2d(n=n, seed=8100 + R)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    P.vie_assemble(h, P.VIE_OPERATOR_BF16X3)
    F = _sources(m, R, seed=300 + R)
    F[R // 2] = 0.0                           # a zero source: U = 0 at once
    U = np.zeros(R * m.N)                     # host pointers
    # 1e-7: the product rounds its FP64 input to FP32 (2^-24 per element, not
    # a linear map), which puts the residual it can reach near 1e-8
    reps = P.vie_solve_gmres(h, F.ravel(), U, rtol=1e-7, nrhs=R)
    want = _lu(m, F)
    for r in range(R):
        assert reps[r]["converged"] and reps[r]["relres"] <= 1e-7
        if r == R // 2:
            assert np.all(U[r * m.N:(r + 1) * m.N] == 0) and reps[r]["iters"] == 0
        else:
            assert rel_l2(U[r * m.N:(r + 1) * m.N], want[r]) < 1e-5


@pytest.mark.parametrize("pre", ["learned", "fft", "diffusion"])
def test_lockstep_flexible_gmres_with_each_preconditioner(pre):
    n, R = 32, 3
    m = V.heterogeneous_2d(n=n, seed=8201)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    P.vie_assemble(h, P.VIE_OPERATOR_BF16X3)
    if pre == "learned":
        net = P.vie_unet_create(4, 8, seed=9)
        P.vie_set_preconditioner(h, net)
    elif pre == "fft":
        P.vie_set_fft_preconditioner(h, True)
    else:
        P.vie_set_diffusion_preconditioner(h, True)
    F = _sources(m, R, seed=400)
    U = torch.empty(R * m.N, dtype=torch.float64, device="cuda:0")
    reps = P.vie_solve_gmres(h, dev(F.ravel()), U, rtol=1e-7, nrhs=R)
    want = _lu(m, F)
    got = host(U).reshape(R, m.N)
    for r in range(R):
        assert reps[r]["converged"] and reps[r]["precond_iters"] >= 1
        assert rel_l2(got[r], want[r]) < 1e-5


def test_lockstep_restarts_and_maxit_per_source():
    n, R = 16, 3
    m = V.heterogeneous_2d(n=n, seed=8301)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    F = _sources(m, R, seed=500)
    U = np.zeros(R * m.N)
    reps = P.vie_solve_gmres(h, F.ravel(), U, rtol=1e-14, restart=3, maxit=5, nrhs=R,
                             raise_on_nonconvergence=False)
    for r in reps:
        assert not r["converged"] and r["iters"] == 5 and r["restarts"] == 2 and r["relres"] > 0
    with pytest.raises(P.VieError):
        P.vie_solve_gmres(h, F.ravel(), U, rtol=1e-14, restart=3, maxit=5, nrhs=R)
    reps = P.vie_solve_gmres(h, F.ravel(), U, rtol=1e-8, restart=3, nrhs=R)
    want = _lu(m, F)
    for r in range(R):
        assert reps[r]["converged"] and reps[r]["restarts"] >= 2
        assert rel_l2(U[r * m.N:(r + 1) * m.N], want[r]) < 1e-5


def test_config4_64_sources_at_128_sampled_oracle_residual():
    # the 64 seeded bump sources on the 128^2 bench medium, solved together to
    # 1e-6 with the assembled BF16 hi/lo operator (one tensor-core product of
    # 64 columns per Arnoldi step); every source's solution is judged by the
    # FP64 oracle's own residual on sampled rows
    m = V.heterogeneous_2d(n=128, seed=V.seed_for(2, 0))
    R = 64
    F = V.bump_sources(2, 128, R, seed=V.seed_for(4))
    h = P.vie_create(2, 128, m.sigma_t, m.sigma_s)
    P.vie_assemble(h, P.VIE_OPERATOR_BF16X3)
    U = torch.empty(R * m.N, dtype=torch.float64, device="cuda:0")
    reps = P.vie_solve_gmres(h, dev(F.ravel()), U, rtol=1e-6, nrhs=R)
    got = host(U).reshape(R, m.N)
    rng = np.random.default_rng(64)
    for r in range(R):
        assert reps[r]["converged"] and reps[r]["relres"] <= 1e-6
        rows = np.unique(rng.choice(m.N, 12, replace=False))
        phi = O.apply(2, m.sigma_t, m.sigma_s, F[r], op=O.OP_A_RAW, rows=rows)
        lhs = O.apply(2, m.sigma_t, m.sigma_s, got[r], op=O.OP_I_MINUS_K, rows=rows)
        assert np.linalg.norm(phi - lhs) <= 1e-5 * np.linalg.norm(phi), r
    # the same sources one at a time give the same solutions to the tolerance
    u1 = torch.empty(m.N, dtype=torch.float64, device="cuda:0")
    for r in (0, 31, 63):
        P.vie_solve_gmres(h, dev(F[r]), u1, rtol=1e-6)
        assert rel_l2(got[r], host(u1)) < 5e-6
