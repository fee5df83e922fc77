"""The dense 3D operator assembled from the 3D displacement kernel's pair
weights (each unordered pair marched once, then expanded along grid lines),
against the oracle's K, the tile-pair assembler and the on-the-fly apply."""
import numpy as np
import pytest

import oracle as O
import vie_synth as V

torch = pytest.importorskip("torch")
import paper_1610_00835_gb300 as P  # noqa: E402
from gpu_util import dev, host, rel_l2  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _apply(h, op, G, nrhs):
    y = torch.empty(G.size, dtype=torch.float64, device="cuda:0")
    P.vie_apply(h, op, dev(G.ravel()), y, nrhs)
    return host(y).reshape(nrhs, -1)


@pytest.mark.parametrize("mode", [P.VIE_OPERATOR_FP32, P.VIE_OPERATOR_BF16X3, P.VIE_OPERATOR_SYM32])
@pytest.mark.parametrize("n", [2, 3, 5, 8, 11])
def test_3d_assembled_all_rows_against_oracle_k(mode, n):
    m = V.heterogeneous_3d(n=n, seed=300 + n)
    h = P.vie_create(3, n, m.sigma_t, m.sigma_s)
    assert P.vie_get_kernel(h) == P.VIE_KERNEL_DISPLACEMENT
    P.vie_assemble(h, mode)
    rng = np.random.default_rng(n)
    G = np.stack([m.f, rng.standard_normal(m.N), np.ones(m.N)])
    K = O.k_matrix(3, m.sigma_t, m.sigma_s)
    got = _apply(h, P.VIE_OP_K_SIGMA_S, G, 3)
    for r in range(3):
        assert rel_l2(got[r], K @ G[r]) < TOL, r
    # (I - K) g and A g through the same matrix
    g = G[1]
    assert rel_l2(_apply(h, P.VIE_OP_I_MINUS_K, g, 1)[0], g - K @ g) < TOL
    A = O.assemble(3, m.sigma_t)
    assert rel_l2(_apply(h, P.VIE_OP_A_RAW, g, 1)[0], A @ g) < TOL
    P.vie_destroy(h)


@pytest.mark.parametrize("n", [16, 32])
def test_3d_displacement_assembly_matches_tile_pair_assembly(n):
    # the same operator from the two assemblers: the stencil march (grouped
    # samples) and the per-sample march of the symmetric tile-pair kernel
    m = V.heterogeneous_3d(n=n, seed=310 + n)
    G = np.stack([m.f, np.random.default_rng(n).standard_normal(m.N)])
    hd = P.vie_create(3, n, m.sigma_t, m.sigma_s)
    ht = P.vie_create(3, n, m.sigma_t, m.sigma_s, kernel=P.VIE_KERNEL_SYMMETRIC)
    assert P.vie_get_kernel(hd) == P.VIE_KERNEL_DISPLACEMENT
    otf = _apply(hd, P.VIE_OP_K_SIGMA_S, G, 2)
    P.vie_assemble(hd, P.VIE_OPERATOR_FP32)
    P.vie_assemble(ht, P.VIE_OPERATOR_FP32)
    yd = _apply(hd, P.VIE_OP_K_SIGMA_S, G, 2)
    yt = _apply(ht, P.VIE_OP_K_SIGMA_S, G, 2)
    for r in range(2):
        assert rel_l2(yd[r], yt[r]) < TOL, r
        assert rel_l2(yd[r], otf[r]) < 2e-6, r   # the same weights, summed in another order
    # the symmetric blocks of grid-line pairs: the same weights, half the storage
    P.vie_assemble(hd, P.VIE_OPERATOR_SYM32)
    ys = _apply(hd, P.VIE_OP_K_SIGMA_S, G, 2)
    for r in range(2):
        assert rel_l2(ys[r], yd[r]) < 2e-6, r
    ys2 = _apply(hd, P.VIE_OP_K_SIGMA_S, G, 2)
    np.testing.assert_array_equal(ys2, ys)  # fixed summation order
    P.vie_destroy(hd)
    P.vie_destroy(ht)


def test_config3_assembled_solve_sampled_oracle_residual():
    # 32^3 (6 bumps, sigma_s = 0.8 sigma_t): GMRES to 1e-6 on the assembled
    # operator, the oracle's own residual on sampled rows, and agreement with
    # the on-the-fly solve
    m = V.heterogeneous_3d()
    assert m.n == 32
    h = P.vie_create(3, m.n, m.sigma_t, m.sigma_s)
    f = dev(m.f)
    U0 = torch.empty(m.N, dtype=torch.float64, device="cuda:0")
    P.vie_solve_gmres(h, f, U0, rtol=1e-6)
    for mode in (P.VIE_OPERATOR_FP32, P.VIE_OPERATOR_BF16X3, P.VIE_OPERATOR_SYM32):
        P.vie_assemble(h, mode)
        U = torch.empty_like(U0)
        rep = P.vie_solve_gmres(h, f, U, rtol=1e-6)
        assert rep["converged"] and rep["relres"] <= 1e-6
        rows = np.unique(np.random.default_rng(34).choice(m.N, 32, replace=False))
        u = host(U)
        phi = O.apply(3, m.sigma_t, m.sigma_s, m.f, op=O.OP_A_RAW, rows=rows)
        lhs = O.apply(3, m.sigma_t, m.sigma_s, u, op=O.OP_I_MINUS_K, rows=rows)
        assert np.linalg.norm(phi - lhs) <= 1e-5 * np.linalg.norm(phi)
        assert rel_l2(u, host(U0)) < 1e-5
    P.vie_destroy(h)
