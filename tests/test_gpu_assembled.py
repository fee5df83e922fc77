"""The assembled operator (FP32 and BF16 hi/lo) and its products, against the oracle."""
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


@pytest.mark.parametrize("mode", [P.VIE_OPERATOR_FP32, P.VIE_OPERATOR_BF16X3, P.VIE_OPERATOR_PAIRS32,
                                  P.VIE_OPERATOR_SYM32])
@pytest.mark.parametrize("n", [2, 7, 24, 45])
def test_single_rhs_all_rows(mode, n):
    m = V.heterogeneous_2d(n=n, seed=91)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    P.vie_assemble(h, mode)
    g = m.f + 0.2 * np.random.default_rng(n).standard_normal(m.N)
    for op in (P.VIE_OP_K_SIGMA_S, P.VIE_OP_I_MINUS_K, P.VIE_OP_A_RAW):
        got = _apply(h, op, g, 1)[0]
        want = O.apply(2, m.sigma_t, m.sigma_s, g, op=op)
        assert rel_l2(got, want) < TOL


@pytest.mark.parametrize("n,nrhs", [(24, 2), (24, 16), (40, 64), (45, 100), (24, 256)])
def test_bf16x3_tensor_core_product(n, nrhs):
    m = V.heterogeneous_2d(n=n, seed=92)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    P.vie_assemble(h, P.VIE_OPERATOR_BF16X3)
    G = V.bump_sources(2, n, nrhs, seed=7000 + nrhs) + 0.01
    got = _apply(h, P.VIE_OP_K_SIGMA_S, G, nrhs)
    K = O.k_matrix(2, m.sigma_t, m.sigma_s)
    want = G @ K.T
    for r in range(nrhs):
        assert rel_l2(got[r], want[r]) < TOL, r


def test_3d_assembled_product():
    m = V.heterogeneous_3d(n=9, seed=93)
    h = P.vie_create(3, 9, m.sigma_t, m.sigma_s)
    P.vie_assemble(h, P.VIE_OPERATOR_BF16X3)
    G = np.stack([m.f, m.f ** 2 + 0.1, np.ones(m.N)])
    got = _apply(h, P.VIE_OP_K_SIGMA_S, G, 3)
    K = O.k_matrix(3, m.sigma_t, m.sigma_s)
    for r in range(3):
        assert rel_l2(got[r], K @ G[r]) < TOL


def test_config4_full_size_64_sources_sampled_rows():
    m = V.heterogeneous_2d()
    h = P.vie_create(2, m.n, m.sigma_t, m.sigma_s)
    G = V.bump_sources(2, m.n, 64, seed=V.seed_for(4))
    y_otf = _apply(h, P.VIE_OP_K_SIGMA_S, G[:2], 2)
    P.vie_assemble(h, P.VIE_OPERATOR_BF16X3)
    got = _apply(h, P.VIE_OP_K_SIGMA_S, G, 64)
    rows = np.unique(np.random.default_rng(4).choice(m.N, 12, replace=False))
    for r in (0, 17, 63):
        want = O.apply(2, m.sigma_t, m.sigma_s, G[r], rows=rows)
        assert rel_l2(got[r][rows], want) < TOL
    for r in range(2):
        assert rel_l2(got[r], y_otf[r]) < TOL


@pytest.mark.parametrize("mode", [P.VIE_OPERATOR_FP32, P.VIE_OPERATOR_BF16X3, P.VIE_OPERATOR_PAIRS32,
                                  P.VIE_OPERATOR_SYM32])
def test_gmres_with_assembled_operator(mode):
    n = 32
    m = V.heterogeneous_2d(n=n)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    U_otf = np.zeros(m.N)
    P.vie_solve_gmres(h, m.f, U_otf, rtol=1e-9)
    P.vie_assemble(h, mode)
    U = np.zeros(m.N)
    rep = P.vie_solve_gmres(h, m.f, U, rtol=1e-9)
    assert rep["converged"]
    phi = O.apply(2, m.sigma_t, m.sigma_s, m.f, op=O.OP_A_RAW)
    U_lu = O.lu_solve(2, m.sigma_t, m.sigma_s, phi)
    assert rel_l2(U, U_lu) < TOL
    assert rel_l2(U, U_otf) < TOL
    P.vie_assemble(h, P.VIE_OPERATOR_OTF)   # back to on-the-fly, matrix freed
    U2 = np.zeros(m.N)
    P.vie_solve_gmres(h, m.f, U2, rtol=1e-9)
    np.testing.assert_array_equal(U2, U_otf)


@pytest.mark.parametrize("n", [2, 3, 9, 37, 64, 128, 133, 233, 234, 256])
def test_pairs32_bitwise_equal_to_on_the_fly(n):
    # the stored weights are the on-the-fly kernel's FP32 weights and the
    # accumulation is the same exact fixed-point sum: identical results
    m = V.heterogeneous_2d(n=n, seed=93)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    assert P.vie_get_kernel(h) == P.VIE_KERNEL_DISPLACEMENT
    G = np.stack([m.f, np.random.default_rng(n).standard_normal(m.N)])
    ops = (P.VIE_OP_K_SIGMA_S, P.VIE_OP_I_MINUS_K, P.VIE_OP_A_RAW)
    otf = [_apply(h, op, G, 2) for op in ops]
    P.vie_assemble(h, P.VIE_OPERATOR_PAIRS32)
    for op, want in zip(ops, otf):
        np.testing.assert_array_equal(_apply(h, op, G, 2), want)
    P.vie_assemble(h, P.VIE_OPERATOR_PAIRS32)   # re-assembled in place
    np.testing.assert_array_equal(_apply(h, ops[0], G, 2), otf[0])


def test_pairs32_switches_with_other_modes():
    n = 24
    m = V.heterogeneous_2d(n=n, seed=94)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    g = m.f[None, :]
    want = O.apply(2, m.sigma_t, m.sigma_s, m.f)
    for mode in (P.VIE_OPERATOR_PAIRS32, P.VIE_OPERATOR_BF16X3, P.VIE_OPERATOR_SYM32, P.VIE_OPERATOR_PAIRS32,
                 P.VIE_OPERATOR_SYM32, P.VIE_OPERATOR_OTF):
        P.vie_assemble(h, mode)
        assert rel_l2(_apply(h, P.VIE_OP_K_SIGMA_S, g, 1)[0], want) < TOL


@pytest.mark.parametrize("mode", [P.VIE_OPERATOR_PAIRS32, P.VIE_OPERATOR_SYM32])
@pytest.mark.parametrize("case", ["3d", "symmetric", "too_large"])
def test_pairs32_unsupported_without_the_displacement_kernel(case, mode):
    if case == "3d":
        # the pair weights are 2D only; the 3D symmetric blocks come from the 3D
        # displacement kernel, so a handle on the tile-pair kernel has none
        m = V.heterogeneous_3d(n=5)
        kernel = P.VIE_KERNEL_SYMMETRIC if mode == P.VIE_OPERATOR_SYM32 else P.VIE_KERNEL_AUTO
        h = P.vie_create(3, 5, m.sigma_t, m.sigma_s, kernel=kernel)
    elif case == "symmetric":
        m = V.heterogeneous_2d(n=16)
        h = P.vie_create(2, 16, m.sigma_t, m.sigma_s, kernel=P.VIE_KERNEL_SYMMETRIC)
    else:
        m = V.heterogeneous_2d(n=259)
        h = P.vie_create(2, 259, m.sigma_t, m.sigma_s)
    with pytest.raises(P.VieError) as e:
        P.vie_assemble(h, mode)
    assert e.value.status == P.vie.VIE_ERR_UNSUPPORTED
    # the handle still applies on the fly
    y = _apply(h, P.VIE_OP_K_SIGMA_S, m.f[None, :], 1)[0]
    assert np.all(np.isfinite(y))


@pytest.mark.parametrize("n", [16, 128, 133, 160])
def test_sym32_full_size_rows_and_symmetry(n):
    # the symmetric blocks against the oracle on sampled rows at full sizes, and
    # against the dense FP32 K applied to the same vector
    m = V.bump_medium(2, n, 4, 0.9, seed=4500 + n)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    g = m.f + 0.05 * np.random.default_rng(n).standard_normal(m.N)
    P.vie_assemble(h, P.VIE_OPERATOR_SYM32)
    got = _apply(h, P.VIE_OP_K_SIGMA_S, g, 1)[0]
    rows = np.unique(np.concatenate([np.random.default_rng(n + 1).choice(m.N, 12, replace=False),
                                     [0, m.N - 1, m.N // 2]]))
    want = O.apply(2, m.sigma_t, m.sigma_s, g, rows=rows)
    assert rel_l2(got[rows], want) < TOL
    P.vie_assemble(h, P.VIE_OPERATOR_FP32)
    assert rel_l2(got, _apply(h, P.VIE_OP_K_SIGMA_S, g, 1)[0]) < 2e-6
    P.vie_assemble(h, P.VIE_OPERATOR_SYM32)
    again = _apply(h, P.VIE_OP_K_SIGMA_S, g, 1)[0]
    np.testing.assert_array_equal(again, got)  # fixed summation order


def test_past_the_expansion_dense_k_comes_from_the_tile_assembler():
    # n = 170: the displacement kernel and the pair weights still apply, the
    # symmetric blocks are refused (past n = 160, and their expansion has no
    # room), and dense K is assembled by the tile-pair assembler instead
    n = 170
    m = V.bump_medium(2, n, 4, 0.9, seed=4670)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    assert P.vie_get_kernel(h) == P.VIE_KERNEL_DISPLACEMENT
    g = m.f + 0.05 * np.random.default_rng(n).standard_normal(m.N)
    otf = _apply(h, P.VIE_OP_K_SIGMA_S, g, 1)[0]
    with pytest.raises(P.VieError) as e:
        P.vie_assemble(h, P.VIE_OPERATOR_SYM32)
    assert e.value.status == P.vie.VIE_ERR_UNSUPPORTED
    P.vie_assemble(h, P.VIE_OPERATOR_PAIRS32)
    np.testing.assert_array_equal(_apply(h, P.VIE_OP_K_SIGMA_S, g, 1)[0], otf)
    P.vie_assemble(h, P.VIE_OPERATOR_FP32)
    dense = _apply(h, P.VIE_OP_K_SIGMA_S, g, 1)[0]
    assert rel_l2(dense, otf) < 2e-6
    rows = np.unique(np.concatenate([np.random.default_rng(n + 1).choice(m.N, 8, replace=False), [0, m.N - 1]]))
    want = O.apply(2, m.sigma_t, m.sigma_s, g, rows=rows)
    assert rel_l2(dense[rows], want) < TOL
