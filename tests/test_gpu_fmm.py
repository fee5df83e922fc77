"""The FMM operator (Section 3.3) on the GPU: against the oracle's FMM (the same
approximation, element by element), and against the direct operator."""
import os

import numpy as np
import pytest

import oracle as O
import vie_synth as V
from oracle import fmm as F

torch = pytest.importorskip("torch")
import paper_1610_00835_gb300 as P  # noqa: E402
from gpu_util import dev, host, rel_l2  # noqa: E402

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
OPS = (P.VIE_OP_K_SIGMA_S, P.VIE_OP_I_MINUS_K, P.VIE_OP_A_RAW)


def gpu_apply(h, op, g):
    y = torch.empty(h.N, dtype=torch.float64, device="cuda:0")
    P.vie_apply(h, op, dev(g), y, 1)
    return host(y)


@pytest.mark.parametrize("n,p", [(32, 6), (48, 4), (64, 4)])
def test_fmm_matches_the_oracle_fmm(n, p):
    # two levels with 8- and 12-cell leaves, three levels with 8-cell leaves
    m = V.bump_medium(2, n, 4, 0.9, seed=5600 + n)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    P.vie_assemble_fmm(h, p)
    g = m.f + 0.05 * np.random.default_rng(n).standard_normal(m.N)
    s = m.sigma_s * g
    want_k = F.apply(m.sigma_t, s, n, p)
    got = {op: gpu_apply(h, op, g) for op in OPS}
    assert rel_l2(got[P.VIE_OP_K_SIGMA_S], want_k) < 2e-5
    assert rel_l2(got[P.VIE_OP_I_MINUS_K], g - want_k) < 2e-5
    assert rel_l2(got[P.VIE_OP_A_RAW], F.apply(m.sigma_t, g, n, p)) < 2e-5


def test_fmm_converges_to_the_direct_operator_on_a_homogeneous_medium():
    # closed-form tau: the far field converges spectrally in the order until
    # the FP32 entries' rounding
    n = 128
    st = np.full(n * n, 2.2)
    h = P.vie_create(2, n, st, st, tau_mode=P.VIE_TAU_CLOSED)
    g = np.random.default_rng(1).standard_normal(n * n)
    direct = gpu_apply(h, P.VIE_OP_K_SIGMA_S, g)
    errs = []
    for p in (3, 5, 7):
        P.vie_assemble_fmm(h, p)
        errs.append(rel_l2(gpu_apply(h, P.VIE_OP_K_SIGMA_S, g), direct))
    assert errs[0] > 10 * errs[1] > 10 * 5 * errs[2]
    assert errs[2] < 2e-6


def test_fmm_solve_at_128_against_the_oracle_solution():
    # the bench medium: GMRES with the FMM operator, against the FP64 oracle's
    # direct solution (the far field's approximation error bounds the gap)
    U_or = np.load(os.path.join(GOLDEN, "bench_U_2d_128.npy"))
    m = V.heterogeneous_2d(n=128, seed=V.seed_for(2, 0))
    h = P.vie_create(2, 128, m.sigma_t, m.sigma_s)
    P.vie_assemble_fmm(h, 6)
    U = torch.empty(m.N, dtype=torch.float64, device="cuda:0")
    rep = P.vie_solve_gmres(h, dev(m.f), U, rtol=1e-6)
    assert rep["converged"]
    assert rel_l2(host(U), U_or) < 1e-4


def test_fmm_at_512_sampled_rows():
    # N = 262144, the paper's largest grid: sampled rows of the direct operator
    n = 512
    m = V.bump_medium(2, n, 4, 0.9, seed=5700)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    P.vie_assemble_fmm(h, 6)
    g = m.f + 0.05 * np.random.default_rng(7).standard_normal(m.N)
    got = gpu_apply(h, P.VIE_OP_K_SIGMA_S, g)
    rows = np.unique(np.concatenate([np.random.default_rng(8).choice(m.N, 6, replace=False),
                                     [0, n - 1, m.N // 2 + n // 2, m.N - 1]]))
    want = O.apply(2, m.sigma_t, m.sigma_s, g, rows=rows)
    assert rel_l2(got[rows], want) < 2e-4


@pytest.mark.parametrize("case", ["shallow", "3d", "fp64", "mii", "order1", "order13"])
def test_fmm_unsupported_and_invalid(case):
    status = P.vie.VIE_ERR_UNSUPPORTED
    order = 6
    if case == "3d":
        m = V.heterogeneous_3d(n=8)
        h = P.vie_create(3, 8, m.sigma_t, m.sigma_s)
    else:
        n = 24 if case == "shallow" else 32          # 24 = 2 x 12: one level, no far field
        m = V.bump_medium(2, n, 2, 0.9, seed=5800)
        kw = {}
        if case == "fp64":
            kw["precision"] = P.VIE_PREC_FP64
        elif case == "mii":
            kw["disc"] = P.VIE_DISC_MII
        h = P.vie_create(2, n, m.sigma_t, m.sigma_s, **kw)
        if case.startswith("order"):
            order = int(case[5:])
            status = P.vie.VIE_ERR_INVALID_ARG
    with pytest.raises(P.VieError) as e:
        P.vie_assemble_fmm(h, order)
    assert e.value.status == status
    y = gpu_apply(h, P.VIE_OP_K_SIGMA_S, m.f)      # still applies on the fly
    assert np.all(np.isfinite(y))
