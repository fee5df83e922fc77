"""Failure detection of the tensor-core kernels without a GPU fault: the first
producer/consumer wait of every CTA is given no budget (a wait that runs out),
the kernels stop, drain what they issued within the full bound, free their
tensor memory and raise their error word; the calls report VIE_ERR_TIMEOUT and
the next call with the normal bounds runs and is correct."""
import numpy as np
import pytest

import oracle as O
import vie_synth as V

torch = pytest.importorskip("torch")
import paper_1610_00835_gb300 as P  # noqa: E402
from gpu_util import dev, host, rel_l2  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture
def first_wait_runs_out():
    P.vie_set_wait_limits(1000.0, 0.0)
    try:
        yield
    finally:
        P.vie_set_wait_limits(1000.0, -1.0)


def _bf16_handle(n=24, seed=8500):
    m = V.heterogeneous_2d(n=n, seed=seed)
    h = P.vie_create(2, n, m.sigma_t, m.sigma_s)
    P.vie_assemble(h, P.VIE_OPERATOR_BF16X3)
    return m, h


def test_limits_are_validated():
    for bad in ((0.0, -1.0), (-5.0, -1.0), (1e6, -1.0), (10.0, 20.0)):
        with pytest.raises(P.VieError) as e:
            P.vie_set_wait_limits(*bad)
        assert e.value.status == 1
    P.vie_set_wait_limits(1000.0, -1.0)


def test_product_timeout_is_reported_then_the_next_call_runs(first_wait_runs_out):
    m, h = _bf16_handle()
    R = 4
    G = V.bump_sources(2, m.n, R, seed=17)
    g = dev(G.ravel())
    y = torch.zeros_like(g)
    P.vie_apply(h, P.VIE_OP_K_SIGMA_S, g, y, R)       # asynchronous: NaN and the error word
    with pytest.raises(P.VieError) as e:
        P.vie_check_device(h)
    assert e.value.status == P.VIE_ERR_TIMEOUT
    assert torch.isnan(y).all()
    with pytest.raises(P.VieError) as e:              # host pointers: reported by the call
        P.vie_apply(h, P.VIE_OP_K_SIGMA_S, G.ravel(), np.empty(R * m.N), R)
    assert e.value.status == P.VIE_ERR_TIMEOUT
    P.vie_set_wait_limits(1000.0, -1.0)
    P.vie_apply(h, P.VIE_OP_K_SIGMA_S, g, y, R)
    P.vie_check_device(h)
    want = np.stack([O.apply(2, m.sigma_t, m.sigma_s, G[r]) for r in range(R)])
    assert rel_l2(host(y), want.ravel()) < 1e-5


def test_lockstep_solve_timeout_is_reported_then_the_next_solve_converges(first_wait_runs_out):
    m, h = _bf16_handle(seed=8501)
    R = 3
    F = V.bump_sources(2, m.n, R, seed=18)
    U = torch.empty(R * m.N, dtype=torch.float64, device="cuda:0")
    with pytest.raises(P.VieError) as e:
        P.vie_solve_gmres(h, dev(F.ravel()), U, rtol=1e-7, nrhs=R)
    assert e.value.status == P.VIE_ERR_TIMEOUT
    P.vie_set_wait_limits(1000.0, -1.0)
    reps = P.vie_solve_gmres(h, dev(F.ravel()), U, rtol=1e-7, nrhs=R)
    assert all(r["converged"] for r in reps)


def test_network_timeout_is_reported_then_the_next_forward_runs(first_wait_runs_out):
    net = P.vie_unet_create(2, 32, seed=3)
    n, B = 32, 2
    x = torch.randn(B * 3 * n * n, dtype=torch.float32, device="cuda:0")
    o = torch.zeros(B * n * n, dtype=torch.float32, device="cuda:0")
    with pytest.raises(P.VieError) as e:
        P.vie_unet_forward(net, x, o, B, n, use_bf16=True)
    assert e.value.status == P.VIE_ERR_TIMEOUT
    assert torch.isnan(o).any()
    P.vie_set_wait_limits(1000.0, -1.0)
    P.vie_unet_forward(net, x, o, B, n, use_bf16=True)
    ref = torch.empty_like(o)
    P.vie_unet_forward(net, x, ref, B, n)             # FP32 weights, CUDA cores
    assert not torch.isnan(o).any()
    assert rel_l2(host(o), host(ref)) < 2e-2
