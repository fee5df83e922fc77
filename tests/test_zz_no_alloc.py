"""vie_apply_noalloc: the apply for callers that cannot allocate device memory.

It must give what vie_apply gives, on two calls in a row (the second call
reuses the fixed scratch array the first one left behind), and refuse sizes
beyond its fixed scratch.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle as O
import vie_synth as V

torch = pytest.importorskip("torch")
import paper_1610_00835_gb300 as P  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-5   # the FP32-tile tolerance of the other apply tests


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("dim,n,op", [(2, 128, P.VIE_OP_K_SIGMA_S), (2, 45, P.VIE_OP_I_MINUS_K),
                                      (3, 25, P.VIE_OP_A_RAW)])
def test_noalloc_matches_vie_apply_twice(dim, n, op):
    dev = "cuda:0"
    media = [V.bump_medium(dim, n, 4, 0.9, seed=6000 + i) for i in range(2)]
    for call, m in enumerate(media):
        st = torch.as_tensor(m.sigma_t, device=dev)
        ss = torch.as_tensor(m.sigma_s, device=dev)
        g = torch.as_tensor(m.f + 0.1 * np.random.default_rng(call).standard_normal(m.N),
                            device=dev)
        y_ref = torch.empty_like(g)
        h = P.vie_create(dim, n, m.sigma_t, m.sigma_s)
        P.vie_apply(h, op, g, y_ref)
        y = torch.full_like(g, float("nan"))
        P.vie_apply_noalloc(dim, n, st, ss, op, g, y)
        torch.cuda.synchronize()
        assert _rel(y, y_ref) < TOL, f"call {call}"
        # and what the FP64 oracle computes, on sampled rows
        rows = np.unique(np.random.default_rng(call).choice(m.N, 16, replace=False))
        want = O.apply(dim, m.sigma_t, m.sigma_s, g.cpu().numpy(), op=op, rows=rows)
        got = y.cpu().numpy()[rows]
        assert np.linalg.norm(got - want) < TOL * np.linalg.norm(want), f"call {call}"
        P.vie_destroy(h)


def test_noalloc_on_a_side_stream_allocates_nothing():
    # a caller that cannot allocate runs it on its own stream: the result is
    # the same, and the device's free memory does not move across the call
    dev = "cuda:0"
    n = 100
    m = V.bump_medium(2, n, 4, 0.9, seed=6100)
    st = torch.as_tensor(m.sigma_t, device=dev)
    ss = torch.as_tensor(m.sigma_s, device=dev)
    g = torch.as_tensor(m.f, device=dev)
    y0 = torch.empty_like(g)
    y1 = torch.full_like(g, float("nan"))
    P.vie_apply_noalloc(2, n, st, ss, P.VIE_OP_K_SIGMA_S, g, y0)   # first call on the device
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    free0 = torch.cuda.mem_get_info()[0]
    with torch.cuda.stream(side):
        P.vie_apply_noalloc(2, n, st, ss, P.VIE_OP_K_SIGMA_S, g, y1, stream=side)
    side.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0
    torch.testing.assert_close(y1, y0, rtol=0, atol=0)


def test_noalloc_rejects_oversize_and_host_pointers():
    dev = "cuda:0"
    n = 129
    st = torch.ones(n * n, dtype=torch.float64, device=dev)
    g = torch.ones_like(st)
    y = torch.empty_like(st)
    with pytest.raises(P.VieError) as e:
        P.vie_apply_noalloc(2, n, st, st, P.VIE_OP_K_SIGMA_S, g, y)
    assert e.value.status == 1
    h = np.ones(16)
    with pytest.raises(P.VieError):
        P.vie_apply_noalloc(2, 4, h, h, P.VIE_OP_K_SIGMA_S, h, np.empty(16))
