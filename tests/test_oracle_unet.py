"""Pins of the FP64 network reference (oracle/unet.py) by finite differences."""
import numpy as np
import pytest

from oracle import unet as R


@pytest.mark.parametrize("levels,channels", [(1, 3), (2, 4), (3, 4)])
def test_gradients_match_central_differences(levels, channels):
    rng = np.random.default_rng(levels)
    n = 8
    params = R.init_params(levels, channels, seed=levels)
    params = [p + 0.05 * rng.standard_normal(p.shape) for p in params]  # nonzero biases
    x = rng.standard_normal((2, 3, n, n))
    t = rng.standard_normal((2, 1, n, n))
    loss, grads, _ = R.loss_and_grads(params, x, t, levels)
    eps = 1e-6
    for pi in range(len(params)):
        flat = params[pi].reshape(-1)
        for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _, _ = R.loss_and_grads(params, x, t, levels)
            flat[idx] = old - eps
            lm, _, _ = R.loss_and_grads(params, x, t, levels)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert grads[pi].reshape(-1)[idx] == pytest.approx(fd, rel=1e-5, abs=1e-9), (pi, idx)


def test_conv_is_a_correlation_with_zero_padding():
    # hand-checked 3x3 example: a delta input reproduces the flipped kernel
    x = np.zeros((1, 1, 5, 5))
    x[0, 0, 2, 2] = 1.0
    w = np.arange(9.0).reshape(1, 1, 3, 3)
    out = R.conv(x, w, np.zeros(1))
    np.testing.assert_array_equal(out[0, 0, 1:4, 1:4], w[0, 0, ::-1, ::-1])
    assert out[0, 0, 0].sum() == 0 and out[0, 0, 4].sum() == 0


def test_pool_and_upsample_are_adjoint_up_to_a_factor():
    rng = np.random.default_rng(0)
    a = rng.standard_normal((1, 2, 4, 4))
    b = rng.standard_normal((1, 2, 2, 2))
    # <pool(a), b> = <a, pool^T b> and pool^T = upsample / 4
    assert np.sum(R.avgpool2(a) * b) == pytest.approx(np.sum(a * R.upsample2(b)) / 4)
