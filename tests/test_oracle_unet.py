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


def test_round_bf16_nearest_ties_to_even():
    # BF16 keeps 7 fraction bits: the spacing above 1 is 2^-7
    x = np.array([1.0, 1 + 2**-8, 1 + 3 * 2**-9, 1 + 2**-7 + 2**-8, -1 - 2**-8 - 2**-20, 2.0**-130, 0.0])
    want = np.array([1.0, 1.0, 1 + 2**-7, 1 + 2**-6, -(1 + 2**-7), 2.0**-130, 0.0])
    np.testing.assert_array_equal(R.round_bf16(x), want)


def test_bf16_forward_rounds_weights_and_conv_inputs_only():
    # weights and input that are BF16 values already, perturbed by less than
    # half a BF16 spacing: the BF16 forward rounds them back and is unchanged,
    # bit for bit, while the exact forward moves; the rounding of the
    # intermediate activations keeps the two forwards within a few 2^-8
    params = R.init_params(2, 4, seed=3)
    params = [R.round_bf16(p) if i % 2 == 0 else p for i, p in enumerate(params)]
    x = R.round_bf16(np.random.default_rng(1).standard_normal((1, 3, 8, 8)))
    o, _ = R.forward(params, x, 2)
    ob, _ = R.forward(params, x, 2, bf16=True)
    assert 0 < np.linalg.norm(ob - o) / np.linalg.norm(o) < 2e-2
    xp = x * (1 + 2.0**-12)
    pp = [p * (1 + 2.0**-12) if i % 2 == 0 else p for i, p in enumerate(params)]
    np.testing.assert_array_equal(R.forward(pp, xp, 2, bf16=True)[0], ob)
    assert not np.array_equal(R.forward(pp, xp, 2)[0], o)
