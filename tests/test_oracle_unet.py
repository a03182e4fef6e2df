"""Pins of the U-Net oracle (the learned Newton initial guess): each layer
against an independent definition, the backward pass against central
differences of the forward loss, Adam's first step against its closed form,
bfloat16 rounding against exact cases."""
import numpy as np
import pytest
import scipy.ndimage

from oracle import unet


def test_conv3x3_is_periodic_cross_correlation():
    rng = np.random.default_rng(0)
    h = rng.standard_normal((2, 3, 8, 12))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    got = unet.conv3x3(h, w, b)
    for bi in range(2):
        for o in range(4):
            ref = b[o] + sum(scipy.ndimage.correlate(h[bi, i], w[o, i], mode="wrap") for i in range(3))
            assert np.allclose(got[bi, o], ref, rtol=0, atol=1e-12)


def test_pool_and_upsample_are_adjoint_to_their_backward_maps():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 8, 16))
    y = rng.standard_normal((2, 3, 4, 8))
    assert np.isclose(np.vdot(unet.pool2(x), y), np.vdot(x, unet.pool2_backward(y)), rtol=1e-13)
    assert np.isclose(np.vdot(unet.up2(y), x), np.vdot(y, unet.up2_backward(x)), rtol=1e-13)
    # 2x2 means and copies, by hand at one point
    assert np.isclose(unet.pool2(x)[1, 2, 3, 5], x[1, 2, 6:8, 10:12].mean())
    assert np.all(unet.up2(y)[:, :, 5, 9] == y[:, :, 2, 4])


def test_layout_counts_and_widths():
    lay = dict(unet.layout(2, 16))
    assert lay["enc0a.w"] == (16, 2, 3, 3) and lay["enc3b.w"] == (128, 128, 3, 3)
    assert lay["dec2a.w"] == (64, 128 + 64, 3, 3) and lay["dec0b.w"] == (16, 16, 3, 3)
    assert lay["out.w"] == (1, 16)
    assert unet.param_count(2, 24) == sum(int(np.prod(s)) for _, s in unet.layout(2, 24))
    assert 0.9e6 < unet.param_count(2, 24) < 1.3e6     # "about 1M parameters" at width 24


def _small(seed=2):
    rng = np.random.default_rng(seed)
    in_ch, width = 2, 2
    theta = rng.standard_normal(unet.param_count(in_ch, width)) * 0.3
    x = rng.standard_normal((2, in_ch, 8, 16))
    t = rng.standard_normal((2, 8, 16))
    return in_ch, width, theta, x, t


def test_gradient_matches_central_differences():
    in_ch, width, theta, x, t = _small()
    loss, g = unet.gradient(theta, x, t, in_ch, width)
    rng = np.random.default_rng(3)
    starts = np.cumsum([0] + [int(np.prod(s)) for _, s in unet.layout(in_ch, width)])[:-1]
    idx = np.unique(np.concatenate([starts, rng.integers(0, theta.size, 60)]))
    eps = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (unet.mse(unet.forward(tp, x, in_ch, width)[0], t)[0] -
              unet.mse(unet.forward(tm, x, in_ch, width)[0], t)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, 10 * abs(g[i])), (i, fd, g[i])


def test_zero_network_outputs_its_bias():
    in_ch, width = 2, 4
    theta = np.zeros(unet.param_count(in_ch, width))
    theta[-1] = 0.75
    y, _ = unet.forward(theta, np.ones((1, 2, 8, 8)), in_ch, width)
    assert np.all(y == 0.75)


def test_first_adam_step_closed_form():
    rng = np.random.default_rng(4)
    th = rng.standard_normal(50)
    g = rng.standard_normal(50)
    new, m, v = unet.adam_step(th, g, np.zeros(50), np.zeros(50), 1, lr=1e-3)
    assert np.allclose(new, th - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_rounding():
    exact = np.array([1.0, 1.5, -2.0 ** -10, 0.0, 3.0 * 2 ** 20])
    assert np.all(unet.bf16(exact) == exact)
    one = 1.0
    assert unet.bf16(np.array([one + 2.0 ** -8]))[0] == 1.0                       # tie -> even
    assert unet.bf16(np.array([one + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6       # tie -> even
    assert unet.bf16(np.array([one + 2.0 ** -8 + 2.0 ** -20]))[0] == 1.0 + 2.0 ** -7
    r = unet.bf16(np.random.default_rng(5).standard_normal(1000))
    assert np.all(r.astype(np.float32).view(np.uint32) & 0xFFFF == 0)


@pytest.mark.parametrize("bf", [False, True])
def test_bf16_storage_changes_little(bf):
    in_ch, width, theta, x, t = _small(6)
    y0, _ = unet.forward(theta, x, in_ch, width)
    y1, _ = unet.forward(theta, x, in_ch, width, bf16_storage=bf)
    rel = np.linalg.norm(y1 - y0) / np.linalg.norm(y0)
    assert (rel == 0.0) if not bf else (0.0 < rel < 5e-2)


def test_spectral_resampling_of_the_learned_start_is_the_band_limited_interpolant():
    """The learned Newton start is predicted on the training grid and
    resampled to the solve grid: every other point of the resampled field is
    the original field, and a band-limited mode is reproduced exactly."""
    from paper_1804_03859_gb300.learned_guess import spectral_resample

    rng = np.random.default_rng(3)
    q = rng.standard_normal((16, 32))
    f = spectral_resample(q, 64, 128)
    assert np.allclose(f[::4, ::4], q, atol=1e-12)
    assert np.allclose(spectral_resample(q, 16, 32), q, atol=1e-12)
    y = np.arange(16)[:, None] / 16
    x = np.arange(32)[None, :] / 32
    g = np.cos(2 * np.pi * 3 * x) * np.sin(2 * np.pi * 2 * y) + 0.3 * np.cos(2 * np.pi * 8 * y)
    Y = np.arange(64)[:, None] / 64
    X = np.arange(128)[None, :] / 128
    G = np.cos(2 * np.pi * 3 * X) * np.sin(2 * np.pi * 2 * Y) + 0.3 * np.cos(2 * np.pi * 8 * Y)
    assert np.allclose(spectral_resample(g, 64, 128), G, atol=1e-12)
