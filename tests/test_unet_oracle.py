"""Pins of the FP64 U-Net oracle (CPU): each layer against an independent library routine or
brute force, and the whole backward pass against central finite differences."""
import numpy as np
import pytest

from oracle import unet_oracle as U

scipy_signal = pytest.importorskip("scipy.signal")


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_conv3x3_matches_scipy_correlate():
    r = rng(1)
    x = r.normal(size=(2, 5, 7, 3))
    w = r.normal(size=(3, 3, 3, 4))
    b = r.normal(size=4)
    y = U.conv3x3(x, w, b)
    for n in range(2):
        for o in range(4):
            want = b[o] + sum(scipy_signal.correlate2d(x[n, :, :, c], w[:, :, c, o], mode="same", boundary="fill")
                              for c in range(3))
            np.testing.assert_allclose(y[n, :, :, o], want, rtol=1e-12, atol=1e-12)


def test_upconv2_is_a_kronecker_expansion():
    r = rng(2)
    x = r.normal(size=(1, 3, 4, 2))
    w = r.normal(size=(2, 2, 2, 3))
    b = r.normal(size=3)
    y = U.upconv2(x, w, b)
    for o in range(3):
        want = b[o] + sum(np.kron(x[0, :, :, c], w[:, :, c, o]) for c in range(2))
        np.testing.assert_allclose(y[0, :, :, o], want, rtol=1e-12, atol=1e-12)


def test_maxpool_and_its_backward_by_brute_force():
    r = rng(3)
    x = r.normal(size=(2, 4, 6, 3))
    y, arg = U.maxpool2(x)
    gy = r.normal(size=y.shape)
    gx = U.maxpool2_backward(arg, gy, x.shape)
    want_gx = np.zeros_like(x)
    for b in range(2):
        for h in range(2):
            for w in range(3):
                for c in range(3):
                    win = [(2 * h + dy, 2 * w + dx) for dy in range(2) for dx in range(2)]
                    vals = [x[b, i, j, c] for i, j in win]
                    k = int(np.argmax(vals))
                    assert y[b, h, w, c] == max(vals)
                    want_gx[b, win[k][0], win[k][1], c] += gy[b, h, w, c]
    np.testing.assert_array_equal(gx, want_gx)


def test_network_gradient_matches_central_differences():
    """Every parameter tensor: a few entries of dL/dp against (L(p + h) - L(p - h)) / 2h."""
    base, c_in = 2, 4
    p = U.init_params(base, c_in, seed=4)
    for k in p:  # nonzero biases so that their gradients are exercised away from ReLU kinks
        if k.endswith(".b"):
            p[k] = rng(5).normal(0, 0.05, p[k].shape)
    r = rng(6)
    x = r.normal(size=(2, 8, 16, c_in))
    target = r.normal(size=(2, 8))
    L, g, _ = U.loss_and_grad(p, x, target)
    h = 1e-6
    for name in p:
        flat = p[name].reshape(-1)
        for idx in r.choice(flat.size, size=min(3, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            Lp, _, _ = U.loss_and_grad(p, x, target)
            flat[idx] = old - h
            Lm, _, _ = U.loss_and_grad(p, x, target)
            flat[idx] = old
            fd = (Lp - Lm) / (2 * h)
            an = g[name].reshape(-1)[idx]
            assert abs(an - fd) <= 1e-6 * max(abs(fd), 1e-3), (name, idx, an, fd)


def test_adam_first_step_is_a_signed_learning_rate():
    p = {"a": np.array([1.0, -2.0, 3.0])}
    g = {"a": np.array([0.5, -4.0, 1e-3])}
    m = {"a": np.zeros(3)}
    v = {"a": np.zeros(3)}
    p, m, v = U.adam(p, g, m, v, 1, lr=0.1)
    np.testing.assert_allclose(p["a"], [1.0 - 0.1, -2.0 + 0.1, 3.0 - 0.1], rtol=0, atol=1e-6)


def test_param_shapes_follow_the_unet_recipe():
    s = dict(U.param_shapes(32, 8))
    assert s["enc0a.w"] == (3, 3, 8, 32) and s["enc3b.w"] == (3, 3, 256, 256)
    assert s["up2.w"] == (2, 2, 256, 128) and s["dec2a.w"] == (3, 3, 256, 128)
    assert s["dec0b.w"] == (3, 3, 32, 32) and s["head.w"] == (32,)


def test_storage_model_identity_changes_nothing_and_rounding_is_applied():
    """forward/backward with an explicit identity store give the same bits as
    the default; a rounding store changes the result by about its unit."""
    base, c_in = 2, 4
    p = U.init_params(base, c_in, seed=7)
    r = rng(8)
    x = r.normal(size=(1, 8, 16, c_in))
    t = r.normal(size=(1, 8))
    L0, g0, o0 = U.loss_and_grad(p, x, t)
    L1, g1, o1 = U.loss_and_grad(p, x, t, store=lambda a: a)
    assert L0 == L1 and all(np.array_equal(g0[k], g1[k]) for k in g0)
    r8 = lambda a: np.round(a * 256.0) / 256.0
    L2, _, o2 = U.loss_and_grad(p, x, t, store=r8)
    assert 0 < np.max(np.abs(o2 - o0)) < 0.1
