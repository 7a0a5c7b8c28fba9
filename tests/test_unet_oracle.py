"""Pins of the FP64 U-Net reference (oracle/unet_oracle.py).

The convolution is checked against its loop definition, the layout helpers
against their inverses, and the whole backward pass against central finite
differences of the FP64 network (no bfloat16 rounding)."""
import numpy as np

from oracle import unet_oracle as U


def test_conv_matches_loop_definition():
    rng = np.random.default_rng(0)
    D, ci, co = 4, 3, 2
    x = rng.standard_normal((D, D, D, ci))
    w = rng.standard_normal((co, 27, ci))
    b = rng.standard_normal(co)
    got = U.conv(x, w, b)
    want = np.zeros((D, D, D, co))
    for z in range(D):
        for y in range(D):
            for xx in range(D):
                for o in range(co):
                    s = b[o]
                    t = 0
                    for dz in (-1, 0, 1):
                        for dy in (-1, 0, 1):
                            for dx in (-1, 0, 1):
                                s += x[(z + dz) % D, (y + dy) % D, (xx + dx) % D] @ w[o, t]
                                t += 1
                    want[z, y, xx, o] = s
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_conv_backward_is_adjoint():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((4, 4, 4, 3))
    w = rng.standard_normal((2, 27, 3))
    dout = rng.standard_normal((4, 4, 4, 2))
    dx, dw, db = U.conv_bwd(x, w, dout)
    # <conv(x), dout> is linear in x and in w
    base = np.sum(U.conv(x, w, np.zeros(2)) * dout)
    assert abs(np.sum(dx * x) - base) < 1e-9 * abs(base)
    assert abs(np.sum(dw * w) - base) < 1e-9 * abs(base)
    np.testing.assert_allclose(db, dout.sum(axis=(0, 1, 2)))


def test_pool_up_adjoints():
    rng = np.random.default_rng(2)
    a = rng.standard_normal((8, 8, 8, 2))
    c = rng.standard_normal((4, 4, 4, 2))
    assert abs(np.sum(U.pool(a) * c) - np.sum(a * U.pool_bwd(c))) < 1e-12
    assert abs(np.sum(U.up(c) * a) - np.sum(c * U.up_bwd(a))) < 1e-12


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 0.0, 3.0e38, 1e-40])
    r = U.bf16(vals)
    assert r[0] == 1.0 and r[1] == 1.0  # halfway rounds to even
    assert r[2] == 1.0 + 2 ** -7  # above halfway rounds up
    assert r[3] == -2.5 and r[4] == 0.0
    m = np.abs(r[:4] - vals[:4]) <= np.abs(vals[:4]) * 2 ** -8
    assert m.all()


def _sample(D=8, seed=3):
    rng = np.random.default_rng(seed)
    rho = np.exp(0.5 * rng.standard_normal((D, D, D)))
    phi = rng.standard_normal((D, D, D))
    phi_next = phi + 0.1 * rng.standard_normal((D, D, D))
    return rho, phi, phi_next


def test_gradient_finite_differences():
    rho, phi, phin = _sample()
    p = U.init_params(4)
    p[-17:-1] = np.random.default_rng(5).normal(0, 0.5, 16)  # a head that passes gradient
    loss, g = U.loss_and_grads(p, rho, phi, phin)
    rng = np.random.default_rng(6)
    idx = list(rng.choice(len(p) - 17, 40, replace=False)) + list(range(len(p) - 17, len(p)))
    eps = 1e-6
    for i in idx:
        if U.n_params() - 17 > i and _is_zero_padding(i):
            continue
        q = p.copy()
        q[i] += eps
        lp, _ = U.loss_and_grads(q, rho, phi, phin)
        q[i] -= 2 * eps
        lm, _ = U.loss_and_grads(q, rho, phi, phin)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-5 * abs(fd), (i, fd, g[i])


def test_base_and_output_scale():
    """delta depends on (rho, field) only; the prediction is base + c rms(field)
    delta; a loss with scale c equals the scale-1 loss of the target pulled
    toward base by 1/c; finite differences still hold with base and c."""
    rho, field, target = _sample(seed=9)
    base = np.random.default_rng(10).standard_normal(field.shape)
    p = U.init_params(11)
    p[-17:-1] = np.random.default_rng(12).normal(0, 0.5, 16)
    d1, pred1, _ = U.forward(p, rho, field)
    d2, pred2, _ = U.forward(p, rho, field, base, scale=3.0)
    assert np.array_equal(d1, d2)
    rms = np.sqrt(np.mean(field ** 2))
    assert np.allclose(pred1, field + rms * d1, rtol=0, atol=1e-12)
    assert np.allclose(pred2, base + 3.0 * rms * d1, rtol=0, atol=1e-12)
    l3, g3 = U.loss_and_grads(p, rho, field, target, base, scale=3.0)
    l1, g1 = U.loss_and_grads(p, rho, field, base + (target - base) / 3.0, base)
    assert abs(l3 - l1) <= 1e-12 * l1
    assert np.allclose(g3, g1, rtol=1e-10, atol=1e-14)
    eps = 1e-6
    for i in [5, 1000, len(p) - 3, len(p) - 1]:
        q = p.copy()
        q[i] += eps
        lp, _ = U.loss_and_grads(q, rho, field, target, base, scale=3.0)
        q[i] -= 2 * eps
        lm, _ = U.loss_and_grads(q, rho, field, target, base, scale=3.0)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g3[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-5 * abs(fd), (i, fd, g3[i])


def _is_zero_padding(i):
    # first-layer weights on the zero input channels 2..15: gradient exactly 0
    if i >= 16 * 27 * 16:
        return False
    return (i % 16) >= 2


def test_zero_padding_channels_get_zero_gradient():
    rho, phi, phin = _sample()
    loss, g = U.loss_and_grads(U.init_params(7), rho, phi, phin)
    w0 = g[:16 * 27 * 16].reshape(16, 27, 16)
    assert np.all(w0[:, :, 2:] == 0.0)
    assert len(g) == U.n_params()


def test_bf16_emulation_stays_close_to_fp64():
    rho, phi, phin = _sample()
    p = U.init_params(8)
    d64, _, _ = U.forward(p, rho, phi, bf=False)
    d16, _, _ = U.forward(p, rho, phi, bf=True)
    assert np.linalg.norm(d16 - d64) <= 0.05 * np.linalg.norm(d64)
