"""Pins of the FP64 network oracle (oracle/net.py) to things other than
itself: brute-force loops on tiny inputs, delta responses, adjoint
identities, closed forms and central differences."""
import numpy as np
import pytest

from oracle import net as onet


def rng(seed):
    return np.random.default_rng(seed)


def test_conv3d_matches_brute_force_loops():
    r = rng(0)
    x = r.standard_normal((2, 4, 3, 5, 3))
    w = r.standard_normal((2, 27, 3))
    b = r.standard_normal(2)
    y = onet.conv3d(x, w, b)
    B, D, H, W, _ = x.shape
    ref = np.zeros((B, D, H, W, 2))
    for bb in range(B):
        for d in range(D):
            for h in range(H):
                for ww in range(W):
                    for co in range(2):
                        s = b[co]
                        for kd in range(3):
                            for kh in range(3):
                                for kw in range(3):
                                    tap = 9 * kd + 3 * kh + kw
                                    q = x[bb, (d + kd - 1) % D, (h + kh - 1) % H, (ww + kw - 1) % W]
                                    s += np.dot(w[co, tap], q)
                        ref[bb, d, h, ww, co] = s
    assert np.max(np.abs(y - ref)) < 1e-12


def test_conv3d_delta_response_is_reflected_kernel():
    """A unit impulse at voxel q, channel ci produces y[q - off(tap), co] = w[co, tap, ci]."""
    r = rng(1)
    w = r.standard_normal((3, 27, 2))
    x = np.zeros((1, 6, 6, 6, 2))
    q = (3, 2, 4)
    x[0, q[0], q[1], q[2], 1] = 1.0
    y = onet.conv3d(x, w)
    for tap, (a, bb, c) in enumerate(onet.TAPS):
        p = ((q[0] - a) % 6, (q[1] - bb) % 6, (q[2] - c) % 6)
        assert np.allclose(y[0, p[0], p[1], p[2]], w[:, tap, 1], atol=1e-14)
    assert np.count_nonzero(np.abs(y) > 0) == 27 * 3


def test_conv3d_adjoint_identities():
    r = rng(2)
    x = r.standard_normal((2, 4, 6, 8, 3))
    w = r.standard_normal((5, 27, 3))
    dy = r.standard_normal((2, 4, 6, 8, 5))
    lhs = np.sum(onet.conv3d(x, w) * dy)
    assert abs(lhs - np.sum(x * onet.conv3d_input_grad(dy, w))) < 1e-10 * abs(lhs)
    dw, db = onet.conv3d_weight_grad(x, dy)
    assert abs(lhs - np.sum(w * dw)) < 1e-10 * abs(lhs)
    assert np.allclose(db, dy.reshape(-1, 5).sum(0))


def test_pool_up_adjoint_and_values():
    r = rng(3)
    x = r.standard_normal((2, 4, 4, 8, 3))
    y = r.standard_normal((2, 2, 2, 4, 3))
    assert abs(np.sum(onet.pool2(x) * y) - np.sum(x * onet.pool2_adj(y))) < 1e-12
    assert abs(np.sum(onet.up2(y) * x) - np.sum(y * onet.up2_adj(x))) < 1e-12
    # pooling a constant, upsampling then pooling
    assert np.allclose(onet.pool2(np.full((1, 4, 4, 4, 1), 2.5)), 2.5)
    assert np.allclose(onet.pool2(onet.up2(y)), y)
    assert abs(onet.pool2(x)[1, 1, 0, 2, 2] - x[1, 2:4, 0:2, 4:6, 2].mean()) < 1e-14


def test_adam_first_step_is_sign_step():
    """After one step m^ = g and s^ = g^2, so the update is lr * g / (|g| + eps)."""
    r = rng(4)
    w = r.standard_normal(50)
    g = r.standard_normal(50)
    w1, m, s = onet.adam(w, g, np.zeros(50), np.zeros(50), 1e-3, 0.9, 0.999, 1e-8, 1)
    assert np.allclose(w1, w - 1e-3 * g / (np.abs(g) + 1e-8), atol=1e-15)
    # second step with the same gradient: same update again
    w2, _, _ = onet.adam(w1, g, m, s, 1e-3, 0.9, 0.999, 1e-8, 2)
    assert np.allclose(w2 - w1, w1 - w, atol=1e-12)


def test_head_and_leaky_by_finite_differences():
    r = rng(5)
    x = r.standard_normal((1, 4, 4, 4, 4))
    wh = r.standard_normal((3, 4))
    bh = r.standard_normal(3)
    dv = r.standard_normal((1, 3, 4, 4, 4))
    dx, dwh, dbh = onet.head_grad(x, wh, 0.7, dv)
    f = lambda xx, ww, bb: np.sum(onet.head(xx, ww, bb, 0.7) * dv)
    e = 1e-6
    tx = r.standard_normal(x.shape)
    tw = r.standard_normal(wh.shape)
    assert abs((f(x + e * tx, wh, bh) - f(x - e * tx, wh, bh)) / (2 * e) - np.sum(dx * tx)) < 1e-7
    assert abs((f(x, wh + e * tw, bh) - f(x, wh - e * tw, bh)) / (2 * e) - np.sum(dwh * tw)) < 1e-7
    assert np.allclose(dbh, 0.7 * dv.sum(axis=(0, 2, 3, 4)))
    y = r.standard_normal(100)
    d = r.standard_normal(100)
    assert np.allclose(onet.leaky_grad(d, onet.leaky(y, 0.1), 0.1), np.where(y > 0, d, 0.1 * d))


@pytest.mark.parametrize("chans", [(16, 32), (16, 32, 64, 128)])
def test_unet_gradient_matches_finite_differences(chans):
    """Directional derivative of <dv, v(params)> along a random direction of
    every parameter equals the reverse-mode gradient (central differences)."""
    r = rng(6)
    n = 8
    layers = onet.unet_layers(chans, cin=4)
    params = {name: (r.standard_normal((co, 27, ci)) / np.sqrt(27 * ci), 0.1 * r.standard_normal(co))
              for name, ci, co in layers}
    params["head"] = (r.standard_normal((3, chans[0])) / np.sqrt(chans[0]), 0.1 * r.standard_normal(3))
    x = r.standard_normal((1, n, n, n, 4))
    dv = r.standard_normal((1, 3, n, n, n))
    v, cache = onet.unet_forward(params, x, chans, slope=0.1, vscale=0.5)
    grads = onet.unet_backward(params, cache, dv, chans, slope=0.1, vscale=0.5)
    dirs = {k: (r.standard_normal(p[0].shape), r.standard_normal(p[1].shape)) for k, p in params.items()}
    pred = sum(np.sum(grads[k][0] * dirs[k][0]) + np.sum(grads[k][1] * dirs[k][1]) for k in params)

    def f(eps):
        pp = {k: (params[k][0] + eps * dirs[k][0], params[k][1] + eps * dirs[k][1]) for k in params}
        return np.sum(onet.unet_forward(pp, x, chans, slope=0.1, vscale=0.5)[0] * dv)

    # small step: the leaky ReLU kinks make the map piecewise smooth, so the
    # step must stay below the distance of every pre-activation from zero
    e = 1e-8
    fd = (f(e) - f(-e)) / (2 * e)
    assert abs(fd - pred) < 1e-6 * abs(pred)
