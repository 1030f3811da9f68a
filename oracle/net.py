"""FP64 CPU oracle for the learned warm start: a 3D U-Net over periodic
volumes that maps an image pair (m0, m1) to an initial velocity.

TEST INFRASTRUCTURE.  Only tests/, ``__graft_entry__.smoke()`` and the CPU
legs of ``bench.py`` may import this module.  It shares no code with the CUDA
path.  The paper has no network; these are the plain definitions of the
layers the extension uses, written out in float64 numpy:

* conv3d: y[p, co] = act(b[co] + sum_{tap, ci} x[p + off(tap), ci] w[co, tap, ci])
  with 27 taps off = (kd-1, kh-1, kw-1), tap = 9 kd + 3 kh + kw, periodic
  wrap-around (the registration domain is the 3-torus); act = identity or
  leaky ReLU.
* Its exact input and weight gradients (the adjoint of a periodic
  correlation is the correlation with the reflected kernel).
* 2x2x2 average pooling, nearest 2x upsampling and their adjoints.
* Output head: a 1x1x1 convolution to the three velocity components (and,
  for the preconditioner head, a fourth channel: the weight's logit).
* Adam (bias-corrected first and second moments).
* The whole U-Net forward pass and its reverse-mode gradient.

Layout as in the CUDA path: activations channels-last [B, D, H, W, C];
conv weights [Cout, 27, Cin]; head weights [3, Cin]; velocity [B, 3, D, H, W].
Each layer's derivative here is pinned by finite differences, adjoint
identities and brute-force loops in tests/test_oracle_net_pins.py.
"""
from __future__ import annotations

import numpy as np

TAPS = [(kd - 1, kh - 1, kw - 1) for kd in range(3) for kh in range(3) for kw in range(3)]


def _f64(a):
    return np.asarray(a, dtype=np.float64)


def shift(x, off):
    """x[p + off] on the periodic grid (axes 1..3 of [B, D, H, W, C])."""
    return np.roll(x, shift=(-off[0], -off[1], -off[2]), axis=(1, 2, 3))


def leaky(y, slope):
    return np.where(y > 0, y, slope * y)


def conv3d(x, w, b=None, act=False, slope=0.1):
    """Periodic 3x3x3 correlation; returns the activated output."""
    x = _f64(x); w = _f64(w)
    y = np.zeros(x.shape[:4] + (w.shape[0],))
    for tap, off in enumerate(TAPS):
        y += shift(x, off) @ w[:, tap, :].T
    if b is not None:
        y += _f64(b)
    return leaky(y, slope) if act else y


def conv3d_input_grad(dy, w):
    """dx[q, ci] = sum_{tap, co} dy[q - off(tap), co] w[co, tap, ci]."""
    dy = _f64(dy); w = _f64(w)
    dx = np.zeros(dy.shape[:4] + (w.shape[2],))
    for tap, off in enumerate(TAPS):
        dx += shift(dy, (-off[0], -off[1], -off[2])) @ w[:, tap, :]
    return dx


def conv3d_weight_grad(x, dy):
    """dw[co, tap, ci] = sum_p dy[p, co] x[p + off(tap), ci]; db = sum_p dy."""
    x = _f64(x); dy = _f64(dy)
    cin, cout = x.shape[-1], dy.shape[-1]
    dyf = dy.reshape(-1, cout)
    dw = np.zeros((cout, 27, cin))
    for tap, off in enumerate(TAPS):
        dw[:, tap, :] = dyf.T @ shift(x, off).reshape(-1, cin)
    return dw, dyf.sum(axis=0)


def leaky_grad(dy, y, slope):
    """Gradient through the leaky ReLU, decided by the sign of its output."""
    return np.where(_f64(y) > 0, _f64(dy), slope * _f64(dy))


def pool2(x):
    x = _f64(x)
    B, D, H, W, C = x.shape
    return x.reshape(B, D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4, 6))


def pool2_adj(dy):
    dy = _f64(dy)
    return np.repeat(np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def up2(x):
    x = _f64(x)
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def up2_adj(dy):
    dy = _f64(dy)
    B, D, H, W, C = dy.shape
    return dy.reshape(B, D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4, 6))


def head(x, wh, bh, scale):
    """v[b, c] = scale (bh[c] + sum_ci x[b, ..., ci] wh[c, ci]), channels-first."""
    y = _f64(x) @ _f64(wh).T + _f64(bh)
    return scale * np.moveaxis(y, -1, 1)


def head_grad(x, wh, scale, dv):
    """Returns (dx, dwh, dbh) for the head."""
    g = scale * np.moveaxis(_f64(dv), 1, -1)          # [B, D, H, W, nout]
    dx = g @ _f64(wh)
    gf = g.reshape(-1, g.shape[-1])
    dwh = gf.T @ _f64(x).reshape(-1, _f64(x).shape[-1])
    return dx, dwh, gf.sum(axis=0)


def adam(w, g, m, s, lr, b1, b2, eps, step):
    """One bias-corrected Adam step; returns (w, m, s)."""
    m = b1 * _f64(m) + (1 - b1) * _f64(g)
    s = b2 * _f64(s) + (1 - b2) * _f64(g) ** 2
    mh = m / (1 - b1 ** step)
    sh = s / (1 - b2 ** step)
    return _f64(w) - lr * mh / (np.sqrt(sh) + eps), m, s


def pack(m0, m1, a0, a1, cin):
    """Network input [B, D, H, W, cin]: channels a0 m0, a1 m1, then zeros."""
    m0 = _f64(m0); m1 = _f64(m1)
    x = np.zeros(m0.shape + (cin,))
    x[..., 0] = a0 * m0
    x[..., 1] = a1 * m1
    return x


# ---------------------------------------------------------------------------
# U-Net
# ---------------------------------------------------------------------------

def unet_layers(chans=(16, 32, 64, 128), cin=16):
    """(name, Cin, Cout) of every 3x3x3 conv, in forward order."""
    L = len(chans)
    out = []
    prev = cin
    for l in range(L - 1):
        out += [("enc%da" % l, prev, chans[l]), ("enc%db" % l, chans[l], chans[l])]
        prev = chans[l]
    out += [("bota", prev, chans[-1]), ("botb", chans[-1], chans[-1])]
    for l in range(L - 2, -1, -1):
        out += [("dec%da" % l, chans[l] + chans[l + 1], chans[l]), ("dec%db" % l, chans[l], chans[l])]
    return out


def unet_forward(params, x, chans=(16, 32, 64, 128), slope=0.1, vscale=1.0):
    """Returns (v, cache).  params: dict name -> (w, b); 'head' -> (wh, bh)."""
    L = len(chans)
    cache = {"x": x}
    h = x
    skips = []
    for l in range(L - 1):
        a = conv3d(h, *params["enc%da" % l], act=True, slope=slope)
        e = conv3d(a, *params["enc%db" % l], act=True, slope=slope)
        cache["enc%da" % l] = (h, a)
        cache["enc%db" % l] = (a, e)
        skips.append(e)
        h = pool2(e)
    a = conv3d(h, *params["bota"], act=True, slope=slope)
    bo = conv3d(a, *params["botb"], act=True, slope=slope)
    cache["bota"] = (h, a)
    cache["botb"] = (a, bo)
    h = bo
    for l in range(L - 2, -1, -1):
        cat = np.concatenate([skips[l], up2(h)], axis=-1)
        a = conv3d(cat, *params["dec%da" % l], act=True, slope=slope)
        d = conv3d(a, *params["dec%db" % l], act=True, slope=slope)
        cache["dec%da" % l] = (cat, a)
        cache["dec%db" % l] = (a, d)
        h = d
    cache["head_in"] = h
    v = head(h, *params["head"], vscale)
    return v, cache


def unet_backward(params, cache, dv, chans=(16, 32, 64, 128), slope=0.1, vscale=1.0):
    """Reverse-mode gradient of <dv, v>: dict name -> (dw, db)."""
    L = len(chans)
    grads = {}
    dh, dwh, dbh = head_grad(cache["head_in"], params["head"][0], vscale, dv)
    grads["head"] = (dwh, dbh)

    def conv_back(name, dout):
        xin, y = cache[name]
        g = leaky_grad(dout, y, slope)
        dw, db = conv3d_weight_grad(xin, g)
        grads[name] = (dw, db)
        return conv3d_input_grad(g, params[name][0])

    dskip = [None] * (L - 1)
    for l in range(L - 1):
        dh = conv_back("dec%da" % l, conv_back("dec%db" % l, dh))
        c = chans[l]
        dskip[l] = dh[..., :c]
        dh = up2_adj(dh[..., c:])
    dh = conv_back("bota", conv_back("botb", dh))
    for l in range(L - 2, -1, -1):
        de = pool2_adj(dh) + dskip[l]
        dh = conv_back("enc%da" % l, conv_back("enc%db" % l, de))
    return grads
