"""Seeded synthetic inputs for the registration hot path.

This module only draws inputs: templates and velocities on the periodic grid
[0, 2 pi)^3 (C order, x3 fastest; vector fields component-major [3][N1][N2][N3]).
It holds none of the method's arithmetic (no transport, no interpolation, no
finite differences, no regularisation); the reference image m1 is made by
whichever transport the caller trusts.

Recipes (all float64, seeded with numpy's PCG64):

* ``blob_template``: sum of Gaussian blobs with periodic minimum-image
  distance (sigma 0.3, centres U[0, 2pi)^3, amplitudes U[0.5, 1]) plus
  0.2 sin x1 sin x2 sin x3, clipped to [0, 1].
* ``mode_velocity``: each component a sum of random Fourier modes
  a cos(k . x + phi) with integer wave vectors 1 <= |k|_2 <= kmax, scaled so
  that max_x |v(x)|_2 equals vmax.
* ``bandlimited_velocity``: random complex spectrum on the ball |k|_2 <= kmax,
  inverse real FFT, same max-norm scaling (fast at 256^3 and above).
* ``label_template``: four nested ellipsoidal label regions with
  intensities 0.2 / 0.5 / 0.8 / 1.0 on a zero background, smoothed by a
  periodic Gaussian of sigma = 1 voxel (separable, direct convolution).
* ``add_noise``: additive N(0, sigma^2) noise.
* ``syn_template`` / ``syn_velocity``: the paper's SYN recipe (Sec. 4,
  "SYN"): m0 is the sum of 10 indicator functions of star-shaped regions
  |x - x_i| <= |Y_l^m(theta + dtheta_i, phi + dphi_i)| (l = 8, m = 6;
  offsets x_i in [-0.4 pi, 0.4 pi]^3; angle perturbations in multiples of
  pi/2), so intensities are the integer overlap counts 0..10; the velocity is
  v_x = sum_k k^-1/2 cos(k y) cos(k x), v_y = sum_k k^-1/2 sin(k z) sin(k y),
  v_z = sum_k k^-1/2 cos(k x) cos(k z), k = 1..K.  Coordinates are the
  paper's (-pi, pi]^3 = our [0, 2 pi)^3 shifted by pi.  Reading of the
  garbled angle ranges: theta is the azimuth (the argument of e^{i m theta}),
  phi the polar angle (the argument of P_l^m(cos phi)).
* ``sphere_template``: three nested spheres (radii 2.0 / 1.4 / 0.8 scaled
  per axis by U[0.9, 1.1], centre pi + U[-0.2, 0.2]) with smooth edges
  (tanh, width 1.5 voxels) and intensities 0.3 / 0.6 / 0.9, plus a blob
  texture (8 periodic Gaussians, sigma 0.15, amplitude 0.1); returns the
  float32 image and the uint8 label map (0 background, 1 outer shell,
  2 middle shell, 3 core).  Evaluated slab by slab, so 1024^3 fits in a few
  GB of host memory.
"""
from __future__ import annotations

import math

import numpy as np


def coords(n):
    """1-D node coordinates x_c = i * 2 pi / N_c for each axis."""
    return [np.arange(int(s)) * (2.0 * math.pi / int(s)) for s in n]


def _scale_to_max(v, vmax):
    mx = float(np.sqrt(np.max(np.sum(v * v, axis=0))))
    return v * (vmax / mx) if mx > 0 else v


def blob_template(n, seed=0, nblobs=8, sigma=0.3, sine=0.2):
    rng = np.random.default_rng(seed)
    x1, x2, x3 = coords(n)
    cen = rng.uniform(0.0, 2.0 * math.pi, size=(nblobs, 3))
    amp = rng.uniform(0.5, 1.0, size=nblobs)
    m = np.zeros(tuple(int(s) for s in n))
    two_pi = 2.0 * math.pi

    def mi(x, c):  # periodic minimum-image distance along one axis
        d = np.abs(x - c)
        return np.minimum(d, two_pi - d)

    for b in range(nblobs):
        d1 = mi(x1, cen[b, 0]) ** 2
        d2 = mi(x2, cen[b, 1]) ** 2
        d3 = mi(x3, cen[b, 2]) ** 2
        r2 = d1[:, None, None] + d2[None, :, None] + d3[None, None, :]
        m += amp[b] * np.exp(-r2 / (2.0 * sigma * sigma))
    m += sine * (np.sin(x1)[:, None, None] * np.sin(x2)[None, :, None]
                 * np.sin(x3)[None, None, :])
    return np.clip(m, 0.0, 1.0)


def _wavevectors(kmax, rng, count):
    """`count` random integer wave vectors with 1 <= |k|_2 <= kmax."""
    ks = []
    r = int(math.floor(kmax))
    while len(ks) < count:
        k = rng.integers(-r, r + 1, size=3)
        kk = float(np.dot(k, k))
        if 1.0 <= kk <= kmax * kmax:
            ks.append(k)
    return np.array(ks, dtype=np.float64)


def mode_velocity(n, seed=0, nmodes=6, kmax=4, vmax=0.5):
    rng = np.random.default_rng(seed)
    x1, x2, x3 = coords(n)
    v = np.zeros((3,) + tuple(int(s) for s in n))
    for c in range(3):
        ks = _wavevectors(kmax, rng, nmodes)
        amps = rng.uniform(0.5, 1.0, size=nmodes)
        phis = rng.uniform(0.0, 2.0 * math.pi, size=nmodes)
        for k, a, ph in zip(ks, amps, phis):
            e = (np.exp(1j * k[0] * x1)[:, None, None] * np.exp(1j * k[1] * x2)[None, :, None]
                 * np.exp(1j * k[2] * x3)[None, None, :])
            v[c] += a * np.real(np.exp(1j * ph) * e)
    return _scale_to_max(v, vmax)


def bandlimited_velocity(n, seed=0, kmax=8, vmax=1.0):
    rng = np.random.default_rng(seed)
    n0, n1, n2 = (int(s) for s in n)
    k0 = np.fft.fftfreq(n0, 1.0 / n0)
    k1 = np.fft.fftfreq(n1, 1.0 / n1)
    k2 = np.fft.rfftfreq(n2, 1.0 / n2)
    kk = k0[:, None, None] ** 2 + k1[None, :, None] ** 2 + k2[None, None, :] ** 2
    mask = (kk >= 1.0) & (kk <= kmax * kmax)
    # keep the random draw small: only the band's index set is drawn
    idx = np.nonzero(mask)
    v = np.empty((3, n0, n1, n2))
    for c in range(3):
        spec = np.zeros((n0, n1, n2 // 2 + 1), dtype=np.complex128)
        cnt = idx[0].size
        spec[idx] = (rng.standard_normal(cnt) + 1j * rng.standard_normal(cnt)) / np.sqrt(1.0 + kk[idx])
        v[c] = np.fft.irfftn(spec, s=(n0, n1, n2), axes=(0, 1, 2))
    return _scale_to_max(v, vmax)


def _blur_axis(f, sigma, axis):
    r = int(math.ceil(4.0 * sigma))
    t = np.arange(-r, r + 1, dtype=np.float64)
    w = np.exp(-t * t / (2.0 * sigma * sigma))
    w /= w.sum()
    out = np.zeros_like(f)
    for s, ws in zip(range(-r, r + 1), w):
        out += ws * np.roll(f, s, axis=axis)
    return out


def label_template(n, seed=0, levels=(0.2, 0.5, 0.8, 1.0), blur_sigma=1.0):
    """Four nested ellipsoids (outermost first) centred near the domain centre."""
    rng = np.random.default_rng(seed)
    x1, x2, x3 = coords(n)
    c = math.pi + rng.uniform(-0.2, 0.2, size=3)
    radii0 = np.array([2.2, 1.9, 2.4]) * rng.uniform(0.9, 1.1, size=3)
    m = np.zeros(tuple(int(s) for s in n))
    for lvl, scale in zip(levels, (1.0, 0.75, 0.5, 0.28)):
        r = radii0 * scale
        q = (((x1 - c[0]) / r[0]) ** 2)[:, None, None] + (((x2 - c[1]) / r[1]) ** 2)[None, :, None] \
            + (((x3 - c[2]) / r[2]) ** 2)[None, None, :]
        m = np.where(q <= 1.0, lvl, m)
    for ax in range(3):
        m = _blur_axis(m, blur_sigma, ax)
    return m


def add_noise(f, sigma=0.02, seed=0):
    rng = np.random.default_rng(seed)
    return f + sigma * rng.standard_normal(f.shape)


def sphere_template(n, seed=0, radii=(2.0, 1.4, 0.8), levels=(0.3, 0.6, 0.9), width_vox=1.5, nblobs=8,
                    blob_sigma=0.15, blob_amp=0.1, slab=16):
    rng = np.random.default_rng(seed)
    n0, n1, n2 = (int(s) for s in n)
    x1, x2, x3 = coords(n)
    c = math.pi + rng.uniform(-0.2, 0.2, size=3)
    axes = rng.uniform(0.9, 1.1, size=3)
    cen = rng.uniform(0.0, 2.0 * math.pi, size=(nblobs, 3))
    w = width_vox * 2.0 * math.pi / min(n0, n1, n2)
    two_pi = 2.0 * math.pi

    def mi(x, cc):
        d = np.abs(x - cc)
        return np.minimum(d, two_pi - d)

    q2 = (((x2 - c[1]) / axes[1]) ** 2)[None, :, None]
    q3 = (((x3 - c[2]) / axes[2]) ** 2)[None, None, :]
    b2 = [(mi(x2, cen[b, 1]) ** 2)[None, :, None] for b in range(nblobs)]
    b3 = [(mi(x3, cen[b, 2]) ** 2)[None, None, :] for b in range(nblobs)]
    m = np.empty((n0, n1, n2), dtype=np.float32)
    lab = np.empty((n0, n1, n2), dtype=np.uint8)

    def fill(i0):
        xs = x1[i0:i0 + slab]
        r = np.sqrt((((xs - c[0]) / axes[0]) ** 2)[:, None, None] + q2 + q3)
        f = np.zeros(r.shape)
        L = np.zeros(r.shape, dtype=np.uint8)
        prev = 0.0
        for k, (R, lv) in enumerate(zip(radii, levels)):
            f += (lv - prev) * 0.5 * (1.0 + np.tanh((R - r) / w))
            prev = lv
            L[r <= R] = k + 1
        for b in range(nblobs):
            d1 = (mi(xs, cen[b, 0]) ** 2)[:, None, None]
            f += blob_amp * np.exp(-(d1 + b2[b] + b3[b]) / (2.0 * blob_sigma * blob_sigma))
        m[i0:i0 + slab] = f
        lab[i0:i0 + slab] = L

    # slabs are independent; numpy releases the interpreter lock inside the
    # array operations, so threads run them in parallel
    import concurrent.futures
    import os
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        list(ex.map(fill, range(0, n0, slab)))
    return m, lab


def _assoc_legendre(l, m, x):
    """P_l^m(x) with the Condon-Shortley phase, by the standard upward
    recurrence in l from P_m^m = (-1)^m (2m-1)!! (1-x^2)^(m/2)."""
    x = np.asarray(x, dtype=np.float64)
    pmm = np.ones_like(x)
    if m > 0:
        somx2 = np.sqrt(np.maximum(0.0, 1.0 - x * x))
        fact = 1.0
        for _ in range(m):
            pmm = -pmm * fact * somx2
            fact += 2.0
    if l == m:
        return pmm
    pmmp1 = x * (2 * m + 1) * pmm
    if l == m + 1:
        return pmmp1
    pll = pmmp1
    for ll in range(m + 2, l + 1):
        pll = ((2 * ll - 1) * x * pmmp1 - (ll + m - 1) * pmm) / (ll - m)
        pmm, pmmp1 = pmmp1, pll
    return pll


def syn_template(n, seed=0, l=8, m=6, count=10, slab=16):
    """The paper's SYN template (see the module docstring): float32 overlap counts 0..count."""
    rng = np.random.default_rng(seed)
    n0, n1, n2 = (int(s) for s in n)
    xs = [c - math.pi for c in coords(n)]  # (-pi, pi]-centred coordinates
    norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m) / math.factorial(l + m))
    off = rng.uniform(-0.4 * math.pi, 0.4 * math.pi, size=(count, 3))
    rng.integers(0, 4, size=count)  # the azimuth perturbations (no effect on |Y|), drawn for the seed sequence
    dph = rng.integers(0, 4, size=count) * (math.pi / 2)
    out = np.zeros((n0, n1, n2), dtype=np.float32)
    for i0 in range(0, n0, slab):
        x = xs[0][i0:i0 + slab][:, None, None]
        y = xs[1][None, :, None]
        z = xs[2][None, None, :]
        acc = np.zeros((x.shape[0], n1, n2))
        for i in range(count):
            dx, dy, dz = x - off[i, 0], y - off[i, 1], z - off[i, 2]
            r = np.sqrt(dx * dx + dy * dy + dz * dz)
            # |Y_l^m(theta + dtheta, phi + dphi)| = norm |P_l^m(cos(phi + dphi))|:
            # the azimuth enters only through |e^{i m theta}| = 1
            phi = np.arccos(np.clip(dz / np.maximum(r, 1e-300), -1.0, 1.0)) + dph[i]
            ylm = norm * np.abs(_assoc_legendre(l, m, np.cos(phi)))
            acc += (r <= ylm)
        out[i0:i0 + slab] = acc
    return out


def syn_velocity(n, K=4):
    """The paper's SYN velocity (see the module docstring), float64 [3, n0, n1, n2]."""
    xs = [c - math.pi for c in coords(n)]
    x = xs[0][:, None, None]
    y = xs[1][None, :, None]
    z = xs[2][None, None, :]
    shape = tuple(int(s) for s in n)
    v = np.zeros((3,) + shape)
    for k in range(1, K + 1):
        a = k ** -0.5
        v[0] += a * np.cos(k * y) * np.cos(k * x)
        v[1] += a * np.sin(k * z) * np.sin(k * y)
        v[2] += a * np.cos(k * x) * np.cos(k * z)
    return v
