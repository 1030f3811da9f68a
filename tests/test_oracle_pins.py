"""Pins of the FP64 oracle against facts fixed outside it: closed forms,
textbook constants, brute force, dot-product identities and convergence orders.

Each test names the part of the method it pins and the mistake it would catch.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2209_08189_gb300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "textbook_constants.json")))
TWO_PI = 2.0 * math.pi


def _xyz(n):
    x1, x2, x3 = synth.coords(n)
    return np.meshgrid(x1, x2, x3, indexing="ij")


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


# ---------------------------------------------------------------------------
# Interpolation (Sec. 3 "IP kernel"): cubic Lagrange / linear, periodic
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("t", ["0", "0.5", "0.25"])
def test_cubic_weights_match_textbook(t):
    """Catches wrong node offsets or a wrong cardinal polynomial."""
    n = (8, 8, 16)
    i0 = 6
    w = []
    for a in range(4):
        f = np.zeros(n)
        f[:, :, i0 - 1 + a] = 1.0
        y = np.array([[2.0], [3.0], [i0 + float(t)]])
        w.append(oracle.interp_points(f, y, 3)[0])
    assert np.allclose(w, GOLD["cubic_lagrange_weights"][t], atol=1e-15, rtol=0)


@pytest.mark.parametrize("order,deg", [(3, 3), (1, 1)])
def test_interp_exact_on_polynomials(order, deg):
    """Tensor-product polynomials of degree <= 3 (cubic) / <= 1 (linear) are
    reproduced exactly at points whose stencil does not wrap."""
    n = (12, 10, 14)
    rng = np.random.default_rng(1)
    I, J, K = np.meshgrid(*[np.arange(s, dtype=float) for s in n], indexing="ij")
    lo, hi = (1.0, 2.0) if order == 3 else (0.0, 1.0)
    y = np.stack([rng.uniform(lo, s - 1 - hi, size=200) for s in n])
    for a in range(deg + 1):
        for b in range(deg + 1):
            for c in range(deg + 1):
                f = (I / 7.0) ** a * (J / 5.0) ** b * (K / 9.0) ** c
                exact = (y[0] / 7.0) ** a * (y[1] / 5.0) ** b * (y[2] / 9.0) ** c
                got = oracle.interp_points(f, y, order)
                assert np.max(np.abs(got - exact)) < 1e-12


@pytest.mark.parametrize("order", [3, 1])
def test_interp_integer_shift_is_periodic_roll(order):
    """Integer displacements return grid values with periodic wrap."""
    n = (8, 6, 10)
    rng = np.random.default_rng(2)
    f = rng.standard_normal(n)
    d = np.zeros((3,) + n)
    d[0] += 3; d[1] -= 7; d[2] += 12
    got = oracle.interp(f, d, order)
    exp = np.roll(f, shift=(-3, 7, -12), axis=(0, 1, 2))
    assert np.array_equal(got, exp)


@pytest.mark.parametrize("order,expect", [(3, 16.0), (1, 4.0)])
def test_interp_convergence_order(order, expect):
    """Error on a smooth periodic function drops by 2^p per halving of h."""
    errs = []
    for N in (32, 64):
        n = (N, N, 8)
        X1, X2, X3 = _xyz(n)
        f = np.sin(X1) * np.cos(2 * X2) * np.sin(X3)
        d = np.full((3,) + n, 0.37)
        d[2] = 0.0  # x3 is not refined: keep it on the nodes
        got = oracle.interp(f, d, order)
        h = TWO_PI / N
        ex = np.sin(X1 + 0.37 * h) * np.cos(2 * (X2 + 0.37 * h)) * np.sin(X3)
        errs.append(np.max(np.abs(got - ex)))
    ratio = errs[0] / errs[1]
    assert 0.8 * expect < ratio < 1.25 * expect, ratio


@pytest.mark.parametrize("order,deg", [(3, 3), (1, 1)])
def test_interp_gradient_exact_on_polynomials(order, deg):
    """The interpolant's gradient reproduces the derivative of tensor-product
    polynomials of degree <= 3 (cubic) / <= 1 (linear) at non-wrapping points."""
    n = (12, 10, 14)
    rng = np.random.default_rng(9)
    I, J, K = np.meshgrid(*[np.arange(s, dtype=float) for s in n], indexing="ij")
    lo, hi = (1.0, 2.0) if order == 3 else (0.0, 1.0)
    ok = (I >= lo + 1) & (I <= n[0] - 2 - hi) & (J >= lo + 1) & (J <= n[1] - 2 - hi) & \
         (K >= lo + 1) & (K <= n[2] - 2 - hi)
    d = rng.uniform(-0.9, 0.9, size=(3,) + n)
    P = lambda x, y, z: (x / 7.0) ** deg * (y / 5.0) ** min(deg, 2) * (z / 9.0) ** 1
    dP = [lambda x, y, z: deg * x ** (deg - 1) / 7.0 ** deg * (y / 5.0) ** min(deg, 2) * (z / 9.0),
          lambda x, y, z: (x / 7.0) ** deg * min(deg, 2) * y ** (min(deg, 2) - 1) / 5.0 ** min(deg, 2) * (z / 9.0),
          lambda x, y, z: (x / 7.0) ** deg * (y / 5.0) ** min(deg, 2) / 9.0]
    got = oracle.interp_grad(P(I, J, K), d, order)
    Y = (I + d[0], J + d[1], K + d[2])
    for c in range(3):
        assert np.max(np.abs(got[c] - dP[c](*Y))[ok]) < 1e-11


@pytest.mark.parametrize("order", [3, 1, 4])
def test_transport_vjp_matches_finite_differences(order):
    """The exact discrete VJP of nt SL steps (image and velocity cotangents)
    agrees with central differences of the discrete forward map."""
    n = (12, 10, 14)
    rng = np.random.default_rng(0)
    m0 = synth.blob_template(n, seed=1, sigma=0.8)
    v = synth.mode_velocity(n, seed=2, vmax=0.6, kmax=2)
    p = oracle.Params(nt=3, order=order)
    gbar = rng.standard_normal(n)
    gm0, gv = oracle.transport_vjp(m0, v, gbar, p)
    L = lambda mm, vv: float(np.sum(gbar * oracle.transport(mm, vv, p)))
    vt = rng.standard_normal(v.shape)
    mt = rng.standard_normal(n)
    eps = 1e-6
    fdv = (L(m0, v + eps * vt) - L(m0, v - eps * vt)) / (2 * eps)
    fdm = (L(m0 + eps * mt, v) - L(m0 - eps * mt, v)) / (2 * eps)
    assert abs(fdv - np.sum(gv * vt)) <= 1e-7 * abs(fdv)
    assert abs(fdm - np.sum(gm0 * mt)) <= 1e-7 * abs(fdm)


def test_interp_transpose_dot_product():
    """<T x, y> = <x, T^T y> for the scatter transpose (DTO pin), wrapping points included."""
    n = (9, 8, 7)
    rng = np.random.default_rng(3)
    d = rng.uniform(-4, 4, size=(3,) + n)
    for order in (3, 1):
        x = rng.standard_normal(n)
        y = rng.standard_normal(n)
        lhs = np.sum(oracle.interp(x, d, order) * y)
        rhs = np.sum(x * oracle.interp_T(y, d, order))
        assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


# ---------------------------------------------------------------------------
# RK2 characteristics (Sec. 2.2)
# ---------------------------------------------------------------------------

def test_backtrace_constant_velocity_exact():
    n = (8, 10, 12)
    v = np.zeros((3,) + n)
    vel = np.array([0.3, -0.7, 1.1])
    for c in range(3):
        v[c] = vel[c]
    h = oracle.spacing(n)
    for sign in (+1, -1):
        d = oracle.backtrace(v, 0.25, sign, 3)
        for c in range(3):
            assert np.allclose(d[c], -sign * 0.25 * vel[c] / h[c], rtol=0, atol=1e-13)


def test_backtrace_shear_exact():
    """v = (a sin x2, 0, 0): x2 is invariant, so RK2 is exact."""
    n = (16, 24, 8)
    X1, X2, X3 = _xyz(n)
    a = 0.8
    v = np.stack([a * np.sin(X2), 0 * X2, 0 * X2])
    d = oracle.backtrace(v, 0.5, +1, 3)
    h = oracle.spacing(n)
    assert np.max(np.abs(d[0] + 0.5 * a * np.sin(X2) / h[0])) < 1e-12
    assert np.max(np.abs(d[1])) == 0 and np.max(np.abs(d[2])) == 0


def _flow_1d(x, s, a):
    """Exact flow of dx/dt = a sin x for time s: tan(y/2) = tan(x/2) e^{a s}."""
    return 2.0 * np.arctan(np.tan(x / 2.0) * np.exp(a * s))


def test_backtrace_1d_flow_local_third_order():
    """Heun's local error is O(dt^3) against the closed-form characteristic."""
    a = 1.0
    errs = []
    for dt in (0.2, 0.1):
        n = (256, 4, 4)
        X1, _, _ = _xyz(n)
        v = np.stack([a * np.sin(X1), 0 * X1, 0 * X1])
        d = oracle.backtrace(v, dt, +1, 3)
        x = X1[:, 0, 0]
        mask = np.abs(x - math.pi) > 0.3  # keep tan() away from its pole
        xd = x + d[0][:, 0, 0] * oracle.spacing(n)[0]
        exact = _flow_1d(x, -dt, a)
        diff = np.mod(xd - exact + math.pi, TWO_PI) - math.pi  # arctan branch: compare mod 2 pi
        errs.append(np.max(np.abs(diff)[mask]))
    assert 6.0 < errs[0] / errs[1] < 10.0, errs


# ---------------------------------------------------------------------------
# 8th-order finite differences (Sec. 2.2, Sec. 3 "FD kernel")
# ---------------------------------------------------------------------------

def test_fd8_coefficients_textbook():
    n = (16, 16, 16)
    f = np.zeros(n)
    f[0, 0, 0] = 1.0
    g = oracle.fd8_grad(f)
    scale = 16 / TWO_PI
    for axis in range(3):
        for s in range(1, 5):
            idx = [0, 0, 0]
            idx[axis] = s
            assert abs(g[axis][tuple(idx)] + GOLD["fd8_coefficients"][s - 1] * scale) < 1e-14


def test_fd8_modified_wavenumber():
    """On sin(k x + phi) the FD8 derivative is k~ cos(k x + phi), k~ = (2/h) sum c_s sin(s k h)."""
    n = (16, 12, 20)
    X = _xyz(n)
    c = [4 / 5, -1 / 5, 4 / 105, -1 / 280]
    k = (3, 5, 2)
    for axis in range(3):
        h = TWO_PI / n[axis]
        f = np.sin(k[axis] * X[axis] + 0.3)
        kt = (2.0 / h) * sum(c[s - 1] * math.sin(s * k[axis] * h) for s in range(1, 5))
        g = oracle.fd8_grad(f)
        assert np.max(np.abs(g[axis] - kt * np.cos(k[axis] * X[axis] + 0.3))) < 1e-12
        others = [e for e in range(3) if e != axis]
        assert all(np.max(np.abs(g[e])) < 1e-12 for e in others)
    v = np.stack([np.sin(2 * X[0]), np.cos(3 * X[1]), np.sin(X[2] + 1.0)])
    div = oracle.fd8_div(v)
    kt = [(2.0 / (TWO_PI / n[a])) * sum(c[s - 1] * math.sin(s * kk * TWO_PI / n[a]) for s in range(1, 5))
          for a, kk in zip(range(3), (2, 3, 1))]
    exp = kt[0] * np.cos(2 * X[0]) - kt[1] * np.sin(3 * X[1]) + kt[2] * np.cos(X[2] + 1.0)
    assert np.max(np.abs(div - exp)) < 1e-12


def test_fd8_eighth_order():
    errs = []
    for N in (24, 48):
        n = (N, 4, 4)
        X1, _, _ = _xyz(n)
        g = oracle.fd8_grad(np.sin(2 * X1))
        errs.append(np.max(np.abs(g[0] - 2 * np.cos(2 * X1))))
    r = errs[0] / errs[1]
    assert 190 < r < 330, r  # 2^8 = 256; a 6th-order stencil would give 64


# ---------------------------------------------------------------------------
# Spectral regularisation, preconditioner and K (Sec. 2.1, Eq. (3))
# ---------------------------------------------------------------------------

def _brute_force_S(v, p):
    """S v by explicit O(N^6) DFT over the full wavenumber grid (no FFT)."""
    n = v.shape[1:]
    N = int(np.prod(n))
    X = [x.ravel() for x in _xyz(n)]
    ks = [np.fft.fftfreq(s, 1.0 / s) for s in n]
    K0, K1, K2 = [k.ravel() for k in np.meshgrid(*ks, indexing="ij")]
    phase = np.exp(-1j * (np.outer(K0, X[0]) + np.outer(K1, X[1]) + np.outer(K2, X[2])))
    vh = np.stack([phase @ v[c].ravel() for c in range(3)])
    kk = K0 ** 2 + K1 ** 2 + K2 ** 2
    u = np.stack([np.where(np.abs(K0) == n[0] / 2, 0, K0), np.where(np.abs(K1) == n[1] / 2, 0, K1),
                  np.where(np.abs(K2) == n[2] / 2, 0, K2)])
    a = p.beta_v * (kk if p.reg == 1 else kk ** 2)
    c = p.beta_w * (1 + kk)
    sh = a * vh + c * u * np.sum(u * vh, axis=0)
    out = np.stack([(phase.conj().T @ sh[cc]) / N for cc in range(3)])
    assert np.max(np.abs(out.imag)) < 1e-10
    return out.real.reshape((3,) + n)


@pytest.mark.parametrize("reg", [1, 2])
def test_reg_apply_matches_brute_force_dft(reg):
    n = (6, 8, 4)
    rng = np.random.default_rng(4)
    v = rng.standard_normal((3,) + n)
    p = oracle.Params(beta_v=0.3, beta_w=0.07, reg=reg)
    assert _rel(oracle.reg_apply(v, p), _brute_force_S(v, p)) < 1e-13


def test_reg_single_mode_closed_form():
    """S on v = e_c cos(k.x): beta_v |k|^2 v + beta_w (1+|k|^2) k k_c cos(k.x)."""
    n = (16, 16, 16)
    X = _xyz(n)
    k = np.array([2.0, -3.0, 1.0])
    ph = k[0] * X[0] + k[1] * X[1] + k[2] * X[2]
    p = oracle.Params(beta_v=0.5, beta_w=0.2)
    kk = float(k @ k)
    for c in range(3):
        v = np.zeros((3,) + n)
        v[c] = np.cos(ph)
        exp = p.beta_v * kk * v + p.beta_w * (1 + kk) * k[:, None, None, None] * k[c] * np.cos(ph)[None]
        assert np.max(np.abs(oracle.reg_apply(v, p) - exp)) < 1e-11


def test_reg_energy_closed_form():
    """v = (sin(k x1), 0, 0): beta_v/2 int|grad v|^2 + beta_w/2 int(|grad w|^2 + w^2), w = div v."""
    n = (16, 8, 8)
    X = _xyz(n)
    kx = 3.0
    v = np.stack([np.sin(kx * X[0]), 0 * X[0], 0 * X[0]])
    p = oracle.Params(beta_v=0.4, beta_w=0.1)
    vol = TWO_PI ** 3
    exact = 0.5 * p.beta_v * kx ** 2 * vol / 2 + 0.5 * p.beta_w * (kx ** 4 + kx ** 2) * vol / 2
    assert abs(oracle.reg_energy(v, p) - exact) < 1e-10 * exact


def test_reg_symmetric_and_inverse():
    n = (8, 10, 6)
    rng = np.random.default_rng(5)
    u = rng.standard_normal((3,) + n)
    w = rng.standard_normal((3,) + n)
    for reg in (1, 2):
        p = oracle.Params(beta_v=0.05, beta_w=0.3, reg=reg)
        a = oracle.inner(oracle.reg_apply(u, p), w, n)
        b = oracle.inner(u, oracle.reg_apply(w, p), n)
        assert abs(a - b) < 1e-13 * max(abs(a), 1)
        um = u - u.mean(axis=(1, 2, 3), keepdims=True)  # k = 0 is not inverted
        assert _rel(oracle.reg_inverse(oracle.reg_apply(um, p), p), um) < 1e-12
        assert _rel(oracle.reg_apply(oracle.reg_inverse(um, p), p), um) < 1e-12
        # k = 0 passes through the preconditioner unchanged
        const = np.ones((3,) + n) * np.array([1.0, -2.0, 0.5])[:, None, None, None]
        assert np.allclose(oracle.reg_inverse(const, p), const, atol=1e-13)


def test_K_limits_and_identity():
    n = (8, 8, 8)
    rng = np.random.default_rng(6)
    b = rng.standard_normal((3,) + n)
    # beta_w -> 0: K -> I
    assert _rel(oracle.project_K(b, oracle.Params(beta_v=1.0, beta_w=1e-14)), b) < 1e-12
    # beta_w -> infinity: K b is divergence free (spectral divergence with the odd symbol)
    Kb = oracle.project_K(b, oracle.Params(beta_v=1.0, beta_w=1e12))
    kh = np.fft.rfftn(Kb, axes=(1, 2, 3))
    ks = [np.fft.fftfreq(8, 1 / 8), np.fft.fftfreq(8, 1 / 8), np.fft.rfftfreq(8, 1 / 8)]
    K = np.meshgrid(*ks, indexing="ij")
    u = [np.where(np.abs(K[c]) == 4, 0, K[c]) for c in range(3)]
    divh = sum(u[c] * kh[c] for c in range(3))
    assert np.max(np.abs(divh)) < 1e-9 * np.max(np.abs(kh))
    # K S = beta_v A (a I): the two gradient forms share stationary points
    p = oracle.Params(beta_v=0.02, beta_w=0.5)
    lhs = oracle.project_K(oracle.reg_apply(b, p), p)
    rhs = oracle.reg_apply(b, oracle.Params(beta_v=0.02, beta_w=0.0))
    assert _rel(lhs, rhs) < 1e-12


def test_k_form_preconditioner_single_modes():
    """Preconditioner of the paper's gradient form (grad_form = 1): on
    v = e_c cos(k.x) it divides by beta_v |k|^2 (H1) or beta_v |k|^4 (H2),
    whatever the direction of e_c relative to k and whatever beta_w; the k = 0
    mode passes unchanged.  Returning S^{-1} instead would divide the
    longitudinal part by beta_v |k|^2 + beta_w (1 + |k|^2) |k|^2."""
    n = (16, 12, 10)
    X = _xyz(n)
    k = np.array([2.0, -3.0, 1.0])
    ph = k[0] * X[0] + k[1] * X[1] + k[2] * X[2]
    kk = float(k @ k)
    for reg, sym in ((1, kk), (2, kk * kk)):
        p = oracle.Params(beta_v=0.05, beta_w=0.4, reg=reg, grad_form=1)
        for e in (np.array([1.0, 0, 0]), k / math.sqrt(kk), np.array([3.0, 2.0, 0.0]) / math.sqrt(13.0)):
            v = e[:, None, None, None] * np.cos(ph)[None]
            assert np.max(np.abs(oracle.precond(v, p) - v / (p.beta_v * sym))) < 1e-12
        const = np.ones((3,) + n) * np.array([0.7, -1.1, 0.2])[:, None, None, None]
        assert np.max(np.abs(oracle.precond(const, p) - const)) < 1e-13
    # the exact form's S^{-1} differs on the longitudinal mode when beta_w > 0
    p0 = oracle.Params(beta_v=0.05, beta_w=0.4, grad_form=0)
    vl = (k / math.sqrt(kk))[:, None, None, None] * np.cos(ph)[None]
    expect0 = vl / (p0.beta_v * kk + p0.beta_w * (1 + kk) * kk)
    assert np.max(np.abs(oracle.precond(vl, p0) - expect0)) < 1e-12


def test_k_form_preconditioner_inverts_K_S():
    """K S = beta_v A, so the K-form preconditioner applied to K(S x) gives x
    back up to its mean (k = 0 is not inverted), for H1 and H2, and with
    beta_w = 0 (K = I) it inverts S itself."""
    n = (8, 10, 6)
    rng = np.random.default_rng(12)
    x = rng.standard_normal((3,) + n)
    xm = x - x.mean(axis=(1, 2, 3), keepdims=True)
    for reg in (1, 2):
        p = oracle.Params(beta_v=0.03, beta_w=0.6, reg=reg, grad_form=1)
        y = oracle.precond(oracle.project_K(oracle.reg_apply(x, p), p), p)
        assert _rel(y, xm) < 1e-12
        p0 = oracle.Params(beta_v=0.03, beta_w=0.0, reg=reg, grad_form=1)
        assert _rel(oracle.precond(oracle.reg_apply(x, p0), p0), xm) < 1e-12


# ---------------------------------------------------------------------------
# Semi-Lagrangian solves (Eqs. (1b)-(1c), (4))
# ---------------------------------------------------------------------------

def test_transport_integer_shift_exact():
    """Constant v with dt v / h integral per axis: transport is a periodic roll."""
    n = (16, 12, 8)
    m0 = synth.blob_template(n, seed=3)
    h = oracle.spacing(n)
    p = oracle.Params(nt=4)
    shift = np.array([2, -1, 3])  # cells per time step
    v = np.zeros((3,) + n)
    for c in range(3):
        v[c] = shift[c] * h[c] / p.dt
    m1 = oracle.transport(m0, v, p)
    exp = np.roll(m0, shift=tuple(4 * shift), axis=(0, 1, 2))
    assert np.max(np.abs(m1 - exp)) < 1e-13


def test_transport_constant_velocity_vs_spectral_shift():
    """Non-integer constant shift: the error against the exact shift stays within
    the cubic Lagrange bound nt * Lambda^2 * sum_c (9/16)/4! h_c^4 max|d_c^4 m0|
    (Lambda = 5/4, the Lebesgue constant of the 4-node stencil) and shrinks fast."""
    errs = []
    for N in (16, 32):
        n = (N, N, N)
        X = _xyz(n)
        m0 = np.sin(X[0]) * np.cos(X[1] + 0.4) + 0.5 * np.sin(2 * X[2])
        vel = np.array([0.3, -0.21, 0.17])
        v = np.stack([np.full(n, vel[c]) for c in range(3)])
        p = oracle.Params(nt=2)
        m1 = oracle.transport(m0, v, p)
        exact = np.sin(X[0] - vel[0]) * np.cos(X[1] - vel[1] + 0.4) + 0.5 * np.sin(2 * (X[2] - vel[2]))
        err = np.max(np.abs(m1 - exact))
        h4 = (TWO_PI / N) ** 4
        bound = p.nt * 1.25 ** 2 * (9.0 / 16.0) / 24.0 * h4 * (1.0 + 1.0 + 0.5 * 16.0)
        assert err <= bound, (err, bound)
        errs.append(err)
    assert errs[0] / errs[1] > 8.0, errs


def _dflow(x, s, a):
    """d/dx of the exact 1-D flow map."""
    t = np.tan(x / 2.0)
    e = math.exp(a * s)
    return e * (1 + t * t) / (1 + (t * e) ** 2)


def test_state_and_adjoint_1d_flow_closed_form():
    """v = (a sin x1, 0, 0): m(x,1) = m0(phi_{-1}(x)); lambda(x,0) = lambda1(phi_1(x)) phi_1'(x).
    Errors shrink at second order in dt (fine grid)."""
    a = 0.6
    es, ea = [], []
    for nt in (4, 8):
        n = (256, 4, 4)
        X1 = _xyz(n)[0]
        v = np.stack([a * np.sin(X1), 0 * X1, 0 * X1])
        m0 = np.exp(np.cos(X1))
        p = oracle.Params(nt=nt)
        m1 = oracle.transport(m0, v, p)
        exm = np.exp(np.cos(_flow_1d(X1, -1.0, a)))
        lam1 = np.cos(X1) + 0.3 * np.sin(2 * X1)
        lam0 = oracle.transport(lam1, v, p, direction="adj")
        y = _flow_1d(X1, 1.0, a)
        exl = (np.cos(y) + 0.3 * np.sin(2 * y)) * _dflow(X1, 1.0, a)
        x = X1[:, 0, 0]
        mask = np.abs(x - math.pi) > 0.2
        es.append(np.max(np.abs(m1 - exm)[mask]))
        ea.append(np.max(np.abs(lam0 - exl)[mask]))
    assert 3.0 < es[0] / es[1] < 5.5, es
    assert 3.0 < ea[0] / ea[1] < 5.5, ea


def test_adjoint_conservation_and_adjoint_error():
    """Eq. (4) is conservative: sum lambda(0) = sum lambda(1) up to the time
    error, which shrinks with n_t on a resolved field; the forward-then-backward
    'adjoint error' (Sec. 3, n_t) shrinks with h."""
    adj_err = []
    for N in (16, 32):
        n = (N, N, N)
        X = _xyz(n)
        v = synth.mode_velocity(n, seed=1, kmax=2, vmax=0.5)
        lam1 = 1 + 0.5 * np.sin(X[0]) * np.cos(X[1]) * np.sin(X[2] + 0.3)
        gaps = []
        for nt in (2, 4, 8):
            p = oracle.Params(nt=nt)
            lam0 = oracle.transport(lam1, v, p, direction="adj")
            gaps.append(abs(lam0.sum() - lam1.sum()) / abs(lam1.sum()))
        p = oracle.Params(nt=4)
        back = oracle.transport(oracle.transport(lam1, v, p), -v, p)
        adj_err.append(np.linalg.norm(back - lam1) / np.linalg.norm(lam1))
    assert gaps[0] > 3 * gaps[1] > 9 * gaps[2] and gaps[2] < 1e-5, gaps
    assert adj_err[1] < adj_err[0] / 6, adj_err


# ---------------------------------------------------------------------------
# Gradient and Gauss-Newton Hessian (Eqs. (3), (6))
# ---------------------------------------------------------------------------

def _problem(N, nt=4, seed=0, vmax=0.5, smooth=False):
    """Template, known velocity v* and m1 = T(v*) m0.  smooth=True uses a
    trigonometric template (no clipping kinks) and |k| <= 2 velocities, so that
    consistency gaps show the scheme's order instead of the data's kinks."""
    n = (N, N, N)
    if smooth:
        X = _xyz(n)
        m0 = 0.5 + 0.3 * np.sin(X[0]) * np.cos(X[1] + 0.5) * np.sin(X[2] + 1.0) \
            + 0.2 * np.cos(2 * X[0] + X[2])
        vs = synth.mode_velocity(n, seed=seed + 10, vmax=vmax, kmax=2)
    else:
        m0 = synth.blob_template(n, seed=seed)
        vs = synth.mode_velocity(n, seed=seed + 10, vmax=vmax)
    p = oracle.Params(nt=nt, beta_v=1e-2, beta_w=1e-4)
    m1 = oracle.transport(m0, vs, p)
    return n, m0, m1, vs, p


def test_zero_residual_gradient_is_regulariser():
    """m1 = T(v*) m0: at v = v* the adjoint vanishes and g = S v* exactly."""
    n, m0, m1, vs, p = _problem(12)
    st = oracle.State(vs, m0, m1, p)
    assert st.mismatch == 0.0
    assert np.array_equal(oracle.gradient(st), oracle.reg_apply(vs, p))


def test_dto_hessian_symmetric_and_spd():
    """With the exact (scatter) transpose, H = S + L^T L: <Hx,y> = <x,Hy> to 1e-10."""
    n, m0, m1, vs, p = _problem(10, nt=3)
    st = oracle.State(0.5 * vs, m0, m1, p)
    rng = np.random.default_rng(7)
    x = rng.standard_normal((3,) + n)
    y = rng.standard_normal((3,) + n)
    hx = oracle.hessian_matvec(st, x, mode="scatter")
    hy = oracle.hessian_matvec(st, y, mode="scatter")
    a, b = oracle.inner(hx, y, n), oracle.inner(x, hy, n)
    assert abs(a - b) <= 1e-10 * max(abs(a), abs(b))
    assert oracle.inner(hx, x, n) > 0
    # L^T is the transpose of L: <L x, r> = <x, L^T r>
    r = rng.standard_normal(n)
    Lx = oracle.incremental_state(st, x)
    LTr, _ = oracle.adjoint_solve(-r, st.ch, st.gms, p, mode="scatter")
    lhs = oracle.inner(Lx, r, n)
    rhs = oracle.inner(x, LTr, n)  # L^T r is the body of a scatter adjoint started from -r
    assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), 1e-30)


def test_otd_matvec_approaches_dto_under_refinement():
    """The paper's SL adjoint (OTD) differs from the exact transpose only by
    discretisation error, which shrinks as h and dt shrink."""
    gaps = []
    for N, nt in ((12, 2), (24, 4)):
        n, m0, m1, vs, p = _problem(N, nt=nt, smooth=True)
        st = oracle.State(0.5 * vs, m0, m1, p)
        x = synth.mode_velocity(n, seed=99, vmax=0.3, kmax=2)
        otd = oracle.hessian_matvec(st, x, mode="sl") - oracle.reg_apply(x, p)
        dto = oracle.hessian_matvec(st, x, mode="scatter") - oracle.reg_apply(x, p)
        gaps.append(_rel(otd, dto))
    assert gaps[1] < 0.5 * gaps[0] and gaps[1] < 0.02, gaps


def test_gradient_consistent_with_objective():
    """<g, vt> vs a central difference of J: the OTD gap shrinks under refinement
    (a dropped term or flipped sign would leave an O(1) gap)."""
    gaps = []
    for N, nt in ((12, 2), (24, 4)):
        n, m0, m1, vs, p = _problem(N, nt=nt, smooth=True)
        v = 0.4 * vs
        st = oracle.State(v, m0, m1, p)
        g = oracle.gradient(st)
        vt = synth.mode_velocity(n, seed=55, vmax=0.3, kmax=2)
        eps = 1e-4
        jp = oracle.objective(v + eps * vt, m0, m1, p)[0]
        jm = oracle.objective(v - eps * vt, m0, m1, p)[0]
        fd = (jp - jm) / (2 * eps)
        gaps.append(abs(oracle.inner(g, vt, n) - fd) / abs(fd))
    assert gaps[1] < 0.35 * gaps[0] and gaps[1] < 0.05, gaps


def test_incremental_state_is_linearised_state():
    """L vt vs a central difference of m(1) along vt, shrinking under refinement."""
    gaps = []
    for N, nt in ((12, 2), (24, 4)):
        n, m0, m1, vs, p = _problem(N, nt=nt, smooth=True)
        v = 0.4 * vs
        st = oracle.State(v, m0, m1, p)
        vt = synth.mode_velocity(n, seed=56, vmax=0.3, kmax=2)
        eps = 1e-4
        fd = (oracle.transport(m0, v + eps * vt, p) - oracle.transport(m0, v - eps * vt, p)) / (2 * eps)
        gaps.append(_rel(oracle.incremental_state(st, vt), fd))
    assert gaps[1] < 0.35 * gaps[0] and gaps[1] < 0.05, gaps


def test_gauss_newton_hessian_matches_gradient_difference_at_zero_residual():
    """At zero residual the full Hessian equals the GN Hessian; compare with a
    central difference of the gradient; the gap shrinks under refinement."""
    gaps = []
    for N, nt in ((12, 2), (24, 4)):
        n, m0, m1, vs, p = _problem(N, nt=nt, smooth=True)
        st = oracle.State(vs, m0, m1, p)
        vt = synth.mode_velocity(n, seed=57, vmax=0.3, kmax=2)
        eps = 1e-4
        gp = oracle.gradient(oracle.State(vs + eps * vt, m0, m1, p))
        gm = oracle.gradient(oracle.State(vs - eps * vt, m0, m1, p))
        gaps.append(_rel(oracle.hessian_matvec(st, vt), (gp - gm) / (2 * eps)))
    assert gaps[1] < 0.35 * gaps[0] and gaps[1] < 0.01, gaps


def test_k_form_is_K_times_exact_form():
    n, m0, m1, vs, p = _problem(10, nt=2)
    st = oracle.State(0.3 * vs, m0, m1, p)
    pk = oracle.Params(**{**p.__dict__, "grad_form": 1})
    stk = oracle.State(0.3 * vs, m0, m1, pk)
    g = oracle.gradient(st)
    assert _rel(oracle.gradient(stk), oracle.project_K(g, p)) < 1e-12
    x = synth.mode_velocity(n, seed=3, vmax=0.2)
    assert _rel(oracle.hessian_matvec(stk, x), oracle.project_K(oracle.hessian_matvec(st, x), p)) < 1e-12


# ---------------------------------------------------------------------------
# Gauss-Newton-Krylov (Eq. (5)), metrics, Jacobian determinant
# ---------------------------------------------------------------------------

def test_registration_recovers_synthetic_velocity():
    """Known v*: the solver drives r << 1, J monotone, J(v) <= J(v*) + tol."""
    n, m0, m1, vs, p = _problem(16, nt=4)
    p.beta_v, p.beta_w = 1e-4, 1e-6
    p.gtol, p.max_gn, p.max_pcg = 1e-2, 20, 30
    v, rep = oracle.register(m0, m1, p)
    assert rep["status"] == "converged"
    assert all(b <= a for a, b in zip(rep["J"], rep["J"][1:]))
    assert rep["r"] < 0.01
    Jstar = oracle.State(vs, m0, m1, p).J
    assert rep["J"][-1] <= Jstar + 1e-3 * abs(Jstar)
    # relative residual is 1 at v = 0
    st0 = oracle.State(np.zeros_like(vs), m0, m1, p)
    assert abs(2 * st0.mismatch / oracle.inner(m0 - m1, m0 - m1, n) - 1.0) < 1e-14


def test_large_beta_gives_small_velocity():
    n, m0, m1, vs, p = _problem(12, nt=2)
    p.beta_v = 1e3
    v, rep = oracle.register(m0, m1, p)
    # the mean (k = 0 translation) is not regularised; everything else vanishes
    vz = v - v.mean(axis=(1, 2, 3), keepdims=True)
    assert np.max(np.abs(vz)) < 1e-3 * np.max(np.abs(vs))


def test_detj_closed_forms():
    n = (16, 16, 16)
    X = _xyz(n)
    p = oracle.Params(nt=4)
    vc = np.stack([np.full(n, 0.3), np.full(n, -0.2), np.full(n, 0.45)])
    assert np.max(np.abs(oracle.detj(vc, p) - 1.0)) < 1e-12
    shear = np.stack([0.7 * np.sin(X[1]), 0 * X[0], 0 * X[0]])
    assert np.max(np.abs(oracle.detj(shear, p) - 1.0)) < 1e-12
    # 1-D sin flow: det = d phi_{-1} / dx (closed form), converging with nt
    errs = []
    for nt in (4, 8):
        n1 = (256, 4, 4)
        X1 = _xyz(n1)[0]
        v = np.stack([0.6 * np.sin(X1), 0 * X1, 0 * X1])
        dj = oracle.detj(v, oracle.Params(nt=nt))
        ex = _dflow(X1, -1.0, 0.6)
        mask = np.abs(X1[:, 0, 0] - math.pi) > 0.2
        errs.append(np.max(np.abs(dj - ex)[mask]))
    assert 3.0 < errs[0] / errs[1] < 5.5, errs


def test_cfl_scales_with_time_step():
    """CFL = max |v|_2 dt / min h is proportional to dt = 1/n_t."""
    n = (32, 32, 32)
    v = synth.mode_velocity(n, seed=0, vmax=0.5)
    c4 = oracle.cfl(v, oracle.Params(nt=4))
    c16 = oracle.cfl(v, oracle.Params(nt=16))
    assert abs(c4 / c16 - 4.0) < 1e-12


def test_cfl_closed_forms_non_cubic_grid():
    """CFL on a non-cubic grid, where the smallest and the largest spacing
    differ: (i) a constant field gives |v|_2 dt / min h exactly; (ii) a field
    whose largest Euclidean norm sits where no component is largest: a
    largest-component reading, or the largest spacing, gives another value."""
    n = (16, 24, 40)
    hmin = 2 * math.pi / 40
    p = oracle.Params(nt=4)
    v = np.stack([np.full(n, 0.3), np.full(n, -0.4), np.full(n, 1.2)])
    assert abs(oracle.cfl(v, p) - 1.3 * 0.25 / hmin) < 1e-12
    w = np.zeros((3,) + n)
    w[0, 2, 3, 4] = 1.0           # largest component, |w| = 1
    w[:, 9, 1, 30] = (0.8, 0.8, 0.0)  # |w| = 0.8 sqrt 2 = 1.1314 > 1
    expect = 0.8 * math.sqrt(2.0) * 0.25 / hmin
    assert abs(oracle.cfl(w, p) - expect) < 1e-12
    assert abs(1.0 * 0.25 / hmin - expect) > 0.1 * expect             # max-component reading
    assert abs(0.8 * math.sqrt(2.0) * 0.25 / (2 * math.pi / 16) - expect) > 0.5 * expect  # largest h


def test_dice_closed_forms():
    """Dice of Sec. 4.1 on sets whose overlap is known by counting: equal sets
    1, disjoint 0, two boxes of 8x8x8 and 8x8x4 voxels sharing 8x8x4 -> 2/3,
    a threshold value itself counts as inside, both empty -> 1."""
    n = (16, 16, 16)
    a = np.zeros(n); b = np.zeros(n)
    a[0:8, 0:8, 0:8] = 1.0
    assert oracle.dice(a, a) == 1.0
    b[8:16, 8:16, 8:16] = 1.0
    assert oracle.dice(a, b) == 0.0
    b[:] = 0.0
    b[0:8, 0:8, 4:8] = 0.9
    assert abs(oracle.dice(a, b) - 2.0 * 256 / (512 + 256)) < 1e-15
    c = np.full(n, 0.5)
    assert oracle.dice(c, c) == 1.0 and oracle.dice(c, a) == 2.0 * 512 / (4096 + 512)
    assert oracle.dice(np.zeros(n), np.full(n, 0.49)) == 1.0


def test_generators_deterministic():
    n = (8, 8, 8)
    a = synth.blob_template(n, seed=0)
    b = synth.blob_template(n, seed=0)
    assert np.array_equal(a, b) and 0 <= a.min() and a.max() <= 1
    v1 = synth.mode_velocity(n, seed=0, vmax=0.5)
    assert abs(np.sqrt(np.max(np.sum(v1 * v1, axis=0))) - 0.5) < 1e-12
    v2 = synth.bandlimited_velocity((16, 16, 16), seed=0, kmax=4, vmax=1.0)
    assert abs(np.sqrt(np.max(np.sum(v2 * v2, axis=0))) - 1.0) < 1e-12


# ---------------------------------------------------------------------------
# Regularisation-parameter search and continuation (Sec. 3)
# ---------------------------------------------------------------------------

def _search_problem():
    n = (16, 16, 16)
    m0 = synth.blob_template(n, seed=3, sigma=0.6)
    vs = synth.mode_velocity(n, seed=4, kmax=2, vmax=1.2)
    p = oracle.Params(nt=4, beta_v=1e-2, beta_w=1e-4, gtol=5e-2, max_gn=10, max_pcg=10)
    return m0, oracle.transport(m0, vs, p), p


def test_param_search_follows_the_schedule():
    """Decades of beta_v until the Jacobian bounds break, bisection between
    the last valid and the breaching value down to 10 %, then decades of
    beta_w while valid; the selected pair is valid."""
    m0, m1, p = _search_problem()
    bv, bw, v, trace = oracle.param_search(m0, m1, p, jmin=0.5, max_solves=20)
    assert trace[0][:2] == (1.0, 1e-5)
    k = 0
    while trace[k][2]:  # stage (i): factors of 10 while valid
        assert abs(trace[k + 1][0] - trace[k][0] / 10) < 1e-15
        k += 1
    hi, lo = trace[k - 1][0], trace[k][0]
    k += 1
    while k < len(trace) and trace[k][1] == 1e-5:  # bisection
        assert abs(trace[k][0] - 0.5 * (hi + lo)) < 1e-15
        hi, lo = (trace[k][0], lo) if trace[k][2] else (hi, trace[k][0])
        k += 1
    assert hi == bv and (hi - lo) <= 0.1 * hi
    for tb, tw, ok in trace[k:]:  # stage (ii)
        assert tb == bv and tw < 1e-5
    q = oracle.Params(**{**p.__dict__, "beta_v": bv, "beta_w": bw})
    dj = oracle.detj(v, q)
    assert dj.min() >= 0.5 and dj.max() <= 2.0


def test_param_continuation_steps():
    m0, m1, p = _search_problem()
    v, steps = oracle.param_continuation(m0, m1, p, 0.03, 1e-7)
    assert steps == [(1.0, 1e-5), (0.1, 1e-5), (0.03, 1e-5), (0.03, 1e-6), (0.03, 1e-7)] or \
        [(round(a, 12), round(b, 14)) for a, b in steps] == [(1.0, 1e-5), (0.1, 1e-5), (0.03, 1e-5), (0.03, 1e-6),
                                                              (0.03, 1e-7)]


# ---------------------------------------------------------------------------
# Cubic B-spline interpolation (Sec. 3, IP kernel alternative)
# ---------------------------------------------------------------------------

def test_bspline_interpolates_grid_values_and_shifts():
    """Prefiltered B-spline interpolation returns the grid values at integer
    displacements (interpolating spline), wrap included."""
    rng = np.random.default_rng(11)
    n = (8, 10, 12)
    f = rng.standard_normal(n)
    d = np.zeros((3,) + n)
    d[0], d[1], d[2] = 2.0, -3.0, 5.0
    ref = np.roll(f, shift=(-2, 3, -5), axis=(0, 1, 2))
    assert np.max(np.abs(oracle.interp(f, d, 4) - ref)) < 1e-12


def test_bspline_half_node_closed_form():
    """At a half-node shift the interpolant of cos(k x1) is cos(k (x1 + h/2))
    times R(k) = [23 cos(kh/2) + cos(3kh/2)] / 24 / ((2 + cos kh) / 3), from
    beta(1/2) = 23/48 and beta(3/2) = 1/48 over the spline symbol."""
    n = (16, 4, 4)
    h = oracle.spacing(n)[0]
    x1 = np.arange(n[0]) * h
    for k in (1, 3, 5):
        f = np.cos(k * x1)[:, None, None] * np.ones(n)
        d = np.zeros((3,) + n)
        d[0] = 0.5
        R = (23 * math.cos(k * h / 2) + math.cos(3 * k * h / 2)) / 24.0 / ((2 + math.cos(k * h)) / 3.0)
        ref = R * np.cos(k * (x1 + h / 2))[:, None, None] * np.ones(n)
        assert np.max(np.abs(oracle.interp(f, d, 4) - ref)) < 1e-12


def test_bspline_fourth_order_convergence_and_transpose():
    errs = []
    for N in (16, 32):
        n = (N, 4, 4)
        x1 = np.arange(N) * (2 * math.pi / N)
        f = np.sin(2 * x1)[:, None, None] * np.ones(n)
        d = np.zeros((3,) + n)
        d[0] = 0.37
        y = x1 + 0.37 * 2 * math.pi / N
        errs.append(np.max(np.abs(oracle.interp(f, d, 4) - np.sin(2 * y)[:, None, None])))
    assert 12 < errs[0] / errs[1] < 20
    rng = np.random.default_rng(12)
    n = (9, 8, 7)
    d = rng.uniform(-3, 3, size=(3,) + n)
    x = rng.standard_normal(n)
    yv = rng.standard_normal(n)
    lhs = np.sum(oracle.interp(x, d, 4) * yv)
    assert abs(lhs - np.sum(x * oracle.interp_T(yv, d, 4))) < 1e-11 * max(1.0, abs(lhs))


# ---------------------------------------------------------------------------
# Zero-velocity Hessian and the two-level preconditioner (Sec. 2.2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("grad_form", [0, 1])
def test_zero_velocity_hessian_is_the_full_matvec_at_zero_velocity(grad_form):
    """At v = 0 the characteristics are the identity, so the full Gauss-Newton
    matvec (incremental state and adjoint solves, trapezoid body) must equal
    S vt + gbar (gbar . vt).  Catches a wrong sign, a missing time weight or a
    missing K in the zero-velocity operator."""
    g = (12, 10, 16)
    m0 = synth.blob_template(g, seed=3)
    m1 = synth.blob_template(g, seed=4)
    p = oracle.Params(grad_form=grad_form)
    st = oracle.state_at(np.zeros((3,) + g), m0, m1, p)
    vt = np.random.default_rng(0).standard_normal((3,) + g)
    h = oracle.hessian_matvec(st, vt)
    h0 = oracle.hessian0_matvec(vt, oracle.mean_state_gradient(st), p)
    assert _rel(h0, h) < 1e-12


def test_spectral_restriction_and_prolongation():
    """A band-limited field restricts to its samples at the coarse nodes and
    prolongs back exactly; E R is an orthogonal projection (idempotent,
    self-adjoint); the coarse Nyquist modes are dropped."""
    n, nc = (16, 12, 20), (8, 6, 10)
    f = synth.bandlimited_velocity(n, seed=1, kmax=2, vmax=1.0).astype(np.float64)
    fc = oracle.restrict_spectral(f, nc)
    assert np.abs(fc - f[:, ::2, ::2, ::2]).max() < 1e-12
    assert np.abs(oracle.prolong_spectral(fc, n) - f).max() < 1e-12
    r = np.random.default_rng(2)
    a, b = r.standard_normal((3,) + n), r.standard_normal((3,) + n)
    Pa = oracle.prolong_spectral(oracle.restrict_spectral(a, nc), n)
    Pb = oracle.prolong_spectral(oracle.restrict_spectral(b, nc), n)
    assert np.abs(oracle.prolong_spectral(oracle.restrict_spectral(Pa, nc), n) - Pa).max() < 1e-12
    assert abs(oracle.inner(Pa, b, n) - oracle.inner(a, Pb, n)) < 1e-10 * abs(oracle.inner(a, b, n)) + 1e-12
    # the coarse Nyquist plane x1 (k1 = 4 on the 8-node axis) is dropped
    x1, _, _ = _xyz(n)
    nyq = np.cos(4.0 * x1)[None]
    assert np.abs(oracle.restrict_spectral(nyq, nc)).max() < 1e-12


def test_two_level_preconditioner_special_cases():
    """gbar = 0 gives exactly S^{-1}; a coarse grid equal to the fine one with a
    tight inner tolerance inverts the mean-free part of H0 and passes the mean
    through; the near-exact preconditioner is self-adjoint and positive.
    Catches a wrong split of low and high modes or a mis-scaled restriction."""
    n = (12, 12, 16)
    r = np.random.default_rng(5)
    res = r.standard_normal((3,) + n)
    other = r.standard_normal((3,) + n)
    p = oracle.Params(pc_tol=1e-13, pc_maxit=400)
    zero = np.zeros((3, 6, 6, 8))
    assert _rel(oracle.precond_two_level(res, zero, p), oracle.precond(res, p)) < 1e-12
    m = synth.blob_template(n, seed=7)
    gbar = oracle.fd8_grad(m)
    # coarse grid = fine grid: H0 is inverted on the mean-free, non-Nyquist
    # modes (the projection Q below); the mean passes through unchanged
    mean_free = lambda f: f - f.mean(axis=(-3, -2, -1), keepdims=True)
    Q = lambda f: mean_free(oracle.prolong_spectral(oracle.restrict_spectral(f, n), n))
    rl = Q(res)
    z = oracle.precond_two_level(rl, gbar, p)
    assert _rel(Q(oracle.hessian0_matvec(z, gbar, p)), rl) < 1e-9
    zm = oracle.precond_two_level(res, gbar, p)
    assert np.abs((zm - mean_free(zm)) - (res - mean_free(res))).max() < 1e-12
    gc = oracle.restrict_spectral(gbar, (6, 6, 8))
    za = oracle.precond_two_level(res, gc, p)
    zb = oracle.precond_two_level(other, gc, p)
    assert abs(oracle.inner(za, other, n) - oracle.inner(res, zb, n)) < 1e-8 * abs(oracle.inner(za, other, n))
    assert oracle.inner(za, res, n) > 0.0


def test_two_level_registration_takes_fewer_iterations():
    """The paper's zero-velocity two-level preconditioner reaches the same
    gradient tolerance with fewer Gauss-Newton and PCG iterations than the
    spectral one on a nested-label pair, ending at the same objective within 1 %."""
    g = (24, 24, 24)
    m0 = synth.label_template(g, seed=0)
    vs = synth.bandlimited_velocity(g, seed=0, kmax=3, vmax=1.0)
    res = {}
    for pc in ("spectral", "2l"):
        p = oracle.Params(beta_v=1e-2, gtol=5e-2, max_gn=20, max_pcg=50, precond=pc)
        m1 = oracle.transport(m0, vs, p)
        _, rep = oracle.register(m0, m1, p)
        assert rep["status"] == "converged"
        res[pc] = rep
    assert sum(res["2l"]["pcg_iters"]) < sum(res["spectral"]["pcg_iters"])
    assert res["2l"]["gn_iters"] <= res["spectral"]["gn_iters"]
    assert res["2l"]["pc_inner_iters"] > 0
    assert abs(res["2l"]["J"][-1] - res["spectral"]["J"][-1]) < 0.01 * res["spectral"]["J"][-1]


def test_two_level_step_falls_back_to_spectral_when_the_line_search_fails(monkeypatch):
    """Safeguard of the two-level solver: a Gauss-Newton step whose two-level
    direction fails every Armijo trial is solved again with S^{-1}.  The
    failure is planted in the oracle: the objective reports +inf for every
    trial of the first step's two-level direction."""
    g = (16, 16, 16)
    m0 = synth.label_template(g, seed=0)
    vs = synth.bandlimited_velocity(g, seed=0, kmax=2, vmax=0.8)
    p = oracle.Params(beta_v=1e-2, gtol=5e-2, max_gn=3, max_pcg=20, precond="2l")
    m1 = oracle.transport(m0, vs, p)
    real_objective = oracle.objective
    calls = {"n": 0}

    def planted(v, a, b, q):
        calls["n"] += 1
        if calls["n"] <= q.max_ls:  # every trial of the first (two-level) direction
            return math.inf, math.inf, math.inf
        return real_objective(v, a, b, q)

    monkeypatch.setattr(oracle, "objective", planted)
    _, rep = oracle.register(m0, m1, p)
    assert rep["pc_fallbacks"] == 1
    assert rep["gn_iters"] >= 1 and rep["status"] != "line_search_failed"
    assert rep["J"][1] < rep["J"][0]
