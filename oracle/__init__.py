"""FP64 CPU oracle for the semi-Lagrangian Gauss-Newton-Krylov hot path of
"CLAIRE at scale" (arXiv 2209.08189).

TEST INFRASTRUCTURE.  Only tests/, ``__graft_entry__.smoke()`` and the CPU
baseline / reference legs of ``bench.py`` may import this package.  It shares
no code with the CUDA path: the pointwise kernels live in ``kernels.c``
(plain double-precision loops) and everything else is numpy.

What it computes, step by step, in the paper's order and notation:

* Objective, Eq. (1a): J(v) = 1/2 ||m(1) - m1||^2 + beta_v/2 reg_v(v)
  + beta_w/2 reg_w(div v), with reg_v the H1 seminorm (or H2) and reg_w the
  H1 norm (Sec. 2.1), evaluated spectrally: 1/2 <v, S v>.
* State, Eqs. (1b)-(1c): semi-Lagrangian (SL) transport with RK2
  characteristics (Sec. 2.2 "Discretization").
* Adjoint, Eq. (4): -d_t lambda - div(lambda v) = 0, lambda(1) = m1 - m(1),
  solved by SL along +v with the source lambda * div v integrated by Heun.
* Reduced gradient, Eq. (3): g = beta_v A v + K int_0^1 lambda grad m dt.
  Default ("exact" form): g = S v + b with the symbol
  S(k) = beta_v |k|^2 I + beta_w (1 + |k|^2) k k^T, the exact gradient of J
  in the continuum.  Opt-in paper form: g = K (S v + b) = beta_v A v + K b.
* Gauss-Newton Hessian matvec, Eq. (6), with the incremental state and
  incremental adjoint solves.
* Gauss-Newton-Krylov with Armijo line search, Eq. (5), matrix-free PCG,
  spectral preconditioner S^{-1}, or the zero-velocity Hessian approximation
  applied through a two-level coarse grid (Sec. 2.2 "Optimization").
* Jacobian determinant det grad y of the deformation map (Sec. 4.1).
* Coarse preconditioner correction of the learned warm start: a pointwise
  weight w >= 0 of the zero-velocity data term on the coarse grid, and its
  least-squares fit to the data term of the Gauss-Newton matvec.

Readings where the paper is silent are listed in the module docstrings below
(interpolation nodes, Heun variant, trapezoidal time quadrature, Nyquist
handling of odd symbols, discrete inner product h1*h2*h3*sum).
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field, replace

import numpy as np

from . import build as _build

__all__ = [
    "Params", "spacing", "bspline_prefilter", "interp", "interp_points", "interp_T", "backtrace",
    "fd8_grad", "fd8_div", "reg_apply", "reg_inverse", "project_K", "reg_energy",
    "characteristics", "forward_solve", "adjoint_solve", "state_at", "objective",
    "gradient", "hessian_matvec", "incremental_state", "precond", "pcg", "register",
    "transport", "transport_vjp", "interp_grad", "deformation_map", "detj", "cfl", "inner",
    "num_threads", "param_search", "param_continuation", "hessian0_matvec", "mean_state_gradient",
    "restrict_spectral", "prolong_spectral", "precond_two_level", "pc_weight_stats", "pc_weight_stats_at",
    "pc_weight_fit",
]

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(ctypes.c_long)
        lib.orc_interp.argtypes = [lp, dp, dp, ctypes.c_int, dp]
        lib.orc_interp_points.argtypes = [lp, dp, dp, ctypes.c_long, ctypes.c_int, dp]
        lib.orc_interp_transpose.argtypes = [lp, dp, dp, ctypes.c_int, dp]
        lib.orc_interp_grad.argtypes = [lp, dp, dp, ctypes.c_int, dp]
        lib.orc_backtrace.argtypes = [lp, dp, dp, ctypes.c_double, ctypes.c_int, ctypes.c_int, dp]
        lib.orc_fd8_grad.argtypes = [lp, dp, dp]
        lib.orc_fd8_div.argtypes = [lp, dp, dp]
        lib.orc_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _n(shape):
    return (ctypes.c_long * 3)(*[int(s) for s in shape])


def _f64(a):
    """float64, C-contiguous (the C kernels read raw pointers)."""
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    """Threads the C kernels use (OpenMP), for reporting the CPU baseline."""
    return int(_load().orc_num_threads())


# ----------------------------------------------------------------------------
# Grid, inner product
# ----------------------------------------------------------------------------

def spacing(n):
    """h_c = 2 pi / N_c on the periodic domain [0, 2 pi)^3 (Sec. 2.2)."""
    return np.array([2.0 * math.pi / int(s) for s in n])


def inner(a, b, n):
    """Discrete L2 inner product h1 h2 h3 sum(a * b) (reading: plain Riemann sum)."""
    return float(np.prod(spacing(n)) * np.sum(_f64(a) * _f64(b)))


# ----------------------------------------------------------------------------
# Pointwise kernels (C)
# ----------------------------------------------------------------------------

def bspline_prefilter(f):
    """Cubic B-spline coefficients c of a periodic field f (Sec. 3, B-spline
    interpolation): sum_j c_j beta(x_i - x_j) = f_i, solved in Fourier space,
    where the sampled spline is the symbol prod_axes (2 + cos(k h)) / 3."""
    f = _f64(f)
    F = np.fft.fftn(f)
    sym = np.ones(f.shape)
    for ax, n in enumerate(f.shape):
        k = np.fft.fftfreq(n, 1.0 / n)
        s = (2.0 + np.cos(2.0 * math.pi * k / n)) / 3.0
        shape = [1] * f.ndim
        shape[ax] = n
        sym = sym * s.reshape(shape)
    return np.ascontiguousarray(np.real(np.fft.ifftn(F / sym)))


def _coef(f, order):
    return bspline_prefilter(f) if order == 4 else _f64(f)


def interp(f, d, order=3):
    """f(x + d) at every grid node; d in grid units, shape (3, *f.shape).

    Sec. 3 "IP kernel": cubic Lagrange (order 3, nodes floor-1..floor+2),
    cubic B-spline on prefiltered coefficients (order 4, same nodes) or
    linear (order 1), periodic wrap.
    """
    f = _coef(f, order); d = _f64(d)
    out = np.empty_like(f)
    _load().orc_interp(_n(f.shape), _dp(f), _dp(d), int(order), _dp(out))
    return out


def interp_points(f, y, order=3):
    """Interpolant of f at explicit grid-unit points y, shape (3, M)."""
    f = _coef(f, order); y = _f64(y)
    out = np.empty(y.shape[1])
    _load().orc_interp_points(_n(f.shape), _dp(f), _dp(y), int(y.shape[1]), int(order), _dp(out))
    return out


def interp_T(yv, d, order=3):
    """Exact transpose of interp(., d): scatter of point values to nodes
    (for B-splines followed by the prefilter, which is symmetric)."""
    yv = _f64(yv); d = _f64(d)
    out = np.empty_like(yv)
    _load().orc_interp_transpose(_n(yv.shape), _dp(yv), _dp(d), int(order), _dp(out))
    return bspline_prefilter(out) if order == 4 else out


def interp_grad(f, d, order=3):
    """Gradient of the interpolant of f at x + d (grid units), shape (3, *f.shape)."""
    f = _coef(f, order); d = _f64(d)
    out = np.empty((3,) + f.shape)
    _load().orc_interp_grad(_n(f.shape), _dp(f), _dp(d), int(order), _dp(out))
    return out


def backtrace(v, dt, sign=+1, order=3):
    """RK2 (Heun) characteristic displacement in grid units (Sec. 2.2).

    sign=+1: X = x - dt/2 [v(x) + v(x - dt v(x))] (state); sign=-1: the
    adjoint characteristic X+ along +v.
    """
    v = _f64(v)
    n = v.shape[1:]
    vc = np.stack([bspline_prefilter(v[c]) for c in range(3)]) if order == 4 else v
    d = np.empty_like(v)
    _load().orc_backtrace(_n(n), _dp(v), _dp(np.ascontiguousarray(vc)), float(dt), int(sign), int(order), _dp(d))
    return d


def fd8_grad(f):
    """8th-order central FD gradient (Sec. 2.2 / Sec. 3 "FD kernel"), periodic."""
    f = _f64(f)
    g = np.empty((3,) + f.shape)
    _load().orc_fd8_grad(_n(f.shape), _dp(f), _dp(g))
    return g


def fd8_div(v):
    """8th-order central FD divergence, periodic."""
    v = _f64(v)
    d = np.empty(v.shape[1:])
    _load().orc_fd8_div(_n(v.shape[1:]), _dp(v), _dp(d))
    return d


# ----------------------------------------------------------------------------
# Spectral operators (Sec. 2.2: "two FFTs and one Hadamard product")
# ----------------------------------------------------------------------------

@dataclass
class Params:
    """Solver parameters (Sec. 3 "Key Solver Parameters")."""
    beta_v: float = 1e-2
    beta_w: float = 1e-4
    reg: int = 1            # 1 = H1 seminorm on v, 2 = H2 seminorm
    nt: int = 4
    order: int = 3          # 3 = cubic Lagrange, 1 = linear
    grad_form: int = 0      # 0 = S v + b (exact gradient of J); 1 = beta_v A v + K b
    gtol: float = 5e-2
    max_gn: int = 50
    max_pcg: int = 10
    pcg_rtol_max: float = 0.5
    pcg_fixed: bool = False  # run exactly max_pcg PCG iterations (fixed schedule)
    armijo_c1: float = 1e-4
    max_ls: int = 10
    adjoint: str = "sl"     # "sl" = paper's SL adjoint (OTD); "scatter" = exact transpose (DTO)
    precond: str = "spectral"  # "spectral" = S^{-1}; "2l" = two-level zero-velocity (Sec. 2.2)
    pc_coarse: int = 2      # fine-to-coarse grid ratio of the two-level preconditioner
    pc_tol: float = 1e-1    # relative residual of its inner PCG (0: run pc_maxit iterations)
    pc_maxit: int = 50
    pc_weight: object = None  # coarse-grid weight w >= 0 of the zero-velocity data term (None: w = 1)
    extra: dict = field(default_factory=dict)

    @property
    def dt(self):
        return 1.0 / self.nt


def _symbols(n, p: Params):
    """Per-mode pieces of S(k) = a(k) I + c(k) u u^T on the rfft half grid.

    a = beta_v |k|^2 (H1) or beta_v |k|^4 (H2); c = beta_w (1 + |k|^2);
    u = k with the Nyquist component set to zero (reading: the first-
    derivative symbol is odd, so on a Nyquist plane it is taken as 0 to keep
    the operator real-symmetric); |k|^2 keeps the Nyquist value (even).
    """
    n0, n1, n2 = (int(s) for s in n)
    k0 = np.fft.fftfreq(n0, 1.0 / n0)
    k1 = np.fft.fftfreq(n1, 1.0 / n1)
    k2 = np.fft.rfftfreq(n2, 1.0 / n2)
    K0, K1, K2 = np.meshgrid(k0, k1, k2, indexing="ij")
    kk = K0 ** 2 + K1 ** 2 + K2 ** 2
    u = np.stack([np.where(np.abs(K0) == n0 / 2, 0.0, K0),
                  np.where(np.abs(K1) == n1 / 2, 0.0, K1),
                  np.where(np.abs(K2) == n2 / 2, 0.0, K2)])
    a = p.beta_v * (kk if p.reg == 1 else kk ** 2)
    c = p.beta_w * (1.0 + kk)
    return a, c, u, kk


def _fft3(v):
    return np.fft.rfftn(_f64(v), axes=(-3, -2, -1))


def _ifft3(vh, n):
    return np.fft.irfftn(vh, s=tuple(int(s) for s in n), axes=(-3, -2, -1))


def reg_apply(v, p: Params):
    """S v = F^{-1}[a v^ + c u (u . v^)] (first variation of the regulariser)."""
    v = _f64(v); n = v.shape[1:]
    a, c, u, _ = _symbols(n, p)
    vh = _fft3(v)
    ud = np.sum(u * vh, axis=0)
    return _ifft3(a * vh + c * u * ud, n)


def reg_inverse(r, p: Params):
    """Preconditioner S^{-1} (Sherman-Morrison on a I + c u u^T); identity at k = 0."""
    r = _f64(r); n = r.shape[1:]
    a, c, u, kk = _symbols(n, p)
    rh = _fft3(r)
    ud = np.sum(u * rh, axis=0)
    nz = kk > 0
    a_safe = np.where(nz, a, 1.0)
    den = a_safe + c * np.sum(u * u, axis=0)
    zh = np.where(nz, (rh - c * u * ud / den) / a_safe, rh)
    return _ifft3(zh, n)


def project_K(b, p: Params):
    """Leray-like operator K = a S^{-1} = I - c u u^T / (a + c |u|^2); K = I at k = 0.

    Reading of Eq. (3): eliminating w and the multiplier p of Eq. (2) gives
    g = beta_v A v + K b with this K; it tends to the Leray projection as
    beta_w -> infinity and to I as beta_w -> 0.
    """
    b = _f64(b); n = b.shape[1:]
    a, c, u, kk = _symbols(n, p)
    bh = _fft3(b)
    ud = np.sum(u * bh, axis=0)
    nz = kk > 0
    den = np.where(nz, a + c * np.sum(u * u, axis=0), 1.0)
    return _ifft3(np.where(nz, bh - c * u * ud / den, bh), n)


def reg_energy(v, p: Params):
    """beta_v/2 reg_v(v) + beta_w/2 reg_w(div v) = 1/2 <v, S v>."""
    return 0.5 * inner(v, reg_apply(v, p), v.shape[1:])


# ----------------------------------------------------------------------------
# Semi-Lagrangian solves
# ----------------------------------------------------------------------------

def _weights(nt):
    """Trapezoidal weights in time for int_0^1 (.) dt on nt+1 points."""
    dt = 1.0 / nt
    w = np.full(nt + 1, dt)
    w[0] = w[-1] = 0.5 * dt
    return w


def characteristics(v, p: Params):
    """Per-velocity data reused by every solve: X (state), X+ (adjoint),
    d = div v and d(X+)."""
    v = _f64(v)
    d_state = backtrace(v, p.dt, +1, p.order)
    d_adj = backtrace(v, p.dt, -1, p.order)
    div = fd8_div(v)
    return {"d": d_state, "dp": d_adj, "div": div, "div_Xp": interp(div, d_adj, p.order)}


def forward_solve(m0, ch, p: Params):
    """m^{j+1} = m^j(X), j = 0..nt-1 (Eq. (1b)-(1c)); returns all nt+1 states."""
    ms = [_f64(m0)]
    for _ in range(p.nt):
        ms.append(interp(ms[-1], ch["d"], p.order))
    return ms


def _adjoint_step(lam_next, ch, p: Params):
    """One SL step of Eq. (4) backwards in time.

    Along the characteristic traced along +v the adjoint obeys
    d lambda / d tau = lambda div v; Heun gives
    lambda^j = a + dt/2 [a d(X+) + (a + dt a d(X+)) d(x)], a = lambda^{j+1}(X+).
    """
    dt = p.dt
    a = interp(lam_next, ch["dp"], p.order)
    pred = a + dt * a * ch["div_Xp"]
    return a + 0.5 * dt * (a * ch["div_Xp"] + pred * ch["div"])


def adjoint_solve(lam_end, ch, gms, p: Params, mode=None):
    """Backward solve from lambda^{nt} and body b = sum_j w_j lambda^j grad m^j.

    mode "sl": the paper's SL adjoint (optimise-then-discretise);
    mode "scatter": lambda^j = T^T lambda^{j+1}, the exact transpose of the
    state step (discretise-then-optimise), used by the symmetry pins.
    Returns (b, lambda^0).
    """
    mode = mode or p.adjoint
    w = _weights(p.nt)
    lam = _f64(lam_end)
    b = w[p.nt] * lam[None] * gms[p.nt]
    for j in range(p.nt - 1, -1, -1):
        if mode == "sl":
            lam = _adjoint_step(lam, ch, p)
        else:
            lam = interp_T(lam, ch["d"], p.order)
        b = b + w[j] * lam[None] * gms[j]
    return b, lam


class State:
    """Linearisation point of the Gauss-Newton step: v, characteristics,
    states m^j and their FD8 gradients."""

    def __init__(self, v, m0, m1, p: Params):
        self.v = _f64(v)
        self.m0 = _f64(m0)
        self.m1 = _f64(m1)
        self.p = p
        self.n = self.m0.shape
        self.ch = characteristics(self.v, p)
        self.ms = forward_solve(self.m0, self.ch, p)
        self.gms = [fd8_grad(m) for m in self.ms]
        self.reg_v = reg_apply(self.v, p)
        res = self.ms[-1] - self.m1
        self.mismatch = 0.5 * inner(res, res, self.n)
        self.reg = 0.5 * inner(self.v, self.reg_v, self.n)
        self.J = self.mismatch + self.reg


def state_at(v, m0, m1, p: Params):
    return State(v, m0, m1, p)


def objective(v, m0, m1, p: Params):
    """J(v), the mismatch term and the regularisation term (Eq. (1a))."""
    v = _f64(v)
    ch = {"d": backtrace(v, p.dt, +1, p.order)}
    m = _f64(m0)
    for _ in range(p.nt):
        m = interp(m, ch["d"], p.order)
    res = m - _f64(m1)
    mis = 0.5 * inner(res, res, m.shape)
    reg = reg_energy(v, p)
    return mis + reg, mis, reg


def _apply_form(x, p: Params):
    return project_K(x, p) if p.grad_form == 1 else x


def gradient(st: State, mode=None):
    """Reduced gradient, Eq. (3): g = S v + b (or K(S v + b) = beta_v A v + K b)."""
    b, _ = adjoint_solve(st.m1 - st.ms[-1], st.ch, st.gms, st.p, mode)
    return _apply_form(st.reg_v + b, st.p)


def incremental_state(st: State, vt):
    """Incremental state of the linearised Eq. (1b):
    d_t mt + v . grad mt = -vt . grad m, mt(0) = 0, SL with Heun sources:
    mt^{j+1} = (mt^j + dt/2 f^j)(X) + dt/2 f^{j+1}, f^j = -vt . grad m^j."""
    p = st.p
    dt = p.dt
    vt = _f64(vt)
    f = [-np.sum(vt * gm, axis=0) for gm in st.gms]
    mt = np.zeros(st.n)
    for j in range(p.nt):
        mt = interp(mt + 0.5 * dt * f[j], st.ch["d"], p.order) + 0.5 * dt * f[j + 1]
    return mt


def hessian_matvec(st: State, vt, mode=None):
    """Gauss-Newton Hessian matvec, Eq. (6): H vt = S vt + int lt grad m dt
    (or K applied to it), with the incremental adjoint lt(1) = -mt(1)."""
    mt = incremental_state(st, vt)
    bt, _ = adjoint_solve(-mt, st.ch, st.gms, st.p, mode)
    return _apply_form(reg_apply(vt, st.p) + bt, st.p)


def precond(r, p: Params):
    """Spectral preconditioner: inverse of the regularisation operator
    (K-form: S^{-1} restricted so that it inverts beta_v A)."""
    if p.grad_form == 1:
        # g = K(S v + b) with K S = a I: precondition with (a I)^{-1}
        r = _f64(r); n = r.shape[1:]
        a, c, u, kk = _symbols(n, p)
        rh = _fft3(r)
        return _ifft3(np.where(kk > 0, rh / np.where(kk > 0, a, 1.0), rh), n)
    return reg_inverse(r, p)


# ----------------------------------------------------------------------------
# Zero-velocity Hessian and the two-level preconditioner (Sec. 2.2)
# ----------------------------------------------------------------------------
#
# The paper preconditions H with a zero-velocity approximation of it, applied
# through a two-level coarse grid, and leaves the construction to a cited
# reference.  Readings taken here:
#
# * Zero velocity: with v = 0 in the incremental equations the characteristics
#   are the identity, so mt(1) = -int vt . grad m dt, lt = -mt(1) is constant
#   in time and the body is (int grad m dt)(int grad m dt . vt).  With the
#   trapezoid rule of the solves, H0 vt = S vt + gbar (gbar . vt), gbar =
#   sum_j w_j grad m^j (FD8 gradients of the current states), or K of that for
#   the paper's gradient form.  At v = 0 this is exactly the full Gauss-Newton
#   matvec.
# * Two levels: Fourier truncation R to the modes |k_i| < nc_i / 2 (the
#   coarse Nyquist planes are dropped, so E R is an orthogonal projection
#   onto low modes, E the zero-padding prolongation), gbar restricted the same
#   way, H0 on the coarse grid inverted by an inner PCG (preconditioner
#   S^{-1}, x0 = 0, relative residual pc_tol or pc_maxit iterations), and
#   S^{-1} on the remaining high modes:
#   P^{-1} r = E H0c^{-1} R r + S^{-1} (r - E R r).
# * The mean (k = 0) is treated as by S^{-1}, with the identity.  The inner
#   PCG works on the coarse modes that R keeps (mean-free, no Nyquist planes),
#   with the operator Q H0c Q, Q the projection onto them; there H0 (S
#   positive, gbar gbar^T semidefinite) is positive definite, and H0c^{-1}
#   means the inverse of Q H0c Q.
# * The outer PCG takes the flexible (Polak-Ribiere) direction update when
#   this inexact preconditioner is in use.
# * Safeguard (ours): a Gauss-Newton step whose two-level solve fails the
#   Armijo line search is solved again with S^{-1}.

def mean_state_gradient(st: State):
    """gbar = sum_j w_j grad m^j (trapezoid weights of the solves)."""
    w = _weights(st.p.nt)
    return sum(w[j] * st.gms[j] for j in range(st.p.nt + 1))


def hessian0_matvec(vt, gbar, p: Params):
    """Zero-velocity Gauss-Newton matvec H0 vt = S vt + gbar (gbar . vt) (or K of it)."""
    vt = _f64(vt); gbar = _f64(gbar)
    return _apply_form(reg_apply(vt, p) + gbar * np.sum(gbar * vt, axis=0), p)


def _low_index(n, nc):
    """Indices of the modes |k| < nc/2 along an FFT axis of length n (and nc)."""
    h = nc // 2
    return np.r_[0:h, n - h + 1:n], np.r_[0:h, nc - h + 1:nc]


def _truncate(Fh, nout, nin):
    """Copy the modes |k_i| < min(nout_i, nin_i)/2 between half spectra of the grids nin -> nout."""
    lo = [min(a, b) for a, b in zip(nout, nin)]
    a_in0 = _low_index(nin[0], lo[0])[0]; a_out0 = _low_index(nout[0], lo[0])[0]
    a_in1 = _low_index(nin[1], lo[1])[0]; a_out1 = _low_index(nout[1], lo[1])[0]
    h2 = lo[2] // 2
    out = np.zeros(Fh.shape[:-3] + (nout[0], nout[1], nout[2] // 2 + 1), dtype=complex)
    out[..., a_out0[:, None, None], a_out1[None, :, None], np.arange(h2)[None, None, :]] = \
        Fh[..., a_in0[:, None, None], a_in1[None, :, None], np.arange(h2)[None, None, :]]
    return out


def restrict_spectral(f, nc):
    """R f: the band-limited part of f (modes |k_i| < nc_i/2) sampled on the grid nc."""
    f = _f64(f); n = f.shape[-3:]
    nc = tuple(int(x) for x in nc)
    Fh = np.fft.rfftn(f, axes=(-3, -2, -1)) / np.prod(n)
    return np.fft.irfftn(_truncate(Fh, nc, n) * np.prod(nc), s=nc, axes=(-3, -2, -1))


def prolong_spectral(fc, n):
    """E fc: trigonometric (zero-padding) interpolation of the coarse field fc to the grid n,
    with the coarse Nyquist modes dropped."""
    fc = _f64(fc); nc = fc.shape[-3:]
    n = tuple(int(x) for x in n)
    Ch = np.fft.rfftn(fc, axes=(-3, -2, -1)) / np.prod(nc)
    return np.fft.irfftn(_truncate(Ch, n, nc) * np.prod(n), s=n, axes=(-3, -2, -1))


def _mean_free(f):
    """f without its k = 0 Fourier mode (the mean of each component)."""
    return f - f.mean(axis=(-3, -2, -1), keepdims=True)


def _kept_modes(f):
    """Q f: f without its mean and without its Nyquist planes (the coarse modes R keeps)."""
    n = f.shape[-3:]
    return _mean_free(restrict_spectral(f, n))


def _pcg_h0(rhs, gbar, p: Params, tol, maxit):
    """Inner PCG for Q H0 Q x = Q rhs (preconditioner S^{-1}, x0 = 0);
    returns (x, iterations)."""
    n = rhs.shape[1:]
    x = np.zeros_like(rhs)
    r = _kept_modes(_f64(rhs))
    r0 = math.sqrt(inner(r, r, n))
    if r0 == 0.0:
        return x, 0
    z = precond(r, p)
    pv = z.copy()
    rz = inner(r, z, n)
    it = 0
    for it in range(1, maxit + 1):
        q = _kept_modes(hessian0_matvec(pv, gbar, p))
        pq = inner(pv, q, n)
        if pq <= 0.0:
            break
        alpha = rz / pq
        x = x + alpha * pv
        r = r - alpha * q
        if tol > 0.0 and math.sqrt(inner(r, r, n)) <= tol * r0:
            break
        z = precond(r, p)
        rz_new = inner(r, z, n)
        pv = z + (rz_new / rz) * pv
        rz = rz_new
    return x, it


def precond_two_level(r, gbar_c, p: Params, stats=None, w=None):
    """P^{-1} r = E H0c^{-1} R r + S^{-1} (r - E R r) (zero-velocity Hessian on
    the coarse grid of gbar_c, spectral inverse on the high modes).  With a
    coarse-grid weight w >= 0 the coarse operator is S + gbar_c w gbar_c^T,
    the zero-velocity operator of sqrt(w) gbar_c."""
    r = _f64(r); n = r.shape[1:]
    nc = gbar_c.shape[1:]
    if w is not None:
        gbar_c = gbar_c * np.sqrt(np.maximum(_f64(w), 0.0))
    rc = restrict_spectral(r, nc)
    xc, its = _pcg_h0(rc, gbar_c, p, p.pc_tol, p.pc_maxit)
    if stats is not None:
        stats.append(its)
    low = prolong_spectral(rc, n)          # E R r, mean included
    mean = r - _mean_free(r)               # identity on k = 0
    return prolong_spectral(xc, n) + precond(r - low, p) + mean


# ----------------------------------------------------------------------------
# Coarse preconditioner correction (the learned warm start's second output)
# ----------------------------------------------------------------------------
#
# The zero-velocity operator keeps only the pointwise rank-one data term
# gbar (gbar . vt).  The correction weights it pointwise on the coarse grid,
# H0w vt = S vt + gbar w (gbar . vt) with w >= 0 (precond_two_level's w);
# w = 1 is the paper's preconditioner.  The weight a predictor should
# reproduce is the least-squares fit of the model D ~ gbar w (gbar . p) to the
# data term D = H p - S p of the true Gauss-Newton matvec on probe fields p,
# pooled over the fine voxels of each coarse cell:
#   w = max(sum a (gbar . D) / sum a^2 |gbar|^2, 0),   a = gbar . p,
# and w = 1 where the pooled denominator vanishes (no image gradient).
# At v = 0 the data term is exactly gbar (gbar . p), so the fit gives w = 1.

def pc_weight_stats(gbar, probes, data_terms):
    """Per-voxel sums num = sum_p a (gbar . D_p) and den = sum_p a^2 |gbar|^2,
    a = gbar . p, over probe fields p and the data terms D_p = H p - S p."""
    gbar = _f64(gbar)
    g2 = np.sum(gbar * gbar, axis=0)
    num = np.zeros(gbar.shape[1:])
    den = np.zeros(gbar.shape[1:])
    for pv, D in zip(probes, data_terms):
        a = np.sum(gbar * _f64(pv), axis=0)
        num += a * np.sum(gbar * _f64(D), axis=0)
        den += a * a * g2
    return num, den


def pc_weight_stats_at(st: State, probes, mode=None):
    """pc_weight_stats with the data terms of the Gauss-Newton matvec at st
    (exact-gradient form: H p = S p + data term)."""
    if st.p.grad_form != 0:
        raise ValueError("the data term is separated from S only in the exact-gradient form")
    gbar = mean_state_gradient(st)
    terms = [hessian_matvec(st, pv, mode) - reg_apply(pv, st.p) for pv in probes]
    return pc_weight_stats(gbar, probes, terms)


def pc_weight_fit(num, den, nc):
    """Fitted weight on the coarse grid nc: the fine sums pooled over the
    (n / nc)^3 voxels of each coarse cell, w = max(num / den, 0), w = 1 where
    den = 0."""
    n = num.shape
    r = [a // b for a, b in zip(n, nc)]
    if any(a != b * c for a, b, c in zip(n, nc, r)):
        raise ValueError("the fine grid must be an integer multiple of the coarse grid")
    pool = lambda f: f.reshape(nc[0], r[0], nc[1], r[1], nc[2], r[2]).sum(axis=(1, 3, 5))
    nu, de = pool(_f64(num)), pool(_f64(den))
    w = np.ones(tuple(nc))
    pos = de > 0
    w[pos] = np.maximum(nu[pos] / de[pos], 0.0)
    return w


def pcg(st: State, rhs, rtol, maxit, mode=None, fixed_iters=False, stats=None):
    """Matrix-free PCG for H x = rhs (Sec. 2.2), x0 = 0; stops when
    ||r|| <= rtol ||r0|| or after maxit matvecs.  Returns (x, iterations).
    With the two-level preconditioner the direction update is the flexible
    (Polak-Ribiere) one, since that preconditioner is an inexact inner solve."""
    n = st.n
    p = st.p
    two_level = p.precond == "2l"
    if two_level:
        nc = tuple(s // p.pc_coarse for s in n)
        gbar_c = restrict_spectral(mean_state_gradient(st), nc)
        apply_p = lambda res: precond_two_level(res, gbar_c, p, stats, p.pc_weight)
    else:
        apply_p = lambda res: precond(res, p)
    x = np.zeros_like(rhs)
    r = _f64(rhs).copy()
    r0 = math.sqrt(inner(r, r, n))
    if r0 == 0.0:
        return x, 0
    z = apply_p(r)
    pv = z.copy()
    rz = inner(r, z, n)
    it = 0
    for it in range(1, maxit + 1):
        q = hessian_matvec(st, pv, mode)
        pq = inner(pv, q, n)
        if pq <= 0.0:
            if it == 1:
                x = pv.copy()
            break
        alpha = rz / pq
        x = x + alpha * pv
        r = r - alpha * q
        if not fixed_iters and math.sqrt(inner(r, r, n)) <= rtol * r0:
            break
        if it == maxit:
            break
        z_new = apply_p(r)
        rz_new = inner(r, z_new, n)
        beta = ((rz_new - inner(r, z, n)) if two_level else rz_new) / rz
        pv = z_new + beta * pv
        z = z_new
        rz = rz_new
    return x, it


def register(m0, m1, p: Params, v0=None, mode=None, log=None):
    """Gauss-Newton-Krylov with Armijo line search, Eq. (5).

    PCG forcing eta_k = min(pcg_rtol_max, sqrt(||g_k|| / ||g_0||)); Armijo
    alpha_0 = 1, halving, sufficient decrease c1; stop when
    ||g|| / ||g_0|| <= gtol or after max_gn steps.
    """
    m0 = _f64(m0); m1 = _f64(m1)
    n = m0.shape
    v = np.zeros((3,) + n) if v0 is None else _f64(v0).copy()
    st = State(v, m0, m1, p)
    g = gradient(st, mode)
    g0 = math.sqrt(inner(g, g, n))
    rep = {"gn_iters": 0, "pcg_iters": [], "alpha": [], "J": [st.J], "gnorm_rel": [1.0],
           "status": "not_converged", "g0": g0, "pc_inner_iters": 0, "pc_fallbacks": 0}
    inner_its = []
    if g0 == 0.0:
        rep["status"] = "converged"
        return v, rep
    for _ in range(p.max_gn):
        rel = math.sqrt(inner(g, g, n)) / g0
        if rel <= p.gtol:
            rep["status"] = "converged"
            break
        eta = min(p.pcg_rtol_max, math.sqrt(rel))
        ok, its_step = False, 0
        # a step whose two-level solve fails the line search is solved again
        # with the spectral preconditioner (once)
        for attempt in range(2):
            if attempt == 1:
                if p.precond != "2l":
                    break
                rep["pc_fallbacks"] = rep.get("pc_fallbacks", 0) + 1
                st_solve = State(v, m0, m1, replace(p, precond="spectral"))
            else:
                st_solve = st
            vt, its = pcg(st_solve, -g, eta, p.max_pcg, mode, fixed_iters=p.pcg_fixed, stats=inner_its)
            its_step += its
            rep["pc_inner_iters"] = sum(inner_its)
            gtv = inner(g, vt, n)
            alpha = 1.0
            for _ls in range(p.max_ls):
                Jt, _, _ = objective(v + alpha * vt, m0, m1, p)
                if Jt <= st.J + p.armijo_c1 * alpha * gtv:
                    ok = True
                    break
                alpha *= 0.5
            if ok:
                break
        its = its_step
        rep["pcg_iters"].append(its)
        if not ok:
            rep["status"] = "line_search_failed"
            break
        rep["alpha"].append(alpha)
        v = v + alpha * vt
        st = State(v, m0, m1, p)
        g = gradient(st, mode)
        rep["gn_iters"] += 1
        rep["J"].append(st.J)
        rep["gnorm_rel"].append(math.sqrt(inner(g, g, n)) / g0)
        if log is not None:
            log(rep)
    else:
        if rep["gnorm_rel"][-1] <= p.gtol:
            rep["status"] = "converged"
    rep["mismatch"] = st.mismatch
    den = inner(m0 - m1, m0 - m1, n)
    rep["r"] = (2.0 * st.mismatch / den) if den > 0 else 0.0
    return v, rep


# ----------------------------------------------------------------------------
# Transport entry points, deformation map, Jacobian determinant, CFL
# ----------------------------------------------------------------------------

def transport(m_in, v, p: Params, direction="fwd"):
    """"fwd": m(1) from m(0) by Eq. (1b); "adj": lambda(0) from lambda(1) by Eq. (4)."""
    v = _f64(v)
    if direction == "fwd":
        d = backtrace(v, p.dt, +1, p.order)
        m = _f64(m_in)
        for _ in range(p.nt):
            m = interp(m, d, p.order)
        return m
    ch = characteristics(v, p)
    lam = _f64(m_in)
    for _ in range(p.nt):
        lam = _adjoint_step(lam, ch, p)
    return lam


def transport_vjp(m0, v, gbar, p: Params):
    """Exact reverse-mode derivative of the discrete forward transport
    m(1) = T(v)^nt m0 (discretise-then-differentiate).

    Forward, per node x (grid units u = v / h): predictor y = x - dt u(x),
    U = I[u](y), displacement d = -dt/2 (u(x) + U), X = x + d and
    m^{j+1}(x) = I[m^j](X(x)).  Given gbar = dL/dm(1) it returns
    (dL/dm0, dL/dv) by the chain rule through the interpolation weights
    (their t-derivatives), the scatter transposes at X and at y, and the
    predictor; the interpolation of v uses the same scheme as the image.
    """
    m0 = _f64(m0); v = _f64(v)
    n = m0.shape
    h = spacing(n)
    dt = p.dt
    u = np.stack([v[c] / h[c] for c in range(3)])
    dpred = -dt * u                       # y - x
    U = np.stack([interp(u[c], dpred, p.order) for c in range(3)])
    d = -0.5 * dt * (u + U)
    ms = [m0]
    for _ in range(p.nt):
        ms.append(interp(ms[-1], d, p.order))
    mbar = _f64(gbar)
    dbar = np.zeros_like(u)
    for j in range(p.nt - 1, -1, -1):
        dbar += mbar[None] * interp_grad(ms[j], d, p.order)
        mbar = interp_T(mbar, d, p.order)
    ubar = -0.5 * dt * dbar               # direct term of d
    Ubar = -0.5 * dt * dbar               # through U = I[u](y)
    ybar = np.zeros_like(u)
    for c in range(3):
        ubar[c] += interp_T(Ubar[c], dpred, p.order)
        ybar += Ubar[c][None] * interp_grad(u[c], dpred, p.order)
    ubar += -dt * ybar                    # y = x - dt u
    vbar = np.stack([ubar[c] / h[c] for c in range(3)])
    return mbar, vbar


def deformation_map(v, p: Params):
    """Displacement u of the map y = x + u with m(1) = m0(y): u^0 = 0,
    u^{j+1} = u^j(X) + (X - x) (reading: transport of the map by the same SL
    steps as the state)."""
    v = _f64(v)
    n = v.shape[1:]
    h = spacing(n)
    d = backtrace(v, p.dt, +1, p.order)
    u = np.zeros_like(v)
    for _ in range(p.nt):
        u = np.stack([interp(u[c], d, p.order) + d[c] * h[c] for c in range(3)])
    return u


def detj(v, p: Params):
    """det F, F = grad y = I + grad u (FD8), in FP64 (Sec. 3 "J_min")."""
    u = deformation_map(v, p)
    F = np.empty((3, 3) + u.shape[1:])
    for c in range(3):
        gu = fd8_grad(u[c])
        for e in range(3):
            F[c, e] = gu[e] + (1.0 if c == e else 0.0)
    return (F[0, 0] * (F[1, 1] * F[2, 2] - F[1, 2] * F[2, 1])
            - F[0, 1] * (F[1, 0] * F[2, 2] - F[1, 2] * F[2, 0])
            + F[0, 2] * (F[1, 0] * F[2, 1] - F[1, 1] * F[2, 0]))


def dice(a, b, threshold=0.5):
    """Dice overlap (Sec. 4.1, measures of performance) of the sets
    A = {a >= threshold} and B = {b >= threshold}: 2 |A and B| / (|A| + |B|),
    1 when both sets are empty.  Labels carried by a map are indicator
    functions transported with the state's SL steps, so a voxel belongs to the
    carried label when its transported indicator is at least 1/2."""
    A = np.asarray(a) >= threshold
    B = np.asarray(b) >= threshold
    na, nb = int(np.count_nonzero(A)), int(np.count_nonzero(B))
    if na + nb == 0:
        return 1.0
    return 2.0 * int(np.count_nonzero(A & B)) / (na + nb)


def cfl(v, p: Params):
    """CFL number: max over x of |v(x)|_2 * dt / min_c h_c."""
    v = _f64(v)
    return float(np.sqrt(np.max(np.sum(v * v, axis=0))) * p.dt / np.min(spacing(v.shape[1:])))


# ---------------------------------------------------------------------------
# Regularisation-parameter search and continuation (Sec. 3, "Parameter
# identification"), on top of register()
# ---------------------------------------------------------------------------

def _valid_solve(m0, m1, p, bv, bw, v0, jmin, check):
    from dataclasses import replace
    q = replace(p, beta_v=bv, beta_w=bw)
    v, rep = register(m0, m1, q, v0=v0)
    dj = detj(v, q)
    ok = rep["status"] != "line_search_failed" and (not check or (dj.min() >= jmin and dj.max() <= 1.0 / jmin))
    return v, ok, (float(dj.min()), float(dj.max()))


def param_search(m0, m1, p: Params, beta_v_max=1.0, beta_v_min=1e-5, beta_w_max=1e-5, beta_w_min=1e-7,
                 jmin=0.1, bisect_rtol=0.1, max_solves=40, v0=None):
    """Two-stage search of the paper: (i) beta_w = beta_w_max, beta_v from
    beta_v_max down by factors of 10 until the Jacobian bounds [jmin, 1/jmin]
    are breached, then bisection (arithmetic midpoints) between the last
    valid and the breaching value until their gap is below bisect_rtol times
    the valid one; (ii) beta_w down by factors of 10 while valid.  Every
    solve starts from the last valid velocity.  Returns (beta_v*, beta_w*,
    v, trace of (beta_v, beta_w, valid))."""
    n = m0.shape
    valid_v = np.zeros((3,) + n) if v0 is None else _f64(v0)
    trace = []
    bw, bv = beta_w_max, beta_v_max
    hi = lo = None
    while len(trace) < max_solves:
        v, ok, _ = _valid_solve(m0, m1, p, bv, bw, valid_v, jmin, True)
        trace.append((bv, bw, ok))
        if not ok:
            lo = bv
            break
        hi, valid_v = bv, v
        if bv / 10.0 < beta_v_min:
            break
        bv /= 10.0
    if hi is None:
        return beta_v_max, bw, v, trace
    if lo is not None:
        while len(trace) < max_solves and (hi - lo) > bisect_rtol * hi:
            mid = 0.5 * (hi + lo)
            v, ok, _ = _valid_solve(m0, m1, p, mid, bw, valid_v, jmin, True)
            trace.append((mid, bw, ok))
            if ok:
                hi, valid_v = mid, v
            else:
                lo = mid
    bw_star = bw
    while len(trace) < max_solves and bw_star / 10.0 >= beta_w_min and bw_star > 0:
        v, ok, _ = _valid_solve(m0, m1, p, hi, bw_star / 10.0, valid_v, jmin, True)
        trace.append((hi, bw_star / 10.0, ok))
        if not ok:
            break
        bw_star /= 10.0
        valid_v = v
    return hi, bw_star, valid_v, trace


def param_continuation(m0, m1, p: Params, target_beta_v, target_beta_w, beta_v_max=1.0, beta_w_max=1e-5,
                       v0=None):
    """beta_v = beta_v_max, /10, ..., 10^ceil(log10 target), then the target
    (beta_w = beta_w_max); then beta_w /10 down to the target.  Each solve
    starts from the previous one.  Returns (v, list of (beta_v, beta_w))."""
    n = m0.shape
    v = np.zeros((3,) + n) if v0 is None else _f64(v0)
    bw0 = max(beta_w_max, target_beta_w)
    stop = 10.0 ** math.ceil(math.log10(target_beta_v))
    steps = []
    bv = beta_v_max
    while bv >= stop * (1 - 1e-12):
        steps.append((bv, bw0))
        bv /= 10.0
    if abs(stop - target_beta_v) > 1e-12 * target_beta_v:
        steps.append((target_beta_v, bw0))
    bw = bw0 / 10.0
    while bw >= target_beta_w * (1 - 1e-12):
        steps.append((target_beta_v, bw))
        bw /= 10.0
    for bv, bw in steps:
        v, _, _ = _valid_solve(m0, m1, p, bv, bw, v, 0.1, False)
    return v, steps
