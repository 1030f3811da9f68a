"""Pins of the oracle's coarse preconditioner correction (no GPU).

The two-level zero-velocity preconditioner (Sec. 2.2) inverts, on a coarse
grid, H0 = S + gbar gbar^T.  The learned correction weights its data term
pointwise, H0w = S + gbar w gbar^T with w >= 0 (w = 1: the paper's operator),
and the weight a predictor should reproduce is the least-squares fit of that
model to the data term of the true Gauss-Newton matvec on probe fields.  Pins:

* at v = 0 the Gauss-Newton data term is exactly gbar (gbar . p), so the fit
  returns w = 1 (a dropped trapezoid weight, a wrong sum or a transposed
  operand in the fit breaks this);
* w = 1 reproduces the paper's preconditioner bit for bit;
* a data term planted with a known block-constant weight is recovered exactly,
  negative fits are clipped to 0 and cells without image gradient get w = 1;
* with an exact inner solve, the coarse part of P^{-1} r solves
  (S + gbar w gbar^T) x = r on the kept coarse modes, the operator formed
  directly with w (a sqrt(w) applied twice, or w applied once to gbar, fails).
"""
import math

import numpy as np

import oracle
from oracle import inner, reg_apply
from paper_2209_08189_gb300 import synth


def _probes(n, count, seed0=100):
    return [synth.mode_velocity(n, seed=seed0 + i, kmax=3, vmax=0.3) for i in range(count)]


def test_fit_is_one_at_zero_velocity():
    n = (16, 16, 16)
    p = oracle.Params(nt=4, beta_v=1e-2, beta_w=1e-4)
    m0 = synth.blob_template(n, seed=2)
    m1 = synth.blob_template(n, seed=3)
    st = oracle.State(np.zeros((3,) + n), m0, m1, p)
    num, den = oracle.pc_weight_stats_at(st, _probes(n, 3))
    big = den > 1e-6 * den.max()
    assert np.max(np.abs(num[big] / den[big] - 1.0)) <= 1e-9
    w = oracle.pc_weight_fit(num, den, (8, 8, 8))
    assert np.max(np.abs(w - 1.0)) <= 1e-9


def test_unit_weight_is_the_paper_preconditioner():
    n, nc = (16, 16, 16), (8, 8, 8)
    p = oracle.Params(nt=4, beta_v=1e-2, beta_w=1e-4)
    gbar_c = oracle.restrict_spectral(synth.mode_velocity(n, seed=5, kmax=4, vmax=2.0), nc)
    r = synth.mode_velocity(n, seed=6, kmax=6, vmax=1.0)
    a = oracle.precond_two_level(r, gbar_c, p)
    b = oracle.precond_two_level(r, gbar_c, p, w=np.ones(nc))
    assert np.array_equal(a, b)


def test_fit_recovers_planted_block_weight():
    n, nc = (8, 8, 8), (4, 4, 4)
    rng = np.random.default_rng(7)
    gbar = synth.mode_velocity(n, seed=8, kmax=3, vmax=1.0)
    wstar = rng.uniform(0.2, 3.0, size=nc)
    wstar[0, 1, 2] = -0.5                  # a negative fit is clipped to 0
    gbar[:, 4:6, 2:4, 6:8] = 0.0           # coarse cell (2, 1, 3) has no gradient: w = 1
    wfine = np.repeat(np.repeat(np.repeat(wstar, 2, 0), 2, 1), 2, 2)
    probes = _probes(n, 4)
    terms = [gbar * wfine * np.sum(gbar * pv, axis=0) for pv in probes]
    num, den = oracle.pc_weight_stats(gbar, probes, terms)
    w = oracle.pc_weight_fit(num, den, nc)
    expect = np.maximum(wstar, 0.0)
    expect[2, 1, 3] = 1.0
    assert np.max(np.abs(w - expect)) <= 1e-12


def test_weighted_coarse_solve_uses_w_once():
    n, nc = (8, 8, 8), (4, 4, 4)
    p = oracle.Params(nt=4, beta_v=1e-2, beta_w=1e-4, pc_tol=0.0, pc_maxit=400)
    gbar_c = oracle.restrict_spectral(synth.mode_velocity(n, seed=9, kmax=2, vmax=3.0), nc)
    rng = np.random.default_rng(10)
    w = rng.uniform(0.1, 4.0, size=nc)
    r = synth.mode_velocity(n, seed=11, kmax=3, vmax=1.0)
    z = oracle.precond_two_level(r, gbar_c, p, w=w)
    # the coarse part of z (the kept coarse modes) and the coarse right-hand side
    xc = oracle._kept_modes(oracle.restrict_spectral(z, nc))
    rc = oracle._kept_modes(oracle.restrict_spectral(r, nc))

    def h0w(x):  # S x + gbar w (gbar . x), formed with w itself
        return oracle._kept_modes(reg_apply(x, p) + gbar_c * (w * np.sum(gbar_c * x, axis=0)))

    res = h0w(xc) - rc
    assert math.sqrt(inner(res, res, nc)) <= 1e-8 * math.sqrt(inner(rc, rc, nc))
    # w^2 in place of w does not solve it
    def h0w2(x):
        return oracle._kept_modes(reg_apply(x, p) + gbar_c * (w * w * np.sum(gbar_c * x, axis=0)))

    res2 = h0w2(xc) - rc
    assert math.sqrt(inner(res2, res2, nc)) > 1e-3 * math.sqrt(inner(rc, rc, nc))
