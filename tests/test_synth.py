"""Seeded input generators: determinism and the closed forms they are built
from (no method arithmetic lives in synth)."""
import math

import numpy as np

from paper_2209_08189_gb300 import synth


def test_assoc_legendre_closed_form():
    """P_8^6(x) = (1 - x^2)^3 (d/dx)^6 P_8(x) = (1 - x^2)^3 (1013512.5 x^2 - 67567.5)."""
    x = np.linspace(-1, 1, 41)
    ref = (1 - x * x) ** 3 * (1013512.5 * x * x - 67567.5)
    assert np.max(np.abs(synth._assoc_legendre(8, 6, x) - ref)) < 1e-9 * np.max(np.abs(ref))
    # P_1^1 = -sqrt(1 - x^2), P_2^0 = (3x^2 - 1)/2
    assert np.allclose(synth._assoc_legendre(1, 1, x), -np.sqrt(1 - x * x))
    assert np.allclose(synth._assoc_legendre(2, 0, x), 0.5 * (3 * x * x - 1))


def test_syn_generators():
    n = (32, 32, 32)
    a = synth.syn_template(n, seed=1)
    b = synth.syn_template(n, seed=1)
    assert np.array_equal(a, b)
    assert set(np.unique(a)) <= set(range(11)) and a.max() >= 1
    v = synth.syn_velocity(n, K=4)
    x = synth.coords(n)[0] - math.pi
    # at y = x-row with j = i index: v_x(x, y, z) = sum k^-1/2 cos(k y) cos(k x)
    i, j, k = 3, 7, 11
    ref = sum(kk ** -0.5 * math.cos(kk * x[j]) * math.cos(kk * x[i]) for kk in range(1, 5))
    assert abs(v[0, i, j, k] - ref) < 1e-12


def test_sphere_template_labels():
    m, lab = synth.sphere_template((32, 32, 32), seed=0)
    assert set(np.unique(lab)) == {0, 1, 2, 3}
    assert m.dtype == np.float32 and 0 <= m.min() and m.max() <= 1.0 + 1e-6
