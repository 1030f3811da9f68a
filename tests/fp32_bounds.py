"""Rounding bound of FP32 spectral operators, used by the GPU parity tests.

The regulariser S v (Sec. 2.1-2.2) is formed on the GPU from an FP32 forward
transform of v.  That transform's roundoff is about eps32 sqrt(log2 N) ||v||
and, unlike the rounding of v itself, is spread roughly evenly over all modes;
the symbol S(k) = a I + c u u^T then multiplies it by up to
beta_w (1 + |k|^2) |k|^2 at the highest wavenumbers (2.4e5 at 256^3), so the
error of S v grows as n^4 while the transport part stays at FP32 rounding.
The bound takes the root mean square of S's eigenvalues over the modes.
"""
import numpy as np

import oracle

EPS32 = 2.0 ** -24


def fft_roundoff_bound(n, p, v):
    """L2 bound on the error of S v (3 components) formed from an FP32 transform of v."""
    a, c, u, kk = oracle._symbols(n, p)
    lam_l = a + c * np.sum(u * u, axis=0)           # longitudinal eigenvalue; a twice transverse
    rms = float(np.sqrt(np.mean((lam_l ** 2 + 2 * a ** 2) / 3.0)))
    return EPS32 * np.sqrt(np.log2(float(np.prod(n)))) * rms * float(np.linalg.norm(v))


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def split_check(total, s_gpu, total_ref, s_ref, bound, body_tol=1e-4):
    """total = S x + body: the body (the SL transport part) at body_tol relative
    L2; S x within twice the transform-roundoff bound; the sum within both."""
    body, body_ref = total - s_gpu, total_ref - s_ref
    assert rel_l2(body, body_ref) <= body_tol, rel_l2(body, body_ref)
    es = float(np.linalg.norm(s_gpu - s_ref))
    assert es <= 2.0 * bound + 1e-6 * float(np.linalg.norm(s_ref)), (es, bound)
    et = float(np.linalg.norm(total - total_ref))
    assert et <= 2.0 * bound + body_tol * float(np.linalg.norm(total_ref)), (et, bound)
