"""GPU parity at the benchmark's full size.

256^3 clinical-size workload (the one bench.py times): nested-label template,
band-limited v* (|k| <= 8, max |v| = 1, CFL 10 at nt = 4), reference by the
ORACLE's FP64 transport of the clean template, N(0, 0.02^2) noise on both
images (seeds 0 / 1), beta_v = 1e-2, beta_w = 1e-4.  Compared element by
element with the FP64 oracle on the same FP32 bits:
  * the full-field reduced gradient (Eq. (3)) and Gauss-Newton Hessian matvec
    (Eq. (6)) at v = v*/2, split as S x + body: the body (the SL transport
    part) at relative L2 1e-4 (2 nt SL steps of ~1e-6 rounding each, amplified
    by the cancellation in m1 - m(1)); S x, formed from an FP32 transform of x,
    within twice the transform roundoff the symbol S(k) amplifies at high |k|
    (fft_roundoff_bound; about 7e-3 of ||S x|| here);
  * a fixed-schedule registration (Eq. (5)), 2 Gauss-Newton x 5 PCG steps from
    v = 0: identical Armijo steps, final velocity relative L2 1e-3 and final
    relative mismatch within 1 % (stated requirements).
512^3 (the mixed-precision case's grid): one backtrace and one tricubic
interpolation checked on 10^6 sampled points, relative L-infinity 1e-5.
"""
import numpy as np
import pytest

import __graft_entry__ as entry
import oracle
from paper_2209_08189_gb300 import synth

from fp32_bounds import fft_roundoff_bound, split_check

pytestmark = pytest.mark.gpu

N256 = (256, 256, 256)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    entry.build()
    from paper_2209_08189_gb300 import claire
    return torch, claire


def f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


@pytest.fixture(scope="module")
def headline():
    """Images and parameters of the 256^3 workload; m1 from the oracle."""
    p = oracle.Params(nt=4, beta_v=1e-2, beta_w=1e-4)
    base = synth.label_template(N256, seed=0)
    vstar = synth.bandlimited_velocity(N256, seed=0, kmax=8, vmax=1.0)
    m1 = f32(synth.add_noise(oracle.transport(base, vstar, p), 0.02, seed=1))
    m0 = f32(synth.add_noise(base, 0.02, seed=0))
    return m0, m1, f32(vstar), p


def _ctx(claire, torch, p, **opts):
    return claire.Context(N256, p.beta_v, p.nt, beta_w=p.beta_w,
                          stream=torch.cuda.current_stream().cuda_stream, **opts)


def test_headline_256_gradient_and_matvec(env, headline):
    torch, claire = env
    m0, m1, vstar, p = headline
    v = f32(0.5 * vstar)
    vt = f32(synth.bandlimited_velocity(N256, seed=5, kmax=8, vmax=0.3))
    ctx = _ctx(claire, torch, p)
    ctx.set_images(torch.from_numpy(m0).cuda(), torch.from_numpy(m1).cuda())
    vd, vtd = torch.from_numpy(v).cuda(), torch.from_numpy(vt).cuda()
    g = torch.empty((3,) + N256, device="cuda")
    J = ctx.gradient(vd, g)
    Hv = torch.empty_like(g)
    ctx.hessian_matvec(vtd, Hv)
    sv = torch.empty_like(g)
    ctx.spectral(vd, sv, claire.SPECTRAL_REG)   # the same S v the gradient formed
    torch.cuda.synchronize()
    g_gpu, sv_gpu = g.cpu().numpy().astype(np.float64), sv.cpu().numpy().astype(np.float64)
    ctx.spectral(vtd, sv, claire.SPECTRAL_REG)
    torch.cuda.synchronize()
    h_gpu, svt_gpu = Hv.cpu().numpy().astype(np.float64), sv.cpu().numpy().astype(np.float64)
    ctx.close()
    del g, Hv, sv, vd, vtd
    st = oracle.State(v.astype(np.float64), m0.astype(np.float64), m1.astype(np.float64), p)
    assert abs(J - st.J) <= 1e-5 * abs(st.J)
    split_check(g_gpu, sv_gpu, oracle.gradient(st), st.reg_v, fft_roundoff_bound(N256, p, v))
    vt64 = vt.astype(np.float64)
    split_check(h_gpu, svt_gpu, oracle.hessian_matvec(st, vt64), oracle.reg_apply(vt64, p),
                 fft_roundoff_bound(N256, p, vt))


def test_headline_256_registration_fixed_schedule(env, headline):
    torch, claire = env
    m0, m1, vstar, p0 = headline
    p = oracle.Params(nt=4, beta_v=1e-2, beta_w=1e-4, gtol=0.0, max_gn=2, max_pcg=5, pcg_fixed=True)
    ctx = _ctx(claire, torch, p, gtol=0.0, max_gn=2, max_pcg=5, pcg_fixed=1)
    ctx.set_images(torch.from_numpy(m0).cuda(), torch.from_numpy(m1).cuda())
    v = torch.zeros((3,) + N256, device="cuda")
    st, rep = ctx.register(v, check=False)
    v_gpu = v.cpu().numpy().astype(np.float64)
    ctx.close()
    del v
    v_ref, rep_ref = oracle.register(m0.astype(np.float64), m1.astype(np.float64), p)
    assert rep["gn_iters"] == rep_ref["gn_iters"] == 2
    assert rep["alpha"] == rep_ref["alpha"]
    assert rel_l2(v_gpu, v_ref) <= 1e-3
    assert abs(rep["r"] - rep_ref["r"]) <= 0.01 * rep_ref["r"]
    assert abs(rep["cfl"] - oracle.cfl(v_gpu, p)) <= 1e-6 * rep["cfl"]


def test_512_backtrace_and_interpolation_sampled(env):
    """512^3 blob template, velocity of 6 modes |k| <= 16 per component with
    max |v| = 0.5 (CFL 10 at nt = 4): X and m0(X) on 10^6 random points."""
    torch, claire = env
    n = (512, 512, 512)
    m0 = f32(synth.blob_template(n, seed=0))
    vs = f32(synth.mode_velocity(n, seed=0, nmodes=6, kmax=16, vmax=0.5))
    ctx = claire.Context(n, 1e-2, 4, stream=torch.cuda.current_stream().cuda_stream)
    vd = torch.from_numpy(vs).cuda()
    d = torch.empty((3,) + n, device="cuda")
    ctx.backtrace(vd, d, 1)
    f = torch.from_numpy(m0).cuda()
    out = torch.empty(n, device="cuda")
    ctx.interp(f, d, out, 3)
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    idx = rng.integers(0, m0.size, size=1_000_000)
    ti = torch.from_numpy(idx).cuda()
    dh = d.reshape(3, -1)[:, ti].cpu().numpy().astype(np.float64)
    got = out.reshape(-1)[ti].cpu().numpy().astype(np.float64)
    ctx.close()
    del d, out, f, vd
    I, J, K = np.unravel_index(idx, n)
    # backtrace X = x - dt/2 (v(x) + v(x - dt v(x))) in grid units, from the FP32 velocity
    h = oracle.spacing(n)
    u = np.stack([vs[c].reshape(-1)[idx].astype(np.float64) / h[c] for c in range(3)])
    ys = np.stack([I - 0.25 * u[0], J - 0.25 * u[1], K - 0.25 * u[2]])
    us = np.stack([oracle.interp_points(vs[c].astype(np.float64), ys, 3) / h[c] for c in range(3)])
    dref = -0.125 * (u + us)
    assert np.max(np.abs(dh - dref)) <= 1e-5 * np.max(np.abs(dref))
    # interpolation at the GPU's departure points
    y = np.stack([I + dh[0], J + dh[1], K + dh[2]])
    ref = oracle.interp_points(m0.astype(np.float64), y, 3)
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(m0))
