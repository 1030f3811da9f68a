"""GPU parity of the reverse-mode (differentiable) SL transport.

claire_transport_vjp returns the exact derivative of the discrete forward
transport m(1) = T(v)^nt m0 (Sec. 2.2 SL scheme with RK2 characteristics).
It is checked against the FP64 oracle's transport_vjp (itself pinned to
central differences of the oracle's forward map), against finite differences
of the GPU forward map, against the adjoint identity at a size the oracle does
not reach, and for bitwise determinism (fixed-point scatter accumulation).

Tolerances: the image cotangent is nt scatter transposes of FP32 weights
(each output a sum of <= 64 FP32 products, summed exactly in 64-bit fixed
point): relative L2 1e-5.  The velocity cotangent adds the interpolant
gradient of each state (64-term FP32 sums of derivative weights) times the
cotangent and the predictor terms: relative L2 1e-4.  Cubic B-splines add one
FP32 prefilter (a forward and an inverse transform, symbol at most 27) per
step and per predictor component, which stays within the same bounds.
"""
import numpy as np
import pytest

import __graft_entry__ as entry
import oracle
from paper_2209_08189_gb300 import synth

pytestmark = pytest.mark.gpu


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


def dev(torch, a):
    return torch.from_numpy(f32(a)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def make_ctx(claire, torch, n, nt=4, **opts):
    return claire.Context(n, 1e-2, nt, stream=torch.cuda.current_stream().cuda_stream, **opts)


def inputs(n, seed, vmax=1.0):
    rng = np.random.default_rng(seed)
    m0 = synth.blob_template(n, seed=seed + 1, sigma=0.9)
    v = synth.mode_velocity(n, seed=seed + 2, vmax=vmax, kmax=3)
    gbar = rng.standard_normal(n)
    return f32(m0), f32(v), f32(gbar)


TOL = {3: (1e-5, 1e-4), 1: (1e-5, 1e-4), 4: (1e-5, 1e-4)}


@pytest.mark.parametrize("order", [3, 1, 4])
@pytest.mark.parametrize("n", [(32, 32, 32), (40, 36, 30), (16, 24, 8)])
def test_vjp_matches_oracle(env, n, order):
    torch, claire = env
    nt = 4
    m0, v, gbar = inputs(n, 11)
    ctx = make_ctx(claire, torch, n, nt=nt, interp=order)
    gm0 = torch.empty(n, device="cuda")
    gv = torch.empty((3,) + n, device="cuda")
    ctx.transport_vjp(dev(torch, v), dev(torch, m0), dev(torch, gbar), gm0, gv)
    torch.cuda.synchronize()
    rm0, rv = oracle.transport_vjp(m0, v, gbar, oracle.Params(nt=nt, order=order))
    e_m, e_v = rel_l2(host(gm0), rm0), rel_l2(host(gv), rv)
    print("order %d grid %s: gm0 rel L2 %.2e, gv rel L2 %.2e" % (order, n, e_m, e_v))
    assert e_m < TOL[order][0]
    assert e_v < TOL[order][1]


def test_vjp_bitwise_deterministic_and_checkpointing(env):
    """Two calls give identical bits (fixed-point scatter), and recomputing the
    states from m0 (checkpointing) gives the same bits as storing them."""
    torch, claire = env
    n = (48, 40, 36)
    m0, v, gbar = inputs(n, 5, vmax=2.0)
    ctx = make_ctx(claire, torch, n, nt=6)
    args = (dev(torch, v), dev(torch, m0), dev(torch, gbar))
    outs = []
    for recompute in (False, False, True):
        gm0 = torch.empty(n, device="cuda")
        gv = torch.empty((3,) + n, device="cuda")
        ctx.transport_vjp(*args, gm0, gv, recompute=recompute)
        outs.append((gm0.clone(), gv.clone()))
    torch.cuda.synchronize()
    for a, b in outs[1:]:
        assert torch.equal(a, outs[0][0])
        assert torch.equal(b, outs[0][1])


@pytest.mark.parametrize("order", [3, 1, 4])
def test_vjp_finite_differences_of_gpu_forward(env, order):
    """Directional derivatives of the mismatch L(m0, v) = 1/2 |m(1) - m1|^2
    (gbar = m(1) - m1) agree with central differences of the GPU forward
    transport: relative error < 1e-3.  The loss is smooth in v except where a
    characteristic crosses a cell face (the interpolant is piecewise
    polynomial); with smooth images those kinks cost < 6e-4 at eps = 3e-3
    (measured on the FP64 oracle), below the bound."""
    torch, claire = env
    n = (32, 32, 32)
    nt = 4
    m0, v, _ = inputs(n, 21)
    m1 = f32(synth.blob_template(n, seed=99, sigma=0.9))
    rng = np.random.default_rng(22)
    dv_dir = f32(synth.mode_velocity(n, seed=23, vmax=1.0, kmax=2))
    dm_dir = f32(rng.standard_normal(n))
    ctx = make_ctx(claire, torch, n, nt=nt, interp=order)

    def fwd(mm, vv):
        out = torch.empty(n, device="cuda")
        ctx.transport(dev(torch, vv), dev(torch, mm), out)
        torch.cuda.synchronize()
        return host(out)

    def L(mm, vv):
        return 0.5 * float(np.sum((fwd(mm, vv) - m1) ** 2))

    gbar = f32(fwd(m0, v) - m1)
    gm0 = torch.empty(n, device="cuda")
    gv = torch.empty((3,) + n, device="cuda")
    ctx.transport_vjp(dev(torch, v), dev(torch, m0), dev(torch, gbar), gm0, gv)
    eps = 3e-3
    fdv = (L(m0, v + eps * dv_dir) - L(m0, v - eps * dv_dir)) / (2 * eps)
    fdm = (L(m0 + eps * dm_dir, v) - L(m0 - eps * dm_dir, v)) / (2 * eps)
    adv = float(np.sum(host(gv) * dv_dir))
    adm = float(np.sum(host(gm0) * dm_dir))
    print("order %d: fd_v %.6e vjp %.6e; fd_m %.6e vjp %.6e" % (order, fdv, adv, fdm, adm))
    assert abs(fdv - adv) < 1e-3 * abs(fdv)
    assert abs(fdm - adm) < 1e-3 * abs(fdm)


def test_vjp_adjoint_identity_128(env):
    """<gm0, x> = <gbar, T x> for any x (the image cotangent is the transpose
    of the linear map m0 -> m(1)); checked at 128^3 where the oracle is slow."""
    torch, claire = env
    n = (128, 128, 128)
    m0, v, gbar = inputs(n, 31, vmax=1.5)
    x = f32(np.random.default_rng(32).standard_normal(n))
    ctx = make_ctx(claire, torch, n, nt=4)
    gm0 = torch.empty(n, device="cuda")
    ctx.transport_vjp(dev(torch, v), dev(torch, m0), dev(torch, gbar), gm0, None, recompute=True)
    tx = torch.empty(n, device="cuda")
    ctx.transport(dev(torch, v), dev(torch, x), tx)
    torch.cuda.synchronize()
    lhs = float(np.sum(host(gm0) * x))
    rhs = float(np.sum(host(tx) * gbar))
    scale = float(np.linalg.norm(host(gm0)) * np.linalg.norm(x))
    assert abs(lhs - rhs) < 1e-6 * scale


def test_vjp_zero_cotangent_and_optional_outputs(env):
    torch, claire = env
    n = (16, 24, 8)
    m0, v, gbar = inputs(n, 41)
    ctx = make_ctx(claire, torch, n)
    gm0 = torch.full(n, 7.0, device="cuda")
    gv = torch.full((3,) + n, 7.0, device="cuda")
    ctx.transport_vjp(dev(torch, v), dev(torch, m0), torch.zeros(n, device="cuda"), gm0, gv)
    torch.cuda.synchronize()
    assert float(gm0.abs().max()) == 0.0 and float(gv.abs().max()) == 0.0
    # each output alone equals the joint call
    a_m = torch.empty(n, device="cuda")
    a_v = torch.empty((3,) + n, device="cuda")
    ctx.transport_vjp(dev(torch, v), dev(torch, m0), dev(torch, gbar), a_m, a_v)
    b_m = torch.empty(n, device="cuda")
    ctx.transport_vjp(dev(torch, v), dev(torch, m0), dev(torch, gbar), b_m, None)
    b_v = torch.empty((3,) + n, device="cuda")
    ctx.transport_vjp(dev(torch, v), dev(torch, m0), dev(torch, gbar), None, b_v)
    torch.cuda.synchronize()
    assert torch.equal(a_m, b_m) and torch.equal(a_v, b_v)
    with pytest.raises(claire.ClaireError):
        claire.claire_transport_vjp(ctx.handle, dev(torch, v), dev(torch, m0), dev(torch, gbar), None, None, 6)


def test_autograd_function(env):
    """sl_transport under torch.autograd returns the C-ABI cotangents."""
    torch, claire = env
    n = (24, 20, 16)
    m0, v, gbar = inputs(n, 51)
    ctx = make_ctx(claire, torch, n)
    tm0 = dev(torch, m0).requires_grad_(True)
    tv = dev(torch, v).requires_grad_(True)
    out = claire.sl_transport(ctx, tm0, tv)
    ref = torch.empty(n, device="cuda")
    ctx.transport(dev(torch, v), dev(torch, m0), ref)
    assert torch.equal(out.detach(), ref)
    (out * dev(torch, gbar)).sum().backward()
    gm0 = torch.empty(n, device="cuda")
    gv = torch.empty((3,) + n, device="cuda")
    ctx.transport_vjp(dev(torch, v), dev(torch, m0), dev(torch, gbar), gm0, gv)
    torch.cuda.synchronize()
    assert torch.equal(tm0.grad, gm0)
    assert torch.equal(tv.grad, gv)
