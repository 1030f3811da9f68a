"""The learned warm start on the GPU: the network trains on pairs the method
generates (its loss falls), and the trained network's guess gains over the
method without it: a lower starting mismatch and fewer Gauss-Newton
iterations to the same absolute gradient tolerance (g0_ref = |g(v=0)|),
ending at the same objective value and mismatch within a few percent.  The
tolerance is 1e-2 here so that both solves end near the same minimiser."""
import numpy as np
import pytest

import __graft_entry__ as entry
from paper_2209_08189_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    entry.build()
    from paper_2209_08189_gb300 import claire, net, warmstart
    return torch, claire, net, warmstart


@pytest.fixture(scope="module")
def trained(env):
    torch, claire, net, warmstart = env
    st = torch.cuda.current_stream().cuda_stream
    src = warmstart.PairSource(32, n_templates=8, n_velocities=24, kmax=(2, 4), vmax=(0.4, 1.0), noise=0.0,
                               seed=5)
    u = net.UNet(seed=1, stream=st)
    hist = warmstart.train(u, src, steps=400, batch=4, lr=2e-3, lr_final=2e-4, wv=1.0, wm=1.0, log_every=50)
    return u, hist


def test_training_reduces_loss(trained):
    u, hist = trained
    for it, lv, lm, t, *_ in hist:
        print("step %4d  Lv %.4f  mismatch rel %.4f  %.1fs" % (it, lv, lm, t))
    first = np.mean([h[1] for h in hist[:1]])
    last = np.mean([h[1] for h in hist[-2:]])
    assert last < 0.5 * first
    assert hist[-1][2] < hist[0][2]


def test_warm_start_gains_over_zero_init(env, trained):
    torch, claire, net, warmstart = env
    u, _ = trained
    n = 32
    grid = (n, n, n)
    st = torch.cuda.current_stream().cuda_stream
    m0 = torch.from_numpy(synth.blob_template(grid, seed=777, nblobs=8, sigma=0.35).astype(np.float32)).cuda()
    vstar = torch.from_numpy(synth.bandlimited_velocity(grid, seed=778, kmax=3, vmax=0.8).astype(np.float32)).cuda()
    ctx = claire.Context(grid, 1e-2, 4, stream=st, gtol=1e-2, max_gn=30)
    m1 = torch.empty(grid, device="cuda")
    ctx.transport(vstar, m0, m1)
    ctx.set_images(m0, m1)
    g = torch.empty((3,) + grid, device="cuda")
    zero = torch.zeros((3,) + grid, device="cuda")
    ctx.gradient(zero, g)
    g0 = float(g.double().norm())
    # from zero
    v = torch.zeros((3,) + grid, device="cuda")
    _, rep0 = ctx.register(v)
    # from the network's guess, same absolute tolerance
    ws = warmstart.WarmStart(u, n)
    vw = torch.empty((3,) + grid, device="cuda")
    ws.predict(m0, m1, vw)
    J_w, mis_w = ctx.objective(vw)
    J_0, mis_0 = ctx.objective(zero)
    ctx.set_opts(g0_ref=g0)
    _, repw = ctx.register(vw)
    print("mismatch at guess %.3e vs at zero %.3e; GN %d (warm) vs %d (zero); PCG %d vs %d; "
          "J %.5e vs %.5e; r %.4f vs %.4f"
          % (mis_w, mis_0, repw["gn_iters"], rep0["gn_iters"], repw["pcg_iters_total"], rep0["pcg_iters_total"],
             repw["J"], rep0["J"], repw["r"], rep0["r"]))
    assert mis_w < 0.5 * mis_0
    assert repw["gn_iters"] < rep0["gn_iters"]
    assert repw["J"] <= 1.03 * rep0["J"]
    assert repw["r"] <= 1.1 * rep0["r"]


def test_warm_start_prolongs_to_finer_grid(env, trained):
    """Inference on a 64^3 pair: images sampled to 32^3, velocity prolonged spectrally."""
    torch, claire, net, warmstart = env
    u, _ = trained
    n = 64
    grid = (n, n, n)
    st = torch.cuda.current_stream().cuda_stream
    m0 = torch.from_numpy(synth.blob_template(grid, seed=779, nblobs=8, sigma=0.35).astype(np.float32)).cuda()
    vstar = torch.from_numpy(synth.bandlimited_velocity(grid, seed=780, kmax=3, vmax=0.8).astype(np.float32)).cuda()
    ctx = claire.Context(grid, 1e-2, 4, stream=st)
    m1 = torch.empty(grid, device="cuda")
    ctx.transport(vstar, m0, m1)
    ctx.set_images(m0, m1)
    vw = torch.empty((3,) + grid, device="cuda")
    warmstart.WarmStart(u, 32).predict(m0, m1, vw)
    _, mis_w = ctx.objective(vw)
    _, mis_0 = ctx.objective(torch.zeros((3,) + grid, device="cuda"))
    print("64^3: mismatch at prolonged guess %.3e vs at zero %.3e" % (mis_w, mis_0))
    assert mis_w < 0.7 * mis_0


def test_resample_spectral_roundtrip_and_nearest(env):
    """Prolongation of a band-limited field is exact; restriction after
    prolongation returns the input; nearest sampling picks grid values."""
    torch, claire, net, warmstart = env
    st = torch.cuda.current_stream().cuda_stream
    c = (16, 12, 20)
    f = (32, 24, 40)
    v = synth.bandlimited_velocity(c, seed=3, kmax=4, vmax=1.0).astype(np.float32)
    vc = torch.from_numpy(v).cuda()
    vf = torch.empty((3,) + f, device="cuda")
    claire.claire_resample(vc, c, vf, f, 3, claire.RESAMPLE_SPECTRAL, st)
    back = torch.empty((3,) + c, device="cuda")
    claire.claire_resample(vf, f, back, c, 3, claire.RESAMPLE_SPECTRAL, st)
    nn_ = torch.empty((3,) + c, device="cuda")
    claire.claire_resample(vf, f, nn_, c, 3, claire.RESAMPLE_NEAREST, st)
    torch.cuda.synchronize()
    assert np.max(np.abs(back.cpu().numpy() - v)) < 1e-5
    # the fine field restricted to even nodes is the coarse field
    assert np.max(np.abs(vf.cpu().numpy()[:, ::2, ::2, ::2] - v)) < 1e-5
    assert np.array_equal(nn_.cpu().numpy(), vf.cpu().numpy()[:, ::2, ::2, ::2])


def test_preconditioner_head_learns_the_weight_fit(env):
    """A network with the preconditioner head fits the weight of one fixed
    pair (the weight-fit loss alone, the same two probe fields every step, so
    the target is fixed):
    the loss falls well below its value at w = 1, the predicted weight is
    positive and finite, and the two-level preconditioner accepts it."""
    torch, claire, net, warmstart = env
    st = torch.cuda.current_stream().cuda_stream
    src = warmstart.PairSource(32, n_templates=1, n_velocities=1, kmax=(3, 3), vmax=(0.8, 0.8), noise=0.0,
                               seed=9)
    u = net.UNet(seed=2, stream=st, pc_head=True)
    hist = warmstart.train(u, src, steps=200, batch=1, lr=1e-3, wv=0.0, wm=0.0, log_every=10, wpc=1.0,
                           pc_probes=2, pc_pool=2, pc_target="fit")
    for it, lv, lm, t, lpc in hist:
        print("step %4d  Lpc %.5f  %.1fs" % (it, lpc, t))
    first = hist[0][4]
    last = float(np.mean([h[4] for h in hist[-4:]]))
    assert np.isfinite(last) and last < 0.5 * first
    ws = warmstart.WarmStart(u, 32)
    grid = (32, 32, 32)
    m0, m1, _ = src.batch(1)
    v = torch.empty((3,) + grid, device="cuda")
    ws.predict(m0[0], m1[0], v)
    w = torch.empty((16, 16, 16), device="cuda")
    ws.pc_weight(w)
    torch.cuda.synchronize()
    wh = w.cpu().numpy()
    assert np.all(np.isfinite(wh)) and wh.min() > 0.0
    ctx = claire.Context(grid, 1e-2, 4, stream=st, precond=claire.PRECOND_TWO_LEVEL)
    ctx.set_images(m0[0].contiguous(), m1[0].contiguous())
    g = torch.empty((3,) + grid, device="cuda")
    ctx.gradient(v, g)
    ctx.set_pc_weight(w)
    z = torch.empty_like(g)
    ctx.precond(g, z)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(z.cpu().numpy()))
    ctx.close()
    src.ctx.close()


def test_scale_target_rule(env):
    """pc_scale_target returns a weight of the list with finite positive
    first-step decreases; on constant images (gbar = 0, g = S v) the coarse
    operator does not depend on the weight, so every decrease is the same
    and the smallest weight, 1, is returned."""
    torch, claire, net, warmstart = env
    st = torch.cuda.current_stream().cuda_stream
    grid = (32, 32, 32)
    m0 = torch.from_numpy(synth.blob_template(grid, seed=4).astype(np.float32)).cuda()
    vstar = torch.from_numpy(synth.bandlimited_velocity(grid, seed=5, kmax=3, vmax=0.8).astype(np.float32)).cuda()
    ctx = claire.Context(grid, 1e-2, 4, stream=st, precond=claire.PRECOND_TWO_LEVEL)
    m1 = torch.empty(grid, device="cuda")
    ctx.transport(vstar, m0, m1)
    ctx.set_images(m0, m1)
    consts = [torch.full((16, 16, 16), c, device="cuda") for c in warmstart.PC_SCALES]
    g, z, hz = (torch.empty((3,) + grid, device="cuda") for _ in range(3))
    c, qs = warmstart.pc_scale_target(ctx, (0.5 * vstar).contiguous(), g, z, hz, consts)
    assert c in warmstart.PC_SCALES and all(np.isfinite(q) and q > 0 for q in qs)
    flat = torch.full(grid, 0.5, device="cuda")
    ctx.set_images(flat, flat)
    c0, q0 = warmstart.pc_scale_target(ctx, (0.5 * vstar).contiguous(), g, z, hz, consts)
    assert c0 == 1.0 and min(q0) > 0 and max(q0) == min(q0)
    ctx.close()
