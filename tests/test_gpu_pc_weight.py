"""GPU parity of the coarse preconditioner correction (the learned warm
start's second output) against the FP64 oracle and plain definitions.

* The weighted two-level preconditioner, coarse operator S + gbar_c w gbar_c^T
  (claire_set_pc_weight), against oracle.precond_two_level(w=...) with a fixed
  number of inner iterations on both sides (relative L2 1e-4, the tolerance of
  the unweighted application test); w = 1 gives the same bits as no weight.
* The mean state gradient gbar (claire_mean_state_gradient) against
  oracle.mean_state_gradient (relative L2 1e-5).
* The fit statistics (claire_net_pcw_stats) against oracle.pc_weight_stats on
  the same FP32 inputs; the training loss and its gradient (claire_net_pcw_loss)
  and the weight w = softplus(o) (claire_net_pcw_weight) against their plain
  numpy definitions (relative 1e-5).
* Argument errors: a weight on the wrong grid, a non-finite weight.
"""
import ctypes

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
    from paper_2209_08189_gb300 import claire, net
    return torch, claire, net


def f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def dev(torch, a):
    return torch.from_numpy(f32(a)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def _setup(claire, torch, n, coarse, grad_form=0, maxit=6):
    m0 = f32(synth.blob_template(n, seed=1))
    vs = synth.mode_velocity(n, seed=2, kmax=3, vmax=0.5)
    p = oracle.Params(nt=4, beta_v=1e-2, beta_w=1e-4, grad_form=grad_form, precond="2l", pc_coarse=coarse,
                      pc_tol=0.0, pc_maxit=maxit)
    m1 = f32(oracle.transport(m0.astype(np.float64), vs, p))
    v = f32(0.5 * vs)
    ctx = claire.Context(n, p.beta_v, p.nt, stream=torch.cuda.current_stream().cuda_stream, beta_w=p.beta_w,
                         grad_form=grad_form, precond=claire.PRECOND_TWO_LEVEL, pc_coarse=coarse, pc_tol=0.0,
                         pc_maxit=maxit)
    ctx.set_images(dev(torch, m0), dev(torch, m1))
    g = torch.empty((3,) + n, device="cuda")
    ctx.gradient(dev(torch, v), g)
    st = oracle.State(v.astype(np.float64), m0.astype(np.float64), m1.astype(np.float64), p)
    return ctx, g, st, p


@pytest.mark.parametrize("n,coarse", [((24, 20, 16), 2), ((32, 32, 32), 4)])
def test_weighted_two_level_application_parity(env, n, coarse):
    torch, claire, _ = env
    ctx, g, st, p = _setup(claire, torch, n, coarse)
    nc = tuple(s // coarse for s in n)
    rng = np.random.default_rng(3)
    w = f32(rng.uniform(0.0, 3.0, size=nc))
    w[0, 0, :2] = -1.0  # negative weights act as 0
    ctx.set_pc_weight(dev(torch, w))
    z = torch.empty_like(g)
    ctx.precond(g, z)
    torch.cuda.synchronize()
    gbar_c = oracle.restrict_spectral(oracle.mean_state_gradient(st), nc)
    ref = oracle.precond_two_level(host(g), gbar_c, p, w=w.astype(np.float64))
    assert rel_l2(host(z), ref) <= 1e-4
    # the weight acts: the unweighted preconditioner differs
    assert rel_l2(ref, oracle.precond_two_level(host(g), gbar_c, p)) > 1e-3
    # host weights are accepted the same way
    ctx.set_pc_weight(w)
    z2 = torch.empty_like(g)
    ctx.precond(g, z2)
    torch.cuda.synchronize()
    assert torch.equal(z, z2)
    ctx.close()


def test_unit_weight_is_bit_identical_to_no_weight(env):
    torch, claire, _ = env
    n = (32, 32, 32)
    ctx, g, _, _ = _setup(claire, torch, n, 2)
    z0 = torch.empty_like(g)
    ctx.precond(g, z0)
    ctx.set_pc_weight(torch.ones((16, 16, 16), device="cuda"))
    z1 = torch.empty_like(g)
    ctx.precond(g, z1)
    ctx.set_pc_weight(None)
    z2 = torch.empty_like(g)
    ctx.precond(g, z2)
    torch.cuda.synchronize()
    assert torch.equal(z0, z1) and torch.equal(z0, z2)
    ctx.close()


def test_mean_state_gradient_parity(env):
    torch, claire, _ = env
    n = (24, 20, 16)
    ctx, g, st, _ = _setup(claire, torch, n, 2)
    gb = torch.empty_like(g)
    ctx.mean_state_gradient(gb)
    torch.cuda.synchronize()
    assert rel_l2(host(gb), oracle.mean_state_gradient(st)) <= 1e-5
    ctx.close()


def test_pc_weight_argument_errors(env):
    torch, claire, _ = env
    n = (32, 32, 32)
    ctx, g, _, _ = _setup(claire, torch, n, 2)
    with pytest.raises(claire.ClaireError) as e:
        ctx.set_pc_weight(torch.ones((8, 8, 8), device="cuda"))
    assert e.value.status == -1  # CLAIRE_EINVAL: not the coarse grid 16^3
    bad = torch.ones((16, 16, 16), device="cuda")
    bad[3, 4, 5] = float("nan")
    with pytest.raises(claire.ClaireError) as e:
        ctx.set_pc_weight(bad)
    assert e.value.status == -5  # CLAIRE_ENONFINITE
    # the rejected weight is not in use: the preconditioner is the paper's
    z0 = torch.empty_like(g)
    ctx.precond(g, z0)
    ctx.set_pc_weight(None)
    z1 = torch.empty_like(g)
    ctx.precond(g, z1)
    torch.cuda.synchronize()
    assert torch.equal(z0, z1)
    ctx.close()


def _softplus(o):
    return np.where(o > 20.0, o, np.log1p(np.exp(np.minimum(o, 20.0))))


def test_pcw_stats_loss_and_weight_kernels(env):
    torch, claire, net = env
    L = net.lib()
    st = torch.cuda.current_stream().cuda_stream
    n = (8, 12, 16)
    N = int(np.prod(n))
    rng = np.random.default_rng(4)
    gbar, pv, hp, sp = (f32(rng.standard_normal((3,) + n)) for _ in range(4))
    num0 = f32(rng.uniform(-0.1, 0.1, size=n))
    den0 = f32(rng.uniform(0.0, 0.1, size=n))
    num, den = dev(torch, num0), dev(torch, den0)
    ins = [dev(torch, a) for a in (gbar, pv, hp, sp)]  # kept alive until the kernels have run
    net._check(L.claire_net_pcw_stats(ins[0].data_ptr(), ins[1].data_ptr(), ins[2].data_ptr(), ins[3].data_ptr(),
                                      N, num.data_ptr(), den.data_ptr(), st), "pcw_stats")
    torch.cuda.synchronize()
    rn, rd = oracle.pc_weight_stats(gbar, [pv], [hp.astype(np.float64) - sp])
    assert rel_l2(host(num), rn + num0) <= 1e-5
    assert rel_l2(host(den), rd + den0) <= 1e-5
    # loss and gradient of w = softplus(o) against the pooled statistics
    o = f32(rng.standard_normal(n) * 2.0)
    o[0, 0, 0] = 25.0  # the linear branch of softplus
    numv, denv = host(num), host(den)
    denv[0:2, 2:4, 4:6] = 0.0  # a cell without statistics
    den = dev(torch, denv)
    dout = torch.empty(n, device="cuda")
    sums = torch.zeros(2, dtype=torch.float64, device="cuda")
    g3 = (ctypes.c_int * 3)(*n)
    od = dev(torch, o)
    net._check(L.claire_net_pcw_loss(od.data_ptr(), num.data_ptr(), den.data_ptr(), g3, 0.5, dout.data_ptr(),
                                     sums.data_ptr(), st), "pcw_loss")
    wdev = torch.empty(n, device="cuda")
    net._check(L.claire_net_pcw_weight(od.data_ptr(), wdev.data_ptr(), N, st), "pcw_weight")
    torch.cuda.synchronize()
    pool = lambda f: f.reshape(n[0] // 2, 2, n[1] // 2, 2, n[2] // 2, 2).sum(axis=(1, 3, 5))
    up = lambda c: np.repeat(np.repeat(np.repeat(c, 2, 0), 2, 1), 2, 2)
    A, B = up(pool(denv)), up(pool(numv))
    T = denv.sum()
    o64 = o.astype(np.float64)
    w = _softplus(o64)
    sig = 1.0 / (1.0 + np.exp(-o64))
    ref_d = 0.5 * 2.0 * (A * w - B) * sig / (8.0 * T)
    pos = A > 0
    ref_L = np.sum((A * w * w - 2.0 * B * w + B * B / np.where(pos, A, 1.0))[pos]) / (8.0 * T)
    s = host(sums)
    assert abs(s[0] - T) <= 1e-6 * T
    assert abs(s[1] - ref_L) <= 1e-5 * abs(ref_L)
    assert rel_l2(host(dout), ref_d) <= 1e-5
    assert rel_l2(host(wdev), w) <= 1e-6


def test_learned_weight_cuts_outer_iterations_at_256(env):
    """The committed network's coarse preconditioner weight on the 256^3
    clinical-size pair (FP16 storage, two-level preconditioner, the network's
    own warm start, stop at 5e-2 |g(v = 0)|): fewer outer PCG iterations than
    the paper's two-level preconditioner alone (w = 1), at the same objective
    within 1 %."""
    torch, claire, net = env
    import os
    from paper_2209_08189_gb300 import warmstart
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2209_08189_gb300",
                        "weights", "unet_warmstart_pc_128.npz")
    if not os.path.exists(path):
        pytest.skip("no network with the preconditioner head")
    st = torch.cuda.current_stream().cuda_stream
    grid = (256, 256, 256)
    N = 256 ** 3
    base = dev(torch, synth.label_template(grid, seed=0))
    vstar = dev(torch, synth.bandlimited_velocity(grid, seed=0, kmax=8, vmax=1.0))
    ctx32 = claire.Context(grid, 1e-2, 4, stream=st, beta_w=1e-4)
    m1c = torch.empty(grid, device="cuda")
    ctx32.transport(vstar, base, m1c, claire.TRANSPORT_FWD)
    m0 = dev(torch, synth.add_noise(host(base), 0.02, seed=0))
    m1 = dev(torch, synth.add_noise(host(m1c), 0.02, seed=1))
    ctx32.set_images(m0, m1)
    zero = torch.zeros((3,) + grid, device="cuda")
    g = torch.empty_like(zero)
    ctx32.gradient(zero, g)
    g0 = float(np.sqrt(claire.claire_dot(ctx32.handle, g, g, 3 * N)))
    ctx = claire.Context(grid, 1e-2, 4, stream=st, beta_w=1e-4, gtol=5e-2, max_gn=50, max_pcg=50,
                         storage=claire.STORAGE_F16, g0_ref=g0, precond=claire.PRECOND_TWO_LEVEL)
    ctx.set_images(m0, m1)
    u = net.UNet.from_file(path, stream=st)
    ws = warmstart.WarmStart(u, int(u.meta["n_net"]))
    v0 = torch.empty_like(zero)
    ws.predict(m0, m1, v0)
    w = torch.empty((128, 128, 128), device="cuda")
    ws.pc_weight(w)
    out = {}
    for name, wt in (("paper", None), ("learned", w)):
        ctx.set_pc_weight(wt)
        v = v0.clone()
        status, rep = ctx.register(v, check=False)
        assert status == 0, (name, rep)
        out[name] = (rep["pcg_iters_total"], ctx32.objective(v)[0])
    print("outer PCG / J: paper %d / %.6f, learned weight %d / %.6f (w mean %.3f)"
          % (out["paper"][0], out["paper"][1], out["learned"][0], out["learned"][1], float(w.mean())))
    assert out["learned"][0] < out["paper"][0]
    assert abs(out["learned"][1] - out["paper"][1]) <= 0.01 * out["paper"][1]
    ctx.close()
    ctx32.close()
