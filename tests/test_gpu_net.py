"""GPU parity of the warm-start network kernels against the FP64 oracle
(oracle/net.py) on identical BF16-representable inputs.

Tolerances: BF16 outputs (activations) are a rounded FP32 accumulation of
exact BF16 products, so each element is within 2^-8 of the FP64 value
relative to its magnitude, plus the FP32 rounding of a sum of up to 27*192
terms (abs 1e-3 of the output's RMS is far above it).  FP32 outputs (weight
gradients, head, Adam) come from FP32 sums of exact products: relative L2
1e-4.  The whole U-Net stores every activation and activation gradient in
BF16.  Its weight gradients are sums over voxels of (gradient x activation);
for a random gradient the sum is incoherent, and the few leaky-ReLU masks that
a rounding-level change of the activations flips move it by about the square
root of their fraction (several percent, measured in FP64 with emulated
rounding).  The network test therefore uses coherent losses: with
dv = v (the gradient of |v|^2 / 2) the emulated rounding moves the weight
gradients by < 1.2e-2 and the output by < 1.2e-2 (slope 0.1), and with a
linear network (slope 1) any dv gives < 1e-2.  Tolerances: output and
gradients relative L2 5e-2.
"""
import numpy as np
import pytest

import __graft_entry__ as entry
from oracle import net as onet

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    entry.build()
    from paper_2209_08189_gb300 import net
    return torch, net


def bf16(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda().to(torch.bfloat16)


def f64(t):
    return t.detach().float().cpu().numpy().astype(np.float64)


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def close_bf16(got, ref):
    tol = 2.0 ** -8 * np.abs(ref) + 1e-3 * np.sqrt(np.mean(ref ** 2))
    return float(np.max(np.abs(got - ref) - tol))


def stream(torch):
    return torch.cuda.current_stream().cuda_stream


CONV_CASES = [
    # (B, D, H, W, Cin, Cout, x_extra, y_extra): extra channels make the slices strided
    (2, 8, 8, 16, 32, 48, 0, 0),
    (1, 4, 4, 4, 16, 16, 16, 8),
    (1, 16, 8, 32, 192, 64, 0, 16),
    (3, 8, 4, 8, 48, 96, 8, 0),
    (1, 8, 8, 8, 128, 128, 0, 0),
    (1, 4, 8, 16, 96, 192, 0, 0),
    # H a multiple of 16 and W of 8: the tcgen05 kernel (TMEM accumulators)
    (1, 4, 16, 8, 16, 16, 0, 0),
    (2, 4, 16, 16, 32, 48, 16, 8),
    (1, 4, 32, 16, 192, 64, 0, 0),
    (1, 4, 16, 8, 96, 192, 0, 0),
    (1, 8, 16, 32, 128, 128, 0, 0),
]


@pytest.mark.parametrize("case", CONV_CASES)
def test_conv3d_forward_and_input_gradient(env, case):
    torch, net = env
    B, D, H, W, ci, co, xe, ye = case
    r = np.random.default_rng(sum(case))
    xbuf = bf16(torch, r.standard_normal((B, D, H, W, ci + xe)))
    w = bf16(torch, r.standard_normal((co, 27, ci)) / np.sqrt(27 * ci))
    bias = torch.from_numpy(r.standard_normal(co).astype(np.float32)).cuda()
    ybuf = torch.zeros((B, D, H, W, co + ye), dtype=torch.bfloat16, device="cuda")
    x = net.Act(xbuf, xe, ci)
    y = net.Act(ybuf, ye, co)
    net.conv3d(x, w, bias, y, 0.1, 1, stream(torch))
    torch.cuda.synchronize()
    xin = f64(xbuf)[..., xe:]
    ref = onet.conv3d(xin, f64(w), f64(bias), act=True, slope=0.1)
    got = f64(ybuf)[..., ye:]
    assert close_bf16(got, ref) <= 0
    if ye:
        assert float(ybuf[..., :ye].abs().max()) == 0.0  # untouched channels
    # input gradient through the flipped weights
    if ci in (16, 32, 48, 64, 96, 128, 192):
        dy = bf16(torch, r.standard_normal((B, D, H, W, co)))
        wf = torch.empty((ci, 27, co), dtype=torch.bfloat16, device="cuda")
        net.conv3d_flip(w, co, ci, wf, stream(torch))
        dx = torch.empty((B, D, H, W, ci), dtype=torch.bfloat16, device="cuda")
        net.conv3d(net.Act(dy, 0, co), wf, None, net.Act(dx, 0, ci), 0.0, 0, stream(torch))
        torch.cuda.synchronize()
        assert close_bf16(f64(dx), onet.conv3d_input_grad(f64(dy), f64(w))) <= 0
    assert net.device_errors() == 0


@pytest.mark.parametrize("tiling", [(1, 1), (2, 2), (4, 1), (4, 2)])
def test_conv3d_tcgen05_tilings(env, tiling):
    """Every forced brick depth / staging of the tcgen05 kernel against the oracle
    (several channel slices, so the two-stage pipeline turns over)."""
    torch, net = env
    B, D, H, W, ci, co = 2, 4, 16, 16, 48, 48
    r = np.random.default_rng(sum(tiling))
    xbuf = bf16(torch, r.standard_normal((B, D, H, W, ci)))
    w = bf16(torch, r.standard_normal((co, 27, ci)) / np.sqrt(27 * ci))
    bias = torch.from_numpy(r.standard_normal(co).astype(np.float32)).cuda()
    y = torch.zeros((B, D, H, W, co), dtype=torch.bfloat16, device="cuda")
    net.set_conv_tiling(*tiling)
    try:
        net.conv3d(net.Act(xbuf, 0, ci), w, bias, net.Act(y, 0, co), 0.1, 1, stream(torch))
        torch.cuda.synchronize()
    finally:
        net.set_conv_tiling(0, 0)
    ref = onet.conv3d(f64(xbuf), f64(w), f64(bias), act=True, slope=0.1)
    assert close_bf16(f64(y), ref) <= 0
    assert net.device_errors() == 0


@pytest.mark.parametrize("case", CONV_CASES)
def test_conv3d_weight_gradient(env, case):
    torch, net = env
    B, D, H, W, ci, co, xe, ye = case
    r = np.random.default_rng(100 + sum(case))
    xbuf = bf16(torch, r.standard_normal((B, D, H, W, ci + xe)))
    dybuf = bf16(torch, r.standard_normal((B, D, H, W, co + ye)))
    x = net.Act(xbuf, xe, ci)
    dy = net.Act(dybuf, ye, co)
    chunks = net.wgrad_chunks(ci, co, (B, D, H, W))
    part = torch.empty(chunks * co * 27 * ci, device="cuda")
    partb = torch.empty(chunks * co, device="cuda")
    dw = torch.empty((co, 27, ci), device="cuda")
    db = torch.empty(co, device="cuda")
    net.conv3d_wgrad(x, dy, chunks, part, partb, dw, db, stream(torch))
    torch.cuda.synchronize()
    rw, rb = onet.conv3d_weight_grad(f64(xbuf)[..., xe:], f64(dybuf)[..., ye:])
    assert rel_l2(f64(dw), rw) < 1e-4
    assert rel_l2(f64(db), rb) < 1e-4
    # deterministic: a second call gives the same bits
    dw2 = torch.empty_like(dw)
    net.conv3d_wgrad(x, dy, chunks, part, partb, dw2, None, stream(torch))
    torch.cuda.synchronize()
    assert torch.equal(dw, dw2)


@pytest.mark.parametrize("co", [144, 32, 16])
@pytest.mark.parametrize("nc", [16, 32, 48, 64])
def test_conv3d_weight_gradient_tcgen05_tilings(env, nc, co):
    """Every input-channel block of the tcgen05 weight gradient against the
    oracle, for output channels as plain MMA rows (144: two blocks, 128 + 16,
    padded TMEM lanes) and as stacked depth-shifted rows (32: 96 of 128
    lanes; 16: 48 of 64), several tap groups where TMEM cannot hold all
    taps, and several bricks per CTA so that both smem stages turn over."""
    torch, net = env
    B, D, H, W, ci = 1, 16, 16, 16, 192
    r = np.random.default_rng(nc + co)
    xbuf = bf16(torch, r.standard_normal((B, D, H, W, ci)))
    dybuf = bf16(torch, r.standard_normal((B, D, H, W, co)))
    net.set_wgrad_tiling(nc)
    try:
        chunks = net.wgrad_chunks(ci, co, (B, D, H, W))
        part = torch.empty(chunks * co * 27 * ci, device="cuda")
        partb = torch.empty(chunks * co, device="cuda")
        dw = torch.empty((co, 27, ci), device="cuda")
        db = torch.empty(co, device="cuda")
        net.conv3d_wgrad(net.Act(xbuf, 0, ci), net.Act(dybuf, 0, co), chunks, part, partb, dw, db, stream(torch))
        torch.cuda.synchronize()
    finally:
        net.set_wgrad_tiling(0)
    rw, rb = onet.conv3d_weight_grad(f64(xbuf), f64(dybuf))
    assert rel_l2(f64(dw), rw) < 1e-4
    assert rel_l2(f64(db), rb) < 1e-4
    assert net.device_errors() == 0


def test_tcgen05_wait_give_up_is_counted_and_returns_cleanly(env):
    """Failure detection without a GPU fault: with the stall hook every CTA of
    the tcgen05 convolution and weight gradient first waits (bounded, a small
    runtime-set number of polls) on a completion phase that nothing signals,
    before any MMA is issued.  The wait runs out, each CTA counts one give-up,
    drains (nothing outstanding), releases its tensor memory and returns; the
    next launches without the hook are correct and count nothing."""
    torch, net = env
    B, D, H, W, ci, co = 1, 4, 16, 8, 16, 16
    r = np.random.default_rng(5)
    xbuf = bf16(torch, r.standard_normal((B, D, H, W, ci)))
    w = bf16(torch, r.standard_normal((co, 27, ci)) / np.sqrt(27 * ci))
    dybuf = bf16(torch, r.standard_normal((B, D, H, W, co)))
    x, dy = net.Act(xbuf, 0, ci), net.Act(dybuf, 0, co)
    chunks = net.wgrad_chunks(ci, co, (B, D, H, W))
    part = torch.empty(chunks * co * 27 * ci, device="cuda")
    partb = torch.empty(chunks * co, device="cuda")
    dw = torch.empty((co, 27, ci), device="cuda")
    db = torch.empty(co, device="cuda")
    y = torch.zeros((B, D, H, W, co), dtype=torch.bfloat16, device="cuda")
    assert net.device_errors() == 0
    try:
        assert net.set_wait_test(2000, True) == 0
        net.conv3d(x, w, None, net.Act(y, 0, co), 0.1, 1, stream(torch))
        torch.cuda.synchronize()
        n_conv = net.device_errors()
        net.conv3d_wgrad(x, dy, chunks, part, partb, dw, db, stream(torch))
        torch.cuda.synchronize()
        n_wgrad = net.device_errors()
    finally:
        kept = net.set_wait_test(0, False)
    assert n_conv >= 1 and n_wgrad >= 1
    assert kept == 0  # every CTA that gave up released its tensor memory
    net.conv3d(x, w, None, net.Act(y, 0, co), 0.1, 1, stream(torch))
    net.conv3d_wgrad(x, dy, chunks, part, partb, dw, db, stream(torch))
    torch.cuda.synchronize()
    assert close_bf16(f64(y), onet.conv3d(f64(xbuf), f64(w), None, act=True, slope=0.1)) <= 0
    rw, rb = onet.conv3d_weight_grad(f64(xbuf), f64(dybuf))
    assert rel_l2(f64(dw), rw) < 1e-4 and rel_l2(f64(db), rb) < 1e-4
    assert net.device_errors() == 0


def test_unet_weight_file_round_trip(env, tmp_path):
    """save_weights / from_file: the reloaded network gives the same output
    bits (conv weights are stored as the BF16 values the forward pass uses)."""
    torch, net = env
    st = stream(torch)
    r = np.random.default_rng(8)
    m0 = torch.from_numpy(r.random((32, 32, 32), dtype=np.float32)).cuda()
    m1 = torch.from_numpy(r.random((32, 32, 32), dtype=np.float32)).cuda()
    for pc_head in (False, True):  # velocity only; velocity + preconditioner-weight logit
        u = net.UNet(seed=3, stream=st, pc_head=pc_head)
        a = u.forward(m0[None], m1[None]).clone()
        path = str(tmp_path / ("w%d.npz" % pc_head))
        u.save_weights(path, meta={"n_net": 32})
        w = net.UNet.from_file(path, stream=st)
        b = w.forward(m0[None], m1[None])
        torch.cuda.synchronize()
        assert w.meta["n_net"] == 32 and w.num_params() == u.num_params() and w.pc_head == pc_head
        assert torch.equal(a, b)
        if pc_head:
            assert torch.equal(u.pc_logit(), w.pc_logit())


def test_pool_up_leaky_pack_head_adam(env):
    torch, net = env
    r = np.random.default_rng(7)
    B, D, H, W, C = 2, 8, 8, 16, 32
    st = stream(torch)
    fine = bf16(torch, r.standard_normal((B, D, H, W, C + 16)))
    coarse = torch.empty((B, D // 2, H // 2, W // 2, C), dtype=torch.bfloat16, device="cuda")
    net.pool2(net.Act(fine, 16, C), net.Act(coarse, 0, C), st)
    up = torch.empty((B, D, H, W, C), dtype=torch.bfloat16, device="cuda")
    net.up2(net.Act(coarse, 0, C), net.Act(up, 0, C), st)
    add = bf16(torch, r.standard_normal((B, D, H, W, C)))
    dfine = torch.empty((B, D, H, W, C), dtype=torch.bfloat16, device="cuda")
    net.pool2_bwd(net.Act(coarse, 0, C), net.Act(add, 0, C), net.Act(dfine, 0, C), st)
    dco = torch.empty((B, D // 2, H // 2, W // 2, C), dtype=torch.bfloat16, device="cuda")
    net.up2_bwd(net.Act(up, 0, C), net.Act(dco, 0, C), st)
    y = bf16(torch, r.standard_normal((B, D, H, W, C)))
    dy = bf16(torch, r.standard_normal((B, D, H, W, C)))
    dp = torch.empty_like(dy)
    net.leaky_bwd(net.Act(dy, 0, C), net.Act(y, 0, C), 0.1, net.Act(dp, 0, C), st)
    torch.cuda.synchronize()
    pc = onet.pool2(f64(fine)[..., 16:])
    assert close_bf16(f64(coarse), pc) <= 0
    assert np.array_equal(f64(up), onet.up2(f64(coarse)))
    assert close_bf16(f64(dfine), onet.pool2_adj(f64(coarse)) + f64(add)) <= 0
    assert close_bf16(f64(dco), onet.up2_adj(f64(up))) <= 0
    assert close_bf16(f64(dp), onet.leaky_grad(f64(dy), f64(y), 0.1)) <= 0
    # pack + head + head backward
    L = net.lib()
    m0 = torch.from_numpy(r.random((B, D, H, W)).astype(np.float32)).cuda()
    m1 = torch.from_numpy(r.random((B, D, H, W)).astype(np.float32)).cuda()
    xb = torch.empty((B, D, H, W, 16), dtype=torch.bfloat16, device="cuda")
    net._check(L.claire_net_pack(m0.data_ptr(), m1.data_ptr(), 2.0, -1.0, m0.numel(), xb.data_ptr(), 16, st), "pack")
    torch.cuda.synchronize()
    rx = onet.pack(m0.cpu().numpy(), m1.cpu().numpy(), 2.0, -1.0, 16)
    assert close_bf16(f64(xb), rx) <= 0
    for nout in (3, 4):  # velocity head; velocity + preconditioner-weight logit
        wh = torch.from_numpy(r.standard_normal((nout, 16)).astype(np.float32)).cuda()
        bh = torch.from_numpy(r.standard_normal(nout).astype(np.float32)).cuda()
        v = torch.empty((B, nout, D, H, W), device="cuda")
        x = net.Act(xb, 0, 16)
        net._check(L.claire_net_head(x.ptr, 16, 16, nout, wh.data_ptr(), bh.data_ptr(), 0.5, v.data_ptr(), x.v4(),
                                     st), "head")
        dv = torch.from_numpy(r.standard_normal((B, nout, D, H, W)).astype(np.float32)).cuda()
        import ctypes
        nb = ctypes.c_int()
        net._check(L.claire_net_head_bwd_blocks(x.v4(), ctypes.byref(nb)), "blocks")
        nr = nout * 16 + nout
        part = torch.empty(nb.value * nr, device="cuda")
        dwb = torch.empty(nr, device="cuda")
        dx = torch.empty((B, D, H, W, 16), dtype=torch.bfloat16, device="cuda")
        net._check(L.claire_net_head_bwd(x.ptr, 16, 16, nout, wh.data_ptr(), 0.5, dv.data_ptr(), dx.data_ptr(), 16,
                                         x.v4(), nb.value, part.data_ptr(), dwb.data_ptr(), st), "head_bwd")
        torch.cuda.synchronize()
        xr = f64(xb)
        assert rel_l2(f64(v), onet.head(xr, f64(wh), f64(bh), 0.5)) < 1e-5
        rdx, rdw, rdb = onet.head_grad(xr, f64(wh), 0.5, f64(dv))
        assert close_bf16(f64(dx), rdx) <= 0
        assert rel_l2(f64(dwb)[:nout * 16].reshape(nout, 16), rdw) < 1e-4
        assert rel_l2(f64(dwb)[nout * 16:], rdb) < 1e-4
    # Adam, three steps
    n = 1000
    w = torch.from_numpy(r.standard_normal(n).astype(np.float32)).cuda()
    m = torch.zeros(n, device="cuda")
    s = torch.zeros(n, device="cuda")
    wb = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    rw, rm, rs = f64(w), np.zeros(n), np.zeros(n)
    for k in range(1, 4):
        g = torch.from_numpy(r.standard_normal(n).astype(np.float32)).cuda()
        net.adam(w, g, m, s, 1e-2, 0.9, 0.999, 1e-8, k, 0.5, wb, st)
        rw, rm, rs = onet.adam(rw, 0.5 * f64(g), rm, rs, 1e-2, 0.9, 0.999, 1e-8, k)
    torch.cuda.synchronize()
    assert rel_l2(f64(w), rw) < 1e-6
    assert np.array_equal(f64(wb), f64(w.to(torch.bfloat16)))


@pytest.mark.parametrize("slope,coherent", [(0.1, True), (1.0, False)])
def test_unet_forward_backward_matches_oracle(env, slope, coherent):
    torch, net = env
    chans = (16, 32, 64, 128)
    u = net.UNet(chans=chans, cin=16, slope=slope, vscale=0.5, seed=3, stream=stream(torch))
    r = np.random.default_rng(9)
    # non-zero head and biases so that every path carries signal
    for name, P in u.p.items():
        P["b"].copy_(torch.from_numpy(0.1 * r.standard_normal(P["b"].shape).astype(np.float32)))
    u.p["head"]["w"].mul_(10.0)
    u._sync_weights()
    B, n = 1, 32
    m0 = torch.from_numpy(r.random((B, n, n, n)).astype(np.float32)).cuda()
    m1 = torch.from_numpy(r.random((B, n, n, n)).astype(np.float32)).cuda()
    v = u.forward(m0, m1)
    if coherent:
        dv = v.clone()
    else:
        dv = torch.from_numpy(r.standard_normal((B, 3, n, n, n)).astype(np.float32)).cuda()
    u.backward(dv)
    torch.cuda.synchronize()
    params = {}
    for name, P in u.p.items():
        w = f64(P["wb"]) if "wb" in P else f64(P["w"])
        params[name] = (w, f64(P["b"]))
    x = onet.pack(m0.cpu().numpy(), m1.cpu().numpy(), 1.0, 1.0, 16)
    x = f64(torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16))
    rv, cache = onet.unet_forward(params, x, chans, slope=slope, vscale=0.5)
    ref_dv = rv if coherent else f64(dv)
    grads = onet.unet_backward(params, cache, ref_dv, chans, slope=slope, vscale=0.5)
    ev = rel_l2(f64(v), rv)
    errs = {name: rel_l2(f64(u.p[name]["gw"]), grads[name][0]) for name in u.p}
    errb = {name: rel_l2(f64(u.p[name]["gb"]), grads[name][1]) for name in u.p}
    print("U-Net slope %g: output rel L2 %.2e; worst weight-gradient %.2e (%s), worst bias-gradient %.2e"
          % (slope, ev, max(errs.values()), max(errs, key=errs.get), max(errb.values())))
    assert ev < 5e-2
    for name in errs:
        assert errs[name] < 5e-2, (name, errs[name])
        assert errb[name] < 5e-2, (name, errb[name])


def test_invalid_shapes_are_rejected(env):
    torch, net = env
    x = torch.zeros((1, 8, 8, 8, 16), dtype=torch.bfloat16, device="cuda")
    w = torch.zeros((80, 27, 16), dtype=torch.bfloat16, device="cuda")
    y = torch.zeros((1, 8, 8, 8, 80), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(net.NetError):
        net.conv3d(net.Act(x, 0, 16), w, None, net.Act(y, 0, 80), 0.1, 1, stream(torch))
    y2 = torch.zeros((1, 8, 8, 6, 16), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(net.NetError):
        net.conv3d(net.Act(x, 0, 16), w[:16], None, net.Act(y2, 0, 16), 0.1, 1, stream(torch))
