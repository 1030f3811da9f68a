"""Training and inference of the learned warm start (network in net.py).

Training pairs are generated by the method itself: a template (the label or
blob families of ``synth``) is advected by a random band-limited velocity v*
with ``claire_transport`` to give the reference image.  The loss of a
predicted velocity v is

    L = wv/2 |v - v*|^2 / (3 N sigma^2) + wm/2 |T(v) m0 - m1|^2 / |m0 - m1|^2,

the second term differentiated by the hand-written SL adjoint
(``claire_transport_vjp``).  Inference on a finer grid samples the images to
the training grid (nearest neighbour), runs the network there and carries
the velocity back by spectral prolongation (``claire_resample``), the
grid-transfer scheme of the paper's downsampled registrations (Sec. 4).

Orchestration only: every numerical step runs in libclaire kernels; torch
provides device memory.  Pair pools are drawn on the host once (numpy, the
``synth`` recipes) and kept on the device.
"""
from __future__ import annotations

import ctypes
import time

import numpy as np

from . import claire, synth
from .net import UNet, lib as _netlib, _check


class PairSource:
    """Pools of templates, velocities and noise fields on the device; a batch
    combines random members and advects on the GPU."""

    def __init__(self, n, n_templates=24, n_velocities=48, kmax=(4, 8), vmax=(0.3, 1.2), noise=0.02, nt=4,
                 seed=0, families=("label", "blob"), n_noise=8):
        import torch
        self.torch = torch
        self.n = int(n)
        self.nt = int(nt)
        grid = (self.n,) * 3
        rng = np.random.default_rng(seed)
        dev = torch.device("cuda", torch.cuda.current_device())
        T = []
        for i in range(n_templates):
            fam = families[i % len(families)]
            s = int(rng.integers(1 << 30))
            if fam == "label":
                T.append(synth.label_template(grid, seed=s))
            else:
                T.append(synth.blob_template(grid, seed=s, nblobs=int(rng.integers(4, 12)),
                                             sigma=float(rng.uniform(0.25, 0.5))))
        V = []
        for i in range(n_velocities):
            V.append(synth.bandlimited_velocity(grid, seed=int(rng.integers(1 << 30)),
                                                kmax=int(rng.integers(kmax[0], kmax[1] + 1)),
                                                vmax=float(rng.uniform(*vmax))))
        f32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
        self.T = f32(np.stack(T))
        self.V = f32(np.stack(V))
        self.negnoise = f32(np.stack([-noise * rng.standard_normal(grid) for _ in range(n_noise)])) \
            if noise > 0 else None
        self.sigma2 = float(np.mean(np.stack(V) ** 2))
        self.ctx = claire.Context(grid, 1e-2, nt, stream=torch.cuda.current_stream().cuda_stream)
        self.rng = np.random.default_rng(seed + 1)
        self._b = None

    def batch(self, B):
        """Returns (m0, m1, vstar): [B, n, n, n], [B, n, n, n], [B, 3, n, n, n] (reused buffers)."""
        torch, n = self.torch, self.n
        if self._b is None or self._b[0].shape[0] != B:
            dev = self.T.device
            self._b = (torch.empty((B, n, n, n), device=dev), torch.empty((B, n, n, n), device=dev),
                       torch.empty((B, 3, n, n, n), device=dev))
        m0, m1, vs = self._b
        st = torch.cuda.current_stream().cuda_stream
        L = _netlib()
        N = n ** 3
        for b in range(B):
            ti = int(self.rng.integers(len(self.T)))
            vi = int(self.rng.integers(len(self.V)))
            vs[b].copy_(self.V[vi])
            self.ctx.transport(vs[b], self.T[ti], m1[b], claire.TRANSPORT_FWD)
            m0[b].copy_(self.T[ti])
            if self.negnoise is not None:
                a = int(self.rng.integers(len(self.negnoise)))
                c = (a + 1 + int(self.rng.integers(len(self.negnoise) - 1))) % len(self.negnoise)
                _check(L.claire_net_residual(m0[b].data_ptr(), self.negnoise[a].data_ptr(), N, m0[b].data_ptr(),
                                             None, st), "residual")
                _check(L.claire_net_residual(m1[b].data_ptr(), self.negnoise[c].data_ptr(), N, m1[b].data_ptr(),
                                             None, st), "residual")
        return m0, m1, vs


def _pc_probes(n, count, seed):
    """Band-limited probe fields of the preconditioner-weight fit (|k| <= 6)."""
    return [synth.mode_velocity((n,) * 3, seed=seed + i, nmodes=8, kmax=6, vmax=0.3) for i in range(count)]


PC_SCALES = (1.0, 1.5, 2.0, 3.0, 4.0, 6.0)
PC_SCALE_FRACTION = 0.96


def pc_scale_target(ctx, v, g, z, hz, consts):
    """Target weight of the "scale" mode: with the two-level context ctx
    linearised at v (the network's prediction), the smallest constant weight
    c of PC_SCALES whose first preconditioned step z = P_c^-1 g achieves at
    least PC_SCALE_FRACTION of the best quadratic-model decrease
    q(c) = (g . z)^2 / (z . H z) over the list (larger weights make the coarse
    inner solves harder for a smaller gain).  consts: constant coarse fields,
    one per scale.  Returns (c, [q(c)])."""
    N3 = g.numel()
    ctx.gradient(v, g)
    qs = []
    for w in consts:
        ctx.set_pc_weight(w)
        ctx.precond(g, z)
        ctx.hessian_matvec(z, hz)
        gz = claire.claire_dot(ctx.handle, g, z, N3)
        zhz = claire.claire_dot(ctx.handle, z, hz, N3)
        qs.append(gz * gz / zhz if zhz > 0 else 0.0)
    ctx.set_pc_weight(None)
    best = max(qs)
    for c, q in zip(PC_SCALES, qs):
        if q >= PC_SCALE_FRACTION * best:
            return c, qs
    return PC_SCALES[-1], qs


def train(net, src, steps, batch=4, lr=1e-3, wv=1.0, wm=1.0, lr_final=None, log_every=0, clip=None, wpc=0.0,
          pc_probes=2, pc_pool=8, pc_target="scale", pc_grid=None):
    """Adam on the loss above; returns a list of (step, Lv, Lm_rel, seconds, Lpc).

    With a preconditioner head (net.pc_head) and wpc > 0, the loss adds wpc
    times the loss of the coarse preconditioner weight w = softplus(o)
    (claire_net_pcw_loss) against a per-sample target:
    * pc_target "scale": the constant of pc_scale_target at the network's own
      prediction of the pair (a spatially constant target), on the pair and
      the prediction carried spectrally to pc_grid^3 (the grid of the
      registrations the weight is meant for; default the training grid);
    * pc_target "fit": the least-squares fit of the weighted zero-velocity
      data term to the true Gauss-Newton data term at the pair's v*, from
      pc_probes probe fields per sample and step (drawn in turn from a pool of
      pc_pool), the mean state gradient (claire_mean_state_gradient), the
      matvec and S p."""
    torch = src.torch
    st = torch.cuda.current_stream().cuda_stream
    L = _netlib()
    n = src.n
    N = n ** 3
    dev = src.T.device
    use_pc = bool(getattr(net, "pc_head", False)) and wpc > 0
    sums = torch.zeros(3 * batch, dtype=torch.float64, device=dev)
    mt = torch.empty((n, n, n), device=dev)
    r = torch.empty((n, n, n), device=dev)
    gv = torch.empty((3, n, n, n), device=dev)
    if use_pc:
        probes = [torch.from_numpy(np.ascontiguousarray(q, dtype=np.float32)).to(dev)
                  for q in _pc_probes(n, pc_pool, 7000)]
        gbar = torch.empty((3, n, n, n), device=dev)
        gtmp = torch.empty((3, n, n, n), device=dev)
        hp = torch.empty((3, n, n, n), device=dev)
        sp = torch.empty((3, n, n, n), device=dev)
        num = torch.empty((batch, n, n, n), device=dev)
        den = torch.empty((batch, n, n, n), device=dev)
        psums = torch.zeros(2 * batch, dtype=torch.float64, device=dev)
        grid3 = (ctypes.c_int * 3)(n, n, n)
        if pc_target == "scale":
            ng = int(pc_grid or n)
            G = (ng,) * 3
            pcctx = claire.Context(G, 1e-2, src.nt, stream=st, precond=claire.PRECOND_TWO_LEVEL)
            consts = [torch.full((ng // 2,) * 3, c, device=dev) for c in PC_SCALES]
            pz = torch.empty((3,) + G, device=dev)
            if ng != n:  # the target is taken on the pair carried to the registration grid
                pg = torch.empty((3,) + G, device=dev)
                phz = torch.empty((3,) + G, device=dev)
                pm0 = torch.empty(G, device=dev)
                pm1 = torch.empty(G, device=dev)
                pv = torch.empty((3,) + G, device=dev)
        elif pc_target != "fit":
            raise ValueError("pc_target: 'scale' or 'fit'")
    hist = []
    t0 = time.perf_counter()
    a = wv / (3.0 * N * src.sigma2)
    kp = 0
    for it in range(steps):
        frac = it / max(1, steps - 1)
        lr_it = lr if lr_final is None else lr * (lr_final / lr) ** frac
        m0, m1, vs = src.batch(batch)
        v = net.forward(m0, m1)
        dv = net.output_grad()
        sums.zero_()
        if use_pc:
            # statistics at v* of each pair, then the weight loss on channel 3
            num.zero_()
            den.zero_()
            psums.zero_()
            o = net.pc_logit()
            for b in range(batch):
                if pc_target == "scale":
                    if ng == n:
                        pcctx.set_images(m0[b], m1[b])
                        c, _ = pc_scale_target(pcctx, v[b], gtmp, pz, hp, consts)
                    else:
                        g3n = (n,) * 3
                        claire.claire_resample(m0[b], g3n, pm0, G, 1, claire.RESAMPLE_SPECTRAL, st)
                        claire.claire_resample(m1[b], g3n, pm1, G, 1, claire.RESAMPLE_SPECTRAL, st)
                        claire.claire_resample(v[b], g3n, pv, G, 3, claire.RESAMPLE_SPECTRAL, st)
                        pcctx.set_images(pm0, pm1)
                        c, _ = pc_scale_target(pcctx, pv, pg, pz, phz, consts)
                    num[b].fill_(c)
                    den[b].fill_(1.0)
                    _check(L.claire_net_pcw_loss(o[b].data_ptr(), num[b].data_ptr(), den[b].data_ptr(), grid3,
                                                 wpc, dv[b, 3].data_ptr(), psums[2 * b:].data_ptr(), st),
                           "pcw_loss")
                    continue
                src.ctx.set_images(m0[b], m1[b])
                src.ctx.gradient(vs[b], gtmp)
                src.ctx.mean_state_gradient(gbar)
                for _ in range(pc_probes):
                    q = probes[kp % len(probes)]
                    kp += 1
                    src.ctx.hessian_matvec(q, hp)
                    src.ctx.spectral(q, sp, claire.SPECTRAL_REG)
                    _check(L.claire_net_pcw_stats(gbar.data_ptr(), q.data_ptr(), hp.data_ptr(), sp.data_ptr(), N,
                                                  num[b].data_ptr(), den[b].data_ptr(), st), "pcw_stats")
                _check(L.claire_net_pcw_loss(o[b].data_ptr(), num[b].data_ptr(), den[b].data_ptr(), grid3,
                                             wpc, dv[b, 3].data_ptr(), psums[2 * b:].data_ptr(), st),
                       "pcw_loss")
        if wm > 0:
            for b in range(batch):
                _check(L.claire_net_residual(m0[b].data_ptr(), m1[b].data_ptr(), N, None,
                                             sums[3 * b + 2:].data_ptr(), st), "residual")
            r0 = sums[2::3].cpu().numpy()
        for b in range(batch):
            if wm > 0:
                src.ctx.transport(v[b], m0[b], mt, claire.TRANSPORT_FWD)
                _check(L.claire_net_residual(mt.data_ptr(), m1[b].data_ptr(), N, r.data_ptr(),
                                             sums[3 * b + 1:].data_ptr(), st), "residual")
                src.ctx.transport_vjp(v[b], m0[b], r, None, gv)
                bcoef = wm / max(float(r0[b]), 1e-30)
                _check(L.claire_net_vel_loss(v[b].data_ptr(), vs[b].data_ptr(), gv.data_ptr(), a, bcoef, 3 * N,
                                             dv[b].data_ptr(), sums[3 * b:].data_ptr(), st), "vel_loss")
            else:
                _check(L.claire_net_vel_loss(v[b].data_ptr(), vs[b].data_ptr(), None, a, 0.0, 3 * N,
                                             dv[b].data_ptr(), sums[3 * b:].data_ptr(), st), "vel_loss")
        net.backward(dv)
        net.step(lr_it / batch)
        if log_every and (it % log_every == 0 or it == steps - 1):
            s = sums.cpu().numpy()
            Lv = 0.5 * a * float(np.sum(s[0::3])) / batch
            Lm = float(np.mean(s[1::3] / np.maximum(s[2::3], 1e-30))) if wm > 0 else float("nan")
            Lpc = float(np.mean(psums.cpu().numpy()[1::2])) if use_pc else float("nan")
            hist.append((it, Lv, Lm, time.perf_counter() - t0, Lpc))
    torch.cuda.synchronize()
    if use_pc and pc_target == "scale":
        pcctx.close()
    return hist


class WarmStart:
    """Predicts an initial velocity for images on any grid whose extents are
    multiples of the network grid's (power-of-two extents >= 16 per axis)."""

    def __init__(self, net, n_net):
        self.net = net
        self.n_net = int(n_net)

    def predict(self, m0, m1, v_out):
        """m0, m1: FP32 CUDA [D, H, W]; v_out: FP32 CUDA [3, D, H, W]."""
        torch = self.net.torch
        grid = tuple(m0.shape)
        g = (self.n_net,) * 3
        st = torch.cuda.current_stream().cuda_stream
        if grid == g:
            v = self.net.forward(m0, m1)
            v_out.copy_(v[0])
            return v_out
        a = torch.empty((2,) + g, device=m0.device)
        claire.claire_resample(m0, grid, a[0], g, 1, claire.RESAMPLE_NEAREST, st)
        claire.claire_resample(m1, grid, a[1], g, 1, claire.RESAMPLE_NEAREST, st)
        v = self.net.forward(a[0], a[1])
        claire.claire_resample(v[0], g, v_out, grid, 3, claire.RESAMPLE_SPECTRAL, st)
        return v_out

    def pc_weight(self, w_out):
        """Coarse preconditioner weight from the last predict() (networks with
        a preconditioner head): the fourth output channel, the logit o, is
        carried to w_out's grid (the two-level preconditioner's coarse grid) by
        spectral resampling and mapped to w = softplus(o) > 0 there; w_out:
        FP32 CUDA [Nc1, Nc2, Nc3]."""
        torch = self.net.torch
        o = self.net.pc_logit()[0]
        g = (self.n_net,) * 3
        wgrid = tuple(w_out.shape)
        st = torch.cuda.current_stream().cuda_stream
        src = o
        if wgrid != g:
            src = torch.empty(wgrid, device=o.device)
            claire.claire_resample(o, g, src, wgrid, 1, claire.RESAMPLE_SPECTRAL, st)
        _check(_netlib().claire_net_pcw_weight(src.data_ptr(), w_out.data_ptr(), w_out.numel(), st), "pcw_weight")
        return w_out
