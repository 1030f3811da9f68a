"""Learned warm start: a 3D U-Net over periodic volumes that maps an image
pair (m0, m1) to an initial velocity for the Gauss-Newton-Krylov solver.

Binding of the network kernels (C ABI in include/claire_net.h) and the
network assembled from them.  Argument marshalling and buffer bookkeeping
only: every layer, its gradients, the loss terms and the optimiser step run
in the library's CUDA kernels; torch supplies device memory.  There is no
fallback: without the library or a CUDA device the calls fail.

Architecture (4 levels, channels 16-32-64-128, ~1.46M parameters): per
level two 3x3x3 convolutions with leaky ReLU; 2x2x2 average pooling down,
nearest 2x upsampling up, skip connections by channel concatenation; a
1x1x1 head to the three velocity components (physical units) and, with
pc_head, a fourth channel: the logit o of the coarse preconditioner weight
w = softplus(o) (the correction of the two-level preconditioner).  Periodic
padding matches the registration domain.  Activations and conv weights are
BF16 with FP32 accumulation; FP32 master weights and Adam moments.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import claire as _c

_vp = ctypes.c_void_p
_I4 = ctypes.c_int * 4
_i, _f, _sz = ctypes.c_int, ctypes.c_float, ctypes.c_size_t
_ip = ctypes.POINTER(ctypes.c_int)

# name -> argtypes (restype claire_status unless listed in _RESTYPE)
_SIGS = {
    "claire_net_conv3d": [_vp, _i, _i, _vp, _vp, _f, _i, _vp, _i, _i, _ip, _vp],
    "claire_net_conv3d_flip": [_vp, _i, _i, _vp, _vp],
    "claire_net_conv3d_wgrad_chunks": [_i, _i, _ip, _ip],
    "claire_net_conv3d_wgrad": [_vp, _i, _i, _vp, _i, _i, _ip, _i, _vp, _vp, _vp, _vp, _vp],
    "claire_net_pool2": [_vp, _i, _i, _vp, _i, _ip, _vp],
    "claire_net_pool2_bwd": [_vp, _i, _vp, _i, _i, _vp, _i, _ip, _vp],
    "claire_net_up2": [_vp, _i, _i, _vp, _i, _ip, _vp],
    "claire_net_up2_bwd": [_vp, _i, _i, _vp, _i, _ip, _vp],
    "claire_net_leaky_bwd": [_vp, _i, _vp, _i, _i, _f, _vp, _i, _ip, _vp],
    "claire_net_pack": [_vp, _vp, _f, _f, _sz, _vp, _i, _vp],
    "claire_net_head": [_vp, _i, _i, _i, _vp, _vp, _f, _vp, _ip, _vp],
    "claire_net_head_bwd_blocks": [_ip, _ip],
    "claire_net_head_bwd": [_vp, _i, _i, _i, _vp, _f, _vp, _vp, _i, _ip, _i, _vp, _vp, _vp],
    "claire_net_adam": [_vp, _vp, _vp, _vp, _sz, _f, _f, _f, _f, _i, _f, _vp, _vp],
    "claire_net_vel_loss": [_vp, _vp, _vp, _f, _f, _sz, _vp, _vp, _vp],
    "claire_net_residual": [_vp, _vp, _sz, _vp, _vp, _vp],
    "claire_net_pcw_stats": [_vp, _vp, _vp, _vp, _sz, _vp, _vp, _vp],
    "claire_net_pcw_loss": [_vp, _vp, _vp, _ip, _f, _vp, _vp, _vp],
    "claire_net_pcw_weight": [_vp, _vp, _sz, _vp],
    "claire_net_device_errors": [_ip, _i],
    "claire_net_set_wait_test": [ctypes.c_uint, _i, _ip],
    "claire_net_set_conv_tiling": [_i, _i],
    "claire_net_set_wgrad_tiling": [_i],
    "claire_net_last_error": [],
}
_RESTYPE = {"claire_net_last_error": ctypes.c_char_p}
_bound = False


class NetError(RuntimeError):
    pass


def lib():
    global _bound
    L = _c.lib()
    if not _bound:
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = _RESTYPE.get(name, ctypes.c_int)
        _bound = True
    return L


def _check(status, what):
    if status < 0:
        raise NetError("%s: %s (%s)" % (what, _c.STATUS_NAMES.get(status, status),
                                        lib().claire_net_last_error().decode()))


def device_errors(reset=True):
    """tcgen05 completion waits that gave up (0 in a healthy run)."""
    n = ctypes.c_int()
    _check(lib().claire_net_device_errors(ctypes.byref(n), int(bool(reset))), "device_errors")
    return n.value


def set_wait_test(spin_limit=0, stall=False):
    """Failure-detection hook of the tcgen05 kernels: the bound of every
    mbarrier wait (0 = default) and, with stall, a first wait on a phase that
    nothing signals in every CTA.  Returns the count of CTAs that kept their
    tensor memory after a give-up (0 when every give-up drained)."""
    kept = ctypes.c_int()
    _check(lib().claire_net_set_wait_test(int(spin_limit), int(bool(stall)), ctypes.byref(kept)),
           "set_wait_test")
    return kept.value


def set_conv_tiling(bdc=0, nstage=0):
    """Force the tcgen05 convolution's brick depth / staging (0, 0 = automatic)."""
    _check(lib().claire_net_set_conv_tiling(int(bdc), int(nstage)), "set_conv_tiling")


def set_wgrad_tiling(nc=0):
    """Force the tcgen05 weight gradient's input-channel block (0 = automatic)."""
    _check(lib().claire_net_set_wgrad_tiling(int(nc)), "set_wgrad_tiling")


def _addr(t):
    return None if t is None else t.data_ptr()


class Act:
    """A channel slice [c0, c0 + C) of a channels-last BF16 buffer."""

    def __init__(self, buf, c0, C):
        self.buf, self.c0, self.C = buf, c0, C
        self.stride = buf.shape[-1]
        self.vol = tuple(buf.shape[:4])

    @property
    def ptr(self):
        return self.buf.data_ptr() + 2 * self.c0

    def v4(self):
        return _I4(*self.vol)


# ---- thin wrappers with the C names' meaning --------------------------------

def conv3d(x, w, bias, y, slope, act, stream):
    _check(lib().claire_net_conv3d(x.ptr, x.stride, x.C, w.data_ptr(), _addr(bias), slope, int(act), y.ptr,
                                   y.stride, y.C, y.v4(), stream), "conv3d")


def conv3d_flip(w, cout, cin, wf, stream):
    _check(lib().claire_net_conv3d_flip(w.data_ptr(), cout, cin, wf.data_ptr(), stream), "conv3d_flip")


def wgrad_chunks(cin, cout, vol):
    n = ctypes.c_int()
    _check(lib().claire_net_conv3d_wgrad_chunks(cin, cout, _I4(*vol), ctypes.byref(n)), "wgrad_chunks")
    return n.value


def conv3d_wgrad(x, dy, chunks, part, partb, dw, db, stream):
    _check(lib().claire_net_conv3d_wgrad(x.ptr, x.stride, x.C, dy.ptr, dy.stride, dy.C, dy.v4(), chunks,
                                         part.data_ptr(), partb.data_ptr(), dw.data_ptr(), _addr(db), stream),
           "conv3d_wgrad")


def pool2(x, y, stream):
    _check(lib().claire_net_pool2(x.ptr, x.stride, x.C, y.ptr, y.stride, y.v4(), stream), "pool2")


def pool2_bwd(dy, add, dx, stream):
    _check(lib().claire_net_pool2_bwd(dy.ptr, dy.stride, add.ptr if add else None, add.stride if add else 0,
                                      dy.C, dx.ptr, dx.stride, dy.v4(), stream), "pool2_bwd")


def up2(x, y, stream):
    _check(lib().claire_net_up2(x.ptr, x.stride, x.C, y.ptr, y.stride, x.v4(), stream), "up2")


def up2_bwd(dy, dx, stream):
    _check(lib().claire_net_up2_bwd(dy.ptr, dy.stride, dx.C, dx.ptr, dx.stride, dx.v4(), stream), "up2_bwd")


def leaky_bwd(dy, y, slope, dp, stream):
    _check(lib().claire_net_leaky_bwd(dy.ptr, dy.stride, y.ptr, y.stride, y.C, slope, dp.ptr, dp.stride, y.v4(),
                                      stream), "leaky_bwd")


def adam(w, g, m, s, lr, b1, b2, eps, step, gscale, wb, stream):
    _check(lib().claire_net_adam(w.data_ptr(), g.data_ptr(), m.data_ptr(), s.data_ptr(), w.numel(), lr, b1, b2,
                                 eps, step, gscale, _addr(wb), stream), "adam")


def unet_layers(chans=(16, 32, 64, 128), cin=16):
    """(name, Cin, Cout) of every 3x3x3 convolution, in forward order."""
    L = len(chans)
    out, prev = [], cin
    for l in range(L - 1):
        out += [("enc%da" % l, prev, chans[l]), ("enc%db" % l, chans[l], chans[l])]
        prev = chans[l]
    out += [("bota", prev, chans[-1]), ("botb", chans[-1], chans[-1])]
    for l in range(L - 2, -1, -1):
        out += [("dec%da" % l, chans[l] + chans[l + 1], chans[l]), ("dec%db" % l, chans[l], chans[l])]
    return out


class UNet:
    """The warm-start network on one CUDA device (see the module docstring).

    forward(m0, m1) -> v [B, 3, D, H, W]; backward(dv) accumulates nothing
    (it overwrites the gradients); step(lr) applies Adam.  Input scaling:
    channel 0 = a0 m0, channel 1 = a1 m1; output = vscale * head(...).
    """

    def __init__(self, chans=(16, 32, 64, 128), cin=16, slope=0.1, vscale=1.0, seed=0, stream=None,
                 pc_head=False):
        import torch
        self.torch = torch
        self.chans, self.cin, self.slope, self.vscale = tuple(chans), cin, float(slope), float(vscale)
        self.pc_head = bool(pc_head)
        self.nout = 4 if self.pc_head else 3
        self.stream = stream
        self.dev = torch.device("cuda", torch.cuda.current_device())
        rng = np.random.default_rng(seed)
        self.layers = unet_layers(self.chans, cin)
        self.p = {}
        for name, ci, co in self.layers:
            std = math.sqrt(2.0 / ((1.0 + self.slope ** 2) * 27 * ci))
            w = rng.standard_normal((co, 27, ci)) * std
            self._add(name, w, np.zeros(co))
        c0 = self.chans[0]
        hw = rng.standard_normal((self.nout, c0)) * (0.1 / math.sqrt(c0))
        hb = np.zeros(self.nout)
        if self.pc_head:
            hb[3] = math.log(math.e - 1.0)  # softplus(o) = 1 at start: the paper's preconditioner
        self._add("head", hw, hb, bf16=False)
        self.t = 0
        self._sync_weights()
        self._bufs = {}

    # ---- parameters ----
    def _add(self, name, w, b, bf16=True):
        torch = self.torch
        P = {"w": torch.from_numpy(np.ascontiguousarray(w, dtype=np.float32)).to(self.dev),
             "b": torch.from_numpy(np.ascontiguousarray(b, dtype=np.float32)).to(self.dev)}
        for k in ("w", "b"):
            P["g" + k] = torch.zeros_like(P[k])
            P["m" + k] = torch.zeros_like(P[k])
            P["s" + k] = torch.zeros_like(P[k])
        if bf16:
            P["wb"] = torch.empty(P["w"].shape, dtype=torch.bfloat16, device=self.dev)
            co, _, ci = P["w"].shape
            P["wf"] = torch.empty((ci, 27, co), dtype=torch.bfloat16, device=self.dev)
        self.p[name] = P

    def _sync_weights(self):
        """BF16 copies (an Adam call with lr = 0 and zero gradient converts) and flipped weights."""
        for name, P in self.p.items():
            if "wb" in P:
                adam(P["w"], P["gw"], P["mw"], P["sw"], 0.0, 0.9, 0.999, 1e-8, 1, 0.0, P["wb"], self.stream)
                co, _, ci = P["w"].shape
                conv3d_flip(P["wb"], co, ci, P["wf"], self.stream)

    def num_params(self):
        return sum(P["w"].numel() + P["b"].numel() for P in self.p.values())

    def state(self):
        return {k: (P["w"].cpu().numpy(), P["b"].cpu().numpy()) for k, P in self.p.items()}

    def load_state(self, st):
        for k, (w, b) in st.items():
            self.p[k]["w"].copy_(self.torch.from_numpy(np.ascontiguousarray(w, dtype=np.float32)))
            self.p[k]["b"].copy_(self.torch.from_numpy(np.ascontiguousarray(b, dtype=np.float32)))
        self._sync_weights()

    # ---- weight files ----
    def save_weights(self, path, meta=None):
        """Write the parameters to an .npz file: convolution weights as BF16
        bit patterns (uint16, round to nearest even; the forward pass uses BF16
        weights, so nothing is lost for inference), biases and the head in
        FP32, and the architecture (channels, input channels, slope, vscale)."""
        import json
        arrays = {}
        for k, (w, b) in self.state().items():
            if "wb" in self.p[k]:
                u = w.astype(np.float32).view(np.uint32)
                arrays[k + ".w_bf16"] = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
            else:
                arrays[k + ".w"] = w.astype(np.float32)
            arrays[k + ".b"] = b.astype(np.float32)
        info = {"chans": list(self.chans), "cin": self.cin, "slope": self.slope, "vscale": self.vscale,
                "pc_head": self.pc_head}
        if meta:
            info.update(meta)
        arrays["__meta__"] = np.frombuffer(json.dumps(info).encode(), dtype=np.uint8)
        np.savez(path, **arrays)

    @staticmethod
    def read_weights(path):
        """(meta dict, state dict name -> (w FP32, b FP32)) of a file written by save_weights."""
        import json
        z = np.load(path)
        meta = json.loads(bytes(z["__meta__"]).decode())
        st = {}
        for key in z.files:
            if key == "__meta__" or key.endswith(".b"):
                continue
            name, kind = key.rsplit(".", 1)
            w = (z[key].astype(np.uint32) << 16).view(np.float32) if kind == "w_bf16" else z[key]
            st[name] = (w, z[name + ".b"])
        return meta, st

    @classmethod
    def from_file(cls, path, stream=None):
        """A network with the architecture and parameters stored in `path`."""
        meta, st = cls.read_weights(path)
        u = cls(chans=tuple(meta["chans"]), cin=meta["cin"], slope=meta["slope"], vscale=meta["vscale"],
                seed=0, stream=stream, pc_head=meta.get("pc_head", False))
        u.load_state(st)
        u.meta = meta
        return u

    # ---- buffers per input shape ----
    def _buffers(self, B, D, H, W):
        key = (B, D, H, W)
        if key in self._bufs:
            return self._bufs[key]
        torch, ch = self.torch, self.chans
        L = len(ch)

        def new(l, C):
            return torch.empty((B, D >> l, H >> l, W >> l, C), dtype=torch.bfloat16, device=self.dev)

        b = {"x": new(0, self.cin)}
        for l in range(L - 1):
            b["a%d" % l] = new(l, ch[l])                     # enc a output
            b["cat%d" % l] = new(l, ch[l] + ch[l + 1])       # [enc b output | upsampled]
            b["p%d" % l] = new(l + 1, ch[l])                 # pooled
            b["da%d" % l] = new(l, ch[l])                    # dec a output
            b["d%d" % l] = new(l, ch[l])                     # dec b output
        b["ba"] = new(L - 1, ch[-1])
        b["bb"] = new(L - 1, ch[-1])
        # gradient scratch: per level two buffers of the widest tensor there
        for l in range(L):
            wmax = max(ch[l] + (ch[l + 1] if l + 1 < L else 0), ch[l], 16)
            b["g%d_0" % l] = new(l, wmax)
            b["g%d_1" % l] = new(l, wmax)
            b["g%d_2" % l] = new(l, wmax)
        maxp = 16
        for name, ci, co in self.layers:
            lvl = self._level(name)
            vol = (B, D >> lvl, H >> lvl, W >> lvl)
            maxp = max(maxp, wgrad_chunks(ci, co, vol) * co * 27 * ci)
        b["part"] = torch.empty(maxp, dtype=torch.float32, device=self.dev)
        b["partb"] = torch.empty(max(16, maxp // 27), dtype=torch.float32, device=self.dev)
        hb = ctypes.c_int()
        _check(lib().claire_net_head_bwd_blocks(_I4(B, D, H, W), ctypes.byref(hb)), "head_bwd_blocks")
        b["hblocks"] = hb.value
        no = self.nout
        b["hpart"] = torch.empty(hb.value * (no * ch[0] + no), dtype=torch.float32, device=self.dev)
        b["hgrad"] = torch.empty(no * ch[0] + no, dtype=torch.float32, device=self.dev)
        b["v"] = torch.empty((B, no, D, H, W), dtype=torch.float32, device=self.dev)
        self._bufs = {key: b}  # keep one shape at a time
        return b

    def _level(self, name):
        if name.startswith("bot"):
            return len(self.chans) - 1
        return int(name[3])

    # ---- forward ----
    def _conv(self, name, x, y):
        P = self.p[name]
        conv3d(x, P["wb"], P["b"], y, self.slope, 1, self.stream)

    def forward(self, m0, m1, a0=1.0, a1=1.0):
        """m0, m1: FP32 CUDA tensors [B, D, H, W] (or [D, H, W]); returns v [B, 3, D, H, W]."""
        if m0.dim() == 3:
            m0, m1 = m0[None], m1[None]
        B, D, H, W = m0.shape
        b = self._buffers(B, D, H, W)
        ch, L = self.chans, len(self.chans)
        _check(lib().claire_net_pack(m0.data_ptr(), m1.data_ptr(), a0, a1, m0.numel(), b["x"].data_ptr(),
                                     self.cin, self.stream), "pack")
        h = Act(b["x"], 0, self.cin)
        for l in range(L - 1):
            a = Act(b["a%d" % l], 0, ch[l])
            e = Act(b["cat%d" % l], 0, ch[l])
            self._conv("enc%da" % l, h, a)
            self._conv("enc%db" % l, a, e)
            p = Act(b["p%d" % l], 0, ch[l])
            pool2(e, p, self.stream)
            h = p
        ba, bb = Act(b["ba"], 0, ch[-1]), Act(b["bb"], 0, ch[-1])
        self._conv("bota", h, ba)
        self._conv("botb", ba, bb)
        h = bb
        for l in range(L - 2, -1, -1):
            cat = b["cat%d" % l]
            up2(h, Act(cat, ch[l], ch[l + 1]), self.stream)
            da, d = Act(b["da%d" % l], 0, ch[l]), Act(b["d%d" % l], 0, ch[l])
            self._conv("dec%da" % l, Act(cat, 0, ch[l] + ch[l + 1]), da)
            self._conv("dec%db" % l, da, d)
            h = d
        P = self.p["head"]
        _check(lib().claire_net_head(h.ptr, h.stride, h.C, self.nout, P["w"].data_ptr(), P["b"].data_ptr(),
                                     self.vscale, b["v"].data_ptr(), h.v4(), self.stream), "head")
        self._last = (B, D, H, W)
        return b["v"][:, :3]

    def pc_logit(self):
        """Channel 3 of the last forward pass (pc_head networks): [B, D, H, W],
        the logit o of the coarse preconditioner weight w = softplus(o)."""
        if not self.pc_head:
            raise NetError("this network has no preconditioner head")
        return self._bufs[self._last]["v"][:, 3]

    def output_grad(self):
        """Buffer [B, nout, D, H, W] (FP32) for the gradient of the loss with
        respect to the head's output, the argument of backward()."""
        B, D, H, W = self._last
        key = ("dout", B, D, H, W)
        if getattr(self, "_dout_key", None) != key:
            self._dout = self.torch.zeros((B, self.nout, D, H, W), dtype=self.torch.float32, device=self.dev)
            self._dout_key = key
        return self._dout

    # ---- backward ----
    def _conv_back(self, name, xin, y, dy, dx):
        """dy: gradient w.r.t. the activated output y; writes dx (may be None)."""
        P = self.p[name]
        b = self._bufs[self._last]
        lvl = self._level(name)
        g = Act(b["g%d_2" % lvl], 0, y.C)
        leaky_bwd(dy, y, self.slope, g, self.stream)
        co, _, ci = P["w"].shape
        chunks = wgrad_chunks(ci, co, y.vol)
        conv3d_wgrad(xin, g, chunks, b["part"], b["partb"], P["gw"], P["gb"], self.stream)
        if dx is not None:
            conv3d(g, P["wf"], None, dx, 0.0, 0, self.stream)

    def backward(self, dv):
        """dv: FP32 [B, nout, D, H, W] (contiguous), gradient of the loss w.r.t.
        the head's output: the velocity and, with pc_head, the logit."""
        if tuple(dv.shape[:2]) != (self._last[0], self.nout) or not dv.is_contiguous():
            raise NetError("backward: dv must be a contiguous [B, %d, D, H, W] tensor" % self.nout)
        b = self._bufs[self._last]
        ch, L = self.chans, len(self.chans)
        B, D, H, W = self._last
        P = self.p["head"]
        d0 = Act(b["d0"], 0, ch[0])
        gh = Act(b["g0_0"], 0, ch[0])
        _check(lib().claire_net_head_bwd(d0.ptr, d0.stride, d0.C, self.nout, P["w"].data_ptr(), self.vscale,
                                         dv.data_ptr(), gh.ptr, gh.stride, d0.v4(), b["hblocks"],
                                         b["hpart"].data_ptr(), b["hgrad"].data_ptr(), self.stream), "head_bwd")
        c0, no = ch[0], self.nout
        P["gw"].copy_(b["hgrad"][:no * c0].view(no, c0))
        P["gb"].copy_(b["hgrad"][no * c0:])
        dh = gh
        for l in range(L - 1):
            cat = b["cat%d" % l]
            da = Act(b["da%d" % l], 0, ch[l])
            d = Act(b["d%d" % l], 0, ch[l])
            dda = Act(b["g%d_1" % l], 0, ch[l])
            self._conv_back("dec%db" % l, da, d, dh, dda)
            dcat = Act(b["g%d_0" % l], 0, ch[l] + ch[l + 1])
            self._conv_back("dec%da" % l, Act(cat, 0, ch[l] + ch[l + 1]), da, dda, dcat)
            # gradient of the upsampled half flows to the coarser decoder output
            dup = Act(b["g%d_1" % (l + 1)], 0, ch[l + 1])
            up2_bwd(Act(dcat.buf, ch[l], ch[l + 1]), dup, self.stream)
            dh = dup
        ba, bb = Act(b["ba"], 0, ch[-1]), Act(b["bb"], 0, ch[-1])
        lb = L - 1
        dba = Act(b["g%d_0" % lb], 0, ch[-1])
        self._conv_back("botb", ba, bb, dh, dba)
        dp = Act(b["g%d_1" % lb], 0, ch[-2])
        self._conv_back("bota", Act(b["p%d" % (L - 2)], 0, ch[-2]), ba, dba, dp)
        for l in range(L - 2, -1, -1):
            # d(enc b output) = pool adjoint of dp + skip part of the concat gradient
            de = Act(b["g%d_1" % l], 0, ch[l])
            pool2_bwd(dp, Act(b["g%d_0" % l], 0, ch[l]), de, self.stream)
            a = Act(b["a%d" % l], 0, ch[l])
            e = Act(b["cat%d" % l], 0, ch[l])
            dga = Act(b["g%d_0" % l], 0, ch[l])  # skip gradient consumed above
            self._conv_back("enc%db" % l, a, e, de, dga)
            xin = Act(b["p%d" % (l - 1)], 0, ch[l - 1]) if l > 0 else Act(b["x"], 0, self.cin)
            if l > 0:
                dpn = Act(b["g%d_1" % l], 0, ch[l - 1])
                self._conv_back("enc%da" % l, xin, a, dga, dpn)
                dp = dpn
            else:
                self._conv_back("enc%da" % l, xin, a, dga, None)

    def step(self, lr, b1=0.9, b2=0.999, eps=1e-8, gscale=1.0):
        self.t += 1
        for name, P in self.p.items():
            adam(P["w"], P["gw"], P["mw"], P["sw"], lr, b1, b2, eps, self.t, gscale, P.get("wb"), self.stream)
            adam(P["b"], P["gb"], P["mb"], P["sb"], lr, b1, b2, eps, self.t, gscale, None, self.stream)
            if "wf" in P:
                co, _, ci = P["w"].shape
                conv3d_flip(P["wb"], co, ci, P["wf"], self.stream)
