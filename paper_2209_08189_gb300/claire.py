"""Thin ctypes binding of libclaire.so (C ABI in include/claire.h).

Argument marshalling only: every numeric step runs in the library's CUDA
kernels (and cuFFT).  Arrays are passed as raw pointers: torch CUDA tensors
(device) or numpy arrays / CPU tensors (host; the library stages them).
Each ``claire_*`` function returns the C status and raises ``ClaireError``
for negative statuses.  There is no fallback: if the library is missing or
no CUDA device is usable, loading or ``claire_create`` fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libclaire.so")

CLAIRE_OK = 0
CLAIRE_ENOTCONVERGED = 1
STATUS_NAMES = {0: "CLAIRE_OK", 1: "CLAIRE_ENOTCONVERGED", -1: "CLAIRE_EINVAL",
                -2: "CLAIRE_ENOMEM", -3: "CLAIRE_ECUDA", -4: "CLAIRE_ECUFFT",
                -5: "CLAIRE_ENONFINITE", -6: "CLAIRE_ELINESEARCH", -7: "CLAIRE_ETIMEOUT",
                -8: "CLAIRE_ESTATE", -9: "CLAIRE_ENOTIMPL", -10: "CLAIRE_ETOOLARGE"}
INTERP_CUBIC, INTERP_LINEAR, INTERP_BSPLINE = 3, 1, 4
TRANSPORT_FWD, TRANSPORT_ADJ = 0, 1
SPECTRAL_REG, SPECTRAL_INV, SPECTRAL_K = 0, 1, 2
STORAGE_F32, STORAGE_F16, STORAGE_BF16 = 0, 1, 2
PRECOND_SPECTRAL, PRECOND_TWO_LEVEL = 0, 1
PHASES = ["backtrace", "state", "adjoint", "incremental", "spectral", "vector", "objective",
          "gather"]
MAX_LOGGED_STEPS = 64


class ClaireError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class claire_opts(ctypes.Structure):
    _fields_ = [("interp", ctypes.c_int), ("reg", ctypes.c_int), ("beta_w", ctypes.c_double),
                ("grad_form", ctypes.c_int), ("gtol", ctypes.c_double), ("max_gn", ctypes.c_int),
                ("max_pcg", ctypes.c_int), ("pcg_rtol_max", ctypes.c_double),
                ("pcg_fixed", ctypes.c_int), ("armijo_c1", ctypes.c_double),
                ("max_ls", ctypes.c_int), ("wall_limit_s", ctypes.c_double),
                ("timing", ctypes.c_int), ("storage", ctypes.c_int), ("g0_ref", ctypes.c_double),
                ("lowmem", ctypes.c_int), ("precond", ctypes.c_int), ("pc_coarse", ctypes.c_int),
                ("pc_tol", ctypes.c_double), ("pc_maxit", ctypes.c_int),
                ("spectral_iterate", ctypes.c_int), ("kernels_only", ctypes.c_int)]


class claire_report(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("gn_iters", ctypes.c_int),
                ("pcg_iters_total", ctypes.c_int),
                ("pcg_iters", ctypes.c_int * MAX_LOGGED_STEPS),
                ("alpha", ctypes.c_double * MAX_LOGGED_STEPS),
                ("J", ctypes.c_double), ("mismatch", ctypes.c_double), ("r", ctypes.c_double),
                ("gnorm_rel", ctypes.c_double), ("detj_min", ctypes.c_double),
                ("detj_max", ctypes.c_double), ("cfl", ctypes.c_double),
                ("t_total_s", ctypes.c_double), ("t_phase_s", ctypes.c_double * 8),
                ("gather_launches", ctypes.c_double), ("interp_points", ctypes.c_double),
                ("interp_bytes", ctypes.c_double), ("pc_inner_iters_total", ctypes.c_int),
                ("pc_fallbacks", ctypes.c_int)]

    def as_dict(self):
        n = min(self.gn_iters, MAX_LOGGED_STEPS)
        return {"status": STATUS_NAMES.get(self.status, self.status), "gn_iters": self.gn_iters,
                "pcg_iters_total": self.pcg_iters_total,
                "pcg_iters": [self.pcg_iters[i] for i in range(n + (1 if self.status < 0 else 0))
                              if i < MAX_LOGGED_STEPS],
                "alpha": [self.alpha[i] for i in range(n)], "J": self.J,
                "mismatch": self.mismatch, "r": self.r, "gnorm_rel": self.gnorm_rel,
                "detj_min": self.detj_min, "detj_max": self.detj_max, "cfl": self.cfl,
                "t_total_s": self.t_total_s,
                "t_phase_s": {k: self.t_phase_s[i] for i, k in enumerate(PHASES)},
                "gather_launches": self.gather_launches, "interp_points": self.interp_points,
                "interp_bytes": self.interp_bytes, "pc_inner_iters_total": self.pc_inner_iters_total,
                "pc_fallbacks": self.pc_fallbacks}


class claire_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_double),
                ("seconds", ctypes.c_double), ("bytes", ctypes.c_double),
                ("points", ctypes.c_double)]


_lib = None
class claire_search_opts(ctypes.Structure):
    _fields_ = [("beta_v_max", ctypes.c_double), ("beta_v_min", ctypes.c_double),
                ("beta_w_max", ctypes.c_double), ("beta_w_min", ctypes.c_double),
                ("jmin", ctypes.c_double), ("bisect_rtol", ctypes.c_double), ("max_solves", ctypes.c_int)]


MAX_SEARCH_SOLVES = 64


class claire_search_report(ctypes.Structure):
    _fields_ = [("beta_v", ctypes.c_double), ("beta_w", ctypes.c_double), ("solves", ctypes.c_int),
                ("trace_beta_v", ctypes.c_double * MAX_SEARCH_SOLVES),
                ("trace_beta_w", ctypes.c_double * MAX_SEARCH_SOLVES),
                ("trace_detj_min", ctypes.c_double * MAX_SEARCH_SOLVES),
                ("trace_detj_max", ctypes.c_double * MAX_SEARCH_SOLVES),
                ("trace_valid", ctypes.c_int * MAX_SEARCH_SOLVES),
                ("trace_gn_iters", ctypes.c_int * MAX_SEARCH_SOLVES),
                ("t_total_s", ctypes.c_double), ("last", claire_report)]

    def as_dict(self):
        n = min(self.solves, MAX_SEARCH_SOLVES)
        return {"beta_v": self.beta_v, "beta_w": self.beta_w, "solves": self.solves,
                "trace": [{"beta_v": self.trace_beta_v[i], "beta_w": self.trace_beta_w[i],
                           "detj_min": self.trace_detj_min[i], "detj_max": self.trace_detj_max[i],
                           "valid": bool(self.trace_valid[i]), "gn_iters": self.trace_gn_iters[i]}
                          for i in range(n)],
                "t_total_s": self.t_total_s, "last": self.last.as_dict()}


_vp = ctypes.c_void_p
_ST = ctypes.c_int

# name -> argtypes (restype claire_status unless listed in _RESTYPE)
_SIGS = {
    "claire_default_opts": [ctypes.POINTER(claire_opts)],
    "claire_create": [ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_int), ctypes.c_double,
                      ctypes.c_int, ctypes.POINTER(claire_opts)],
    "claire_destroy": [_vp],
    "claire_set_stream": [_vp, _vp],
    "claire_query_workspace": [ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                               ctypes.POINTER(claire_opts), ctypes.POINTER(ctypes.c_size_t)],
    "claire_set_images": [_vp, _vp, _vp],
    "claire_objective": [_vp, _vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
    "claire_gradient": [_vp, _vp, _vp, ctypes.POINTER(ctypes.c_double)],
    "claire_hessian_matvec": [_vp, _vp, _vp],
    "claire_precond": [_vp, _vp, _vp],
    "claire_set_pc_weight": [_vp, _vp, ctypes.POINTER(ctypes.c_int)],
    "claire_mean_state_gradient": [_vp, _vp],
    "claire_register": [_vp, _vp, ctypes.POINTER(claire_report)],
    "claire_transport": [_vp, _vp, _vp, _vp, ctypes.c_int],
    "claire_detj": [_vp, _vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
    "claire_transport_vjp": [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int],
    "claire_resample_release": [],
    "claire_set_opts": [_vp, ctypes.POINTER(claire_opts)],
    "claire_set_beta": [_vp, ctypes.c_double, ctypes.c_double],
    "claire_get_beta": [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
    "claire_default_search_opts": [ctypes.POINTER(claire_search_opts)],
    "claire_param_search": [_vp, _vp, ctypes.POINTER(claire_search_opts), ctypes.POINTER(claire_search_report)],
    "claire_param_continuation": [_vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.POINTER(claire_search_opts),
                                  ctypes.POINTER(claire_search_report)],
    "claire_get_opts": [_vp, ctypes.POINTER(claire_opts)],
    "claire_resample": [_vp, ctypes.POINTER(ctypes.c_int), _vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                        ctypes.c_int, _vp],
    "claire_interp": [_vp, _vp, _vp, _vp, ctypes.c_int],
    "claire_interp_fields": [_vp, _vp, ctypes.c_int, _vp, _vp, ctypes.c_int],
    "claire_dice": [_vp, _vp, _vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_double)],
    "claire_gather_fallback_tiles": [ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_int],
    "claire_backtrace": [_vp, _vp, _vp, ctypes.c_int],
    "claire_fd8_grad": [_vp, _vp, _vp],
    "claire_fd8_div": [_vp, _vp, _vp],
    "claire_spectral": [_vp, _vp, _vp, ctypes.c_int],
    "claire_dot": [_vp, _vp, _vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_double)],
    "claire_dot_noalloc": [_vp, _vp, ctypes.c_size_t, ctypes.c_double, _vp,
                           ctypes.POINTER(ctypes.c_double)],
    "claire_kernel_stats": [_vp, ctypes.POINTER(claire_kernel_stat), ctypes.c_int,
                            ctypes.POINTER(ctypes.c_int), ctypes.c_int],
    "claire_set_timing": [_vp, ctypes.c_int],
    "claire_last_error": [_vp],
}
_RESTYPE = {"claire_last_error": ctypes.c_char_p}


def lib():
    """Load libclaire.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libclaire.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = _RESTYPE.get(name, _ST)
        _lib = L
    return _lib


def exported_symbols():
    return sorted(_SIGS)


def _ptr(a):
    """Raw address of a torch tensor or numpy array (contiguous float32)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy arrays must be contiguous float32")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if a.dtype.__repr__() != "torch.float32" or not a.is_contiguous():
            raise ValueError("tensors must be contiguous float32")
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError("unsupported array type %r" % type(a))


def _check(ctx, status):
    if status < 0:
        msg = lib().claire_last_error(ctx).decode() if ctx else ""
        raise ClaireError(status, msg)
    return status


# ---- functions with the C names (argument marshalling only) ----

def claire_default_opts():
    o = claire_opts()
    _check(None, lib().claire_default_opts(ctypes.byref(o)))
    return o


def claire_create(grid, beta_v, nt, opts=None):
    h = _vp()
    g = (ctypes.c_int * 3)(*[int(x) for x in grid])
    st = lib().claire_create(ctypes.byref(h), g, float(beta_v), int(nt),
                             ctypes.byref(opts) if opts is not None else None)
    if st < 0:
        raise ClaireError(st, "claire_create(grid=%s, beta_v=%g, nt=%d)" % (tuple(grid), beta_v, nt))
    return h


def claire_destroy(ctx):
    return lib().claire_destroy(ctx)


def claire_set_stream(ctx, stream_handle):
    return _check(ctx, lib().claire_set_stream(ctx, stream_handle))


def claire_query_workspace(grid, nt, opts=None):
    b = ctypes.c_size_t()
    g = (ctypes.c_int * 3)(*[int(x) for x in grid])
    _check(None, lib().claire_query_workspace(g, int(nt), ctypes.byref(opts) if opts else None,
                                              ctypes.byref(b)))
    return b.value


def claire_set_images(ctx, m0, m1):
    return _check(ctx, lib().claire_set_images(ctx, _ptr(m0), _ptr(m1)))


def claire_objective(ctx, v):
    J = ctypes.c_double()
    mis = ctypes.c_double()
    _check(ctx, lib().claire_objective(ctx, _ptr(v), ctypes.byref(J), ctypes.byref(mis)))
    return J.value, mis.value


def claire_gradient(ctx, v, g):
    J = ctypes.c_double()
    _check(ctx, lib().claire_gradient(ctx, _ptr(v), _ptr(g), ctypes.byref(J)))
    return J.value


def claire_hessian_matvec(ctx, vt, Hvt):
    return _check(ctx, lib().claire_hessian_matvec(ctx, _ptr(vt), _ptr(Hvt)))


def claire_precond(ctx, r, z):
    return _check(ctx, lib().claire_precond(ctx, _ptr(r), _ptr(z)))


def claire_set_pc_weight(ctx, w, wgrid=None):
    """Install (w: FP32 [Nc1, Nc2, Nc3], device or host) or clear (w None) the
    coarse preconditioner weight of the two-level preconditioner."""
    if w is None:
        return _check(ctx, lib().claire_set_pc_weight(ctx, None, None))
    g = (ctypes.c_int * 3)(*(int(x) for x in (wgrid if wgrid is not None else w.shape)))
    return _check(ctx, lib().claire_set_pc_weight(ctx, _ptr(w), g))


def claire_mean_state_gradient(ctx, gbar):
    return _check(ctx, lib().claire_mean_state_gradient(ctx, _ptr(gbar)))


def claire_register(ctx, v_inout, check=True):
    """check=False returns a failure status (with the report of the run) instead of raising."""
    rep = claire_report()
    st = lib().claire_register(ctx, _ptr(v_inout), ctypes.byref(rep))
    if check:
        _check(ctx, st)
    return st, rep


def claire_transport(ctx, v, m_in, m_out, flags=TRANSPORT_FWD):
    return _check(ctx, lib().claire_transport(ctx, _ptr(v), _ptr(m_in), _ptr(m_out), int(flags)))


VJP_RECOMPUTE = 1


def claire_transport_vjp(ctx, v, m0, gbar, gm0=None, gv=None, flags=0):
    return _check(ctx, lib().claire_transport_vjp(ctx, _ptr(v), _ptr(m0), _ptr(gbar), _ptr(gm0), _ptr(gv),
                                                  int(flags)))


RESAMPLE_SPECTRAL, RESAMPLE_NEAREST = 0, 1


def claire_resample(inp, from_grid, out, to_grid, ncomp=1, mode=RESAMPLE_SPECTRAL, stream=None):
    f = (ctypes.c_int * 3)(*[int(x) for x in from_grid])
    t = (ctypes.c_int * 3)(*[int(x) for x in to_grid])
    st = lib().claire_resample(_ptr(inp), f, _ptr(out), t, int(ncomp), int(mode), stream)
    if st < 0:
        raise ClaireError(st, "claire_resample %s -> %s" % (tuple(from_grid), tuple(to_grid)))
    return st


def claire_set_opts(ctx, opts):
    return _check(ctx, lib().claire_set_opts(ctx, ctypes.byref(opts)))


def claire_set_beta(ctx, beta_v, beta_w):
    return _check(ctx, lib().claire_set_beta(ctx, float(beta_v), float(beta_w)))


def claire_get_beta(ctx):
    bv, bw = ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib().claire_get_beta(ctx, ctypes.byref(bv), ctypes.byref(bw)))
    return bv.value, bw.value


def claire_default_search_opts(**kw):
    o = claire_search_opts()
    _check(None, lib().claire_default_search_opts(ctypes.byref(o)))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError("unknown search option %r" % k)
        setattr(o, k, v)
    return o


def claire_param_search(ctx, v_inout, opts=None):
    rep = claire_search_report()
    st = _check(ctx, lib().claire_param_search(ctx, _ptr(v_inout), ctypes.byref(opts) if opts else None,
                                               ctypes.byref(rep)))
    return st, rep.as_dict()


def claire_param_continuation(ctx, v_inout, target_beta_v, target_beta_w, opts=None):
    rep = claire_search_report()
    st = _check(ctx, lib().claire_param_continuation(ctx, _ptr(v_inout), float(target_beta_v), float(target_beta_w),
                                                     ctypes.byref(opts) if opts else None, ctypes.byref(rep)))
    return st, rep.as_dict()


def claire_get_opts(ctx):
    o = claire_opts()
    _check(ctx, lib().claire_get_opts(ctx, ctypes.byref(o)))
    return o


def claire_detj(ctx, v):
    lo = ctypes.c_double()
    hi = ctypes.c_double()
    _check(ctx, lib().claire_detj(ctx, _ptr(v), ctypes.byref(lo), ctypes.byref(hi)))
    return lo.value, hi.value


def claire_interp(ctx, f, d, out, order=INTERP_CUBIC):
    return _check(ctx, lib().claire_interp(ctx, _ptr(f), _ptr(d), _ptr(out), int(order)))


def claire_interp_fields(ctx, f, nf, d, out, order=INTERP_CUBIC):
    return _check(ctx, lib().claire_interp_fields(ctx, _ptr(f), int(nf), _ptr(d), _ptr(out), int(order)))


def claire_dice(ctx, a, b, n=None):
    """Dice overlap of {a >= 1/2} and {b >= 1/2} (device float32 arrays)."""
    out = ctypes.c_double()
    _check(ctx, lib().claire_dice(ctx, _ptr(a), _ptr(b), int(n if n is not None else a.numel()), ctypes.byref(out)))
    return out.value


def claire_gather_fallback_tiles(reset=False):
    """CTAs of the tiled gathers that took the global-memory path (current device)."""
    n = ctypes.c_ulonglong()
    st = lib().claire_gather_fallback_tiles(ctypes.byref(n), int(bool(reset)))
    if st < 0:
        raise ClaireError(st, "claire_gather_fallback_tiles")
    return int(n.value)


def claire_backtrace(ctx, v, d, direction=1):
    return _check(ctx, lib().claire_backtrace(ctx, _ptr(v), _ptr(d), int(direction)))


def claire_fd8_grad(ctx, f, g):
    return _check(ctx, lib().claire_fd8_grad(ctx, _ptr(f), _ptr(g)))


def claire_fd8_div(ctx, v, dv):
    return _check(ctx, lib().claire_fd8_div(ctx, _ptr(v), _ptr(dv)))


def claire_spectral(ctx, x, out, op):
    return _check(ctx, lib().claire_spectral(ctx, _ptr(x), _ptr(out), int(op)))


def claire_dot(ctx, x, y, n):
    out = ctypes.c_double()
    _check(ctx, lib().claire_dot(ctx, _ptr(x), _ptr(y), int(n), ctypes.byref(out)))
    return out.value


def claire_dot_noalloc(x, y, n, scale, stream=None):
    """FP64 scale * sum(x * y) over n floats without any device allocation
    (for callers that cannot allocate; see include/claire.h).  Returns
    (status, value); negative statuses raise ClaireError."""
    out = ctypes.c_double()
    st = lib().claire_dot_noalloc(_ptr(x), _ptr(y), int(n), float(scale), stream,
                                  ctypes.byref(out))
    if st < 0:
        raise ClaireError(st, "claire_dot_noalloc(n=%d)" % int(n))
    return st, out.value


def claire_kernel_stats(ctx, reset=False):
    arr = (claire_kernel_stat * 32)()
    cnt = ctypes.c_int()
    _check(ctx, lib().claire_kernel_stats(ctx, arr, 32, ctypes.byref(cnt), int(bool(reset))))
    return [{"name": arr[i].name.decode(), "launches": arr[i].launches,
             "seconds": arr[i].seconds, "bytes": arr[i].bytes, "points": arr[i].points}
            for i in range(cnt.value)]


def claire_set_timing(ctx, on):
    return _check(ctx, lib().claire_set_timing(ctx, int(bool(on))))


def claire_last_error(ctx):
    return lib().claire_last_error(ctx).decode()


class Context:
    """Owning wrapper: ``Context(grid, beta_v, nt, **opts)``; methods take
    torch CUDA tensors (or host numpy arrays) and call the C ABI."""

    def __init__(self, grid, beta_v, nt, stream=None, **opts):
        o = claire_default_opts()
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError("unknown option %r" % k)
            setattr(o, k, v)
        self.grid = tuple(int(x) for x in grid)
        self.N = int(np.prod(self.grid))
        self.nt = int(nt)
        self.beta_v = float(beta_v)
        self.opts = o
        self.handle = claire_create(self.grid, beta_v, nt, o)
        if stream is not None:
            claire_set_stream(self.handle, stream)

    def close(self):
        if getattr(self, "handle", None):
            claire_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_handle):
        claire_set_stream(self.handle, stream_handle)

    def set_beta(self, beta_v, beta_w):
        claire_set_beta(self.handle, beta_v, beta_w)

    def param_search(self, v_inout, **search_opts):
        return claire_param_search(self.handle, v_inout, claire_default_search_opts(**search_opts))

    def param_continuation(self, v_inout, target_beta_v, target_beta_w, **search_opts):
        return claire_param_continuation(self.handle, v_inout, target_beta_v, target_beta_w,
                                         claire_default_search_opts(**search_opts))

    def set_opts(self, **opts):
        """Change options of the live context (storage excluded)."""
        o = claire_get_opts(self.handle)
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError("unknown option %r" % k)
            setattr(o, k, v)
        claire_set_opts(self.handle, o)
        self.opts = o

    def set_images(self, m0, m1):
        claire_set_images(self.handle, m0, m1)

    def objective(self, v):
        return claire_objective(self.handle, v)

    def gradient(self, v, g):
        return claire_gradient(self.handle, v, g)

    def hessian_matvec(self, vt, Hvt):
        claire_hessian_matvec(self.handle, vt, Hvt)

    def precond(self, r, z):
        claire_precond(self.handle, r, z)

    def set_pc_weight(self, w, wgrid=None):
        claire_set_pc_weight(self.handle, w, wgrid)

    def mean_state_gradient(self, gbar):
        claire_mean_state_gradient(self.handle, gbar)

    def register(self, v_inout, check=True):
        st, rep = claire_register(self.handle, v_inout, check)
        return st, rep.as_dict()

    def transport(self, v, m_in, m_out, flags=TRANSPORT_FWD):
        claire_transport(self.handle, v, m_in, m_out, flags)

    def detj(self, v):
        return claire_detj(self.handle, v)

    def transport_vjp(self, v, m0, gbar, gm0=None, gv=None, recompute=False):
        claire_transport_vjp(self.handle, v, m0, gbar, gm0, gv, VJP_RECOMPUTE if recompute else 0)

    def interp(self, f, d, out, order=INTERP_CUBIC):
        claire_interp(self.handle, f, d, out, order)

    def dice(self, a, b):
        return claire_dice(self.handle, a, b)

    def interp_fields(self, f, nf, d, out, order=INTERP_CUBIC):
        claire_interp_fields(self.handle, f, nf, d, out, order)

    def backtrace(self, v, d, direction=1):
        claire_backtrace(self.handle, v, d, direction)

    def fd8_grad(self, f, g):
        claire_fd8_grad(self.handle, f, g)

    def fd8_div(self, v, dv):
        claire_fd8_div(self.handle, v, dv)

    def spectral(self, x, out, op):
        claire_spectral(self.handle, x, out, op)

    def dot(self, x, y, n=None):
        return claire_dot(self.handle, x, y, n if n is not None else x.numel())

    def kernel_stats(self, reset=False):
        return claire_kernel_stats(self.handle, reset)

    def set_timing(self, on):
        claire_set_timing(self.handle, on)


def sl_transport(context, m0, v, recompute=False):
    """Differentiable semi-Lagrangian transport m(1) = T(v)^nt m0 on the GPU.

    Forward: claire_transport; backward: claire_transport_vjp (exact
    derivative of the discrete map, hand-written scatter-transpose and
    interpolant-gradient kernels).  m0: (N1,N2,N3), v: (3,N1,N2,N3) float32
    CUDA tensors; context: a Context on the same grid.  torch is imported
    here only for the autograd plumbing.
    """
    import torch

    class _SLTransport(torch.autograd.Function):
        @staticmethod
        def forward(fctx, m0_, v_):
            m0c, vc = m0_.detach().contiguous(), v_.detach().contiguous()
            out = torch.empty_like(m0c)
            context.transport(vc, m0c, out, TRANSPORT_FWD)
            fctx.save_for_backward(m0c, vc)
            return out

        @staticmethod
        def backward(fctx, gout):
            m0c, vc = fctx.saved_tensors
            gm0 = torch.empty_like(m0c) if fctx.needs_input_grad[0] else None
            gv = torch.empty_like(vc) if fctx.needs_input_grad[1] else None
            context.transport_vjp(vc, m0c, gout.detach().contiguous(), gm0, gv, recompute)
            return gm0, gv

    return _SLTransport.apply(m0, v)
