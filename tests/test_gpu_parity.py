"""GPU parity: every entry point of the C ABI against the FP64 oracle on the
same seeded FP32 inputs (the oracle reads the FP32 bits upcast to FP64).

Tolerances (CUDA path computes in FP32, reductions in FP64):
  * interpolation: relative L-infinity 1e-5 (stated requirement);
  * transported image: relative L2 2e-4 (stated requirement);
  * backtrace, FD8, spectral operators, single SL steps: 1e-5 relative — each
    output is a short FP32 sum (<= 64 terms, |weights| summing to <= 2), so
    the rounding error is a few units of 6e-8 times the largest term;
  * gradient and Hessian matvec: relative L2 1e-4 — 2 nt SL steps of 1e-6
    relative rounding each, amplified by the cancellation in m1 - m(1)
    (|m| / |m - m1| <= 10 on these inputs);
  * registration: final velocity relative L2 1e-3 and final relative
    mismatch within 1 % of the oracle (stated requirements).
"""
import math

import numpy as np
import pytest

import __graft_entry__ as entry
import oracle
from paper_2209_08189_gb300 import synth

from fp32_bounds import fft_roundoff_bound, split_check

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


def rel_linf(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def make_ctx(claire, torch, n, beta_v=1e-2, nt=4, **opts):
    return claire.Context(n, beta_v, nt, stream=torch.cuda.current_stream().cuda_stream, **opts)


# (40,36,30): N = 43200, ragged last block.  Along x3 a tile's departure box
# (32 columns plus the stencil and the spread) is wider than these three grids,
# so they run the global-memory path of the tiled gathers; (70,44,104) is ragged
# along every axis (partial tiles) and wide enough for the shared-memory box.
SHAPES = [(32, 32, 32), (40, 36, 30), (16, 24, 8), (70, 44, 104)]


def _disp(n, seed, cfl):
    """Smooth displacement (grid units) with max about cfl cells, plus a wrap-crossing offset."""
    v = synth.mode_velocity(n, seed=seed, kmax=3, vmax=1.0)
    h = oracle.spacing(n)
    d = np.stack([v[c] / h[c] * cfl * h.min() for c in range(3)])
    return d


# ---------------------------------------------------------------------------
# kernels
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("order", [3, 1, 4])
@pytest.mark.parametrize("n", SHAPES)
@pytest.mark.parametrize("cfl", [0.4, 6.0])
def test_interp_parity(env, n, order, cfl):
    torch, claire = env
    f = f32(synth.blob_template(n, seed=1))
    d = f32(_disp(n, 2, cfl))
    ctx = make_ctx(claire, torch, n)
    out = torch.empty(n, device="cuda")
    ctx.interp(dev(torch, f), dev(torch, d), out, order)
    torch.cuda.synchronize()
    ref = oracle.interp(f.astype(np.float64), d.astype(np.float64), order)
    assert rel_linf(host(out), ref) <= 1e-5


@pytest.mark.parametrize("order", [3, 1, 4])
def test_interp_parity_random_displacement_fallback(env, order):
    """Uniform random displacements (+-9 cells, no spatial smoothness) give
    departure boxes larger than the shared-memory tile, so the kernel takes
    its direct global-memory gather; one half of the domain is smooth so both
    paths run in the same launch."""
    torch, claire = env
    n = (32, 40, 64)
    rng = np.random.default_rng(11)
    f = f32(rng.standard_normal(n))
    d = f32(_disp(n, 3, 2.0))
    d[:, : n[0] // 2] = rng.uniform(-9, 9, size=(3, n[0] // 2) + n[1:])
    ctx = make_ctx(claire, torch, n)
    out = torch.empty(n, device="cuda")
    ctx.interp(dev(torch, f), dev(torch, d), out, order)
    torch.cuda.synchronize()
    ref = oracle.interp(f.astype(np.float64), d.astype(np.float64), order)
    assert rel_linf(host(out), ref) <= 1e-5


@pytest.mark.parametrize("order", [3, 1])
@pytest.mark.parametrize("n", [(32, 32, 32), (70, 44, 104)])
def test_interp_fields_parity_and_fallback_count(env, n, order):
    """Three fields at one displacement in one kernel (claire_interp_fields):
    each equals the oracle's interpolation of that field (rel L-inf 1e-5).
    With uniform random displacements (+-9 cells) every tile's box is too
    large, so each of the launch's tiles is counted as a global-memory tile."""
    torch, claire = env
    rng = np.random.default_rng(17)
    f = f32(rng.standard_normal((3,) + n))
    d = f32(_disp(n, 4, 3.0))
    ctx = make_ctx(claire, torch, n)
    out = torch.empty((3,) + n, device="cuda")
    claire.claire_gather_fallback_tiles(reset=True)
    ctx.interp_fields(dev(torch, f), 3, dev(torch, d), out, order)
    torch.cuda.synchronize()
    for q in range(3):
        ref = oracle.interp(f[q].astype(np.float64), d.astype(np.float64), order)
        assert rel_linf(host(out[q]), ref) <= 1e-5
    tiles = -(-n[0] // 4) * -(-n[1] // 8) * -(-n[2] // 32)
    assert claire.claire_gather_fallback_tiles(reset=True) <= tiles
    dr = f32(rng.uniform(-9, 9, size=(3,) + n))
    ctx.interp_fields(dev(torch, f), 3, dev(torch, dr), out, order)
    torch.cuda.synchronize()
    assert claire.claire_gather_fallback_tiles(reset=True) == tiles
    ref = oracle.interp(f[1].astype(np.float64), dr.astype(np.float64), order)
    assert rel_linf(host(out[1]), ref) <= 1e-5


def test_dice_parity(env):
    """claire_dice against the oracle's definition (Sec. 4.1): identical
    values, since both count voxels exactly; on label indicators carried by a
    transport, on equal, disjoint and empty sets, and at the threshold 1/2."""
    torch, claire = env
    n = (40, 36, 30)
    m0 = synth.blob_template(n, seed=2)
    vs = f32(synth.mode_velocity(n, seed=5, vmax=0.5))
    ctx = make_ctx(claire, torch, n, kernels_only=1)
    full = make_ctx(claire, torch, n)
    lab = f32(m0 > 0.5)
    carried = torch.empty(n, device="cuda")
    full.transport(dev(torch, vs), dev(torch, lab), carried)
    torch.cuda.synchronize()
    got = ctx.dice(carried, dev(torch, lab))
    assert got == oracle.dice(host(carried), lab) and 0.0 < got < 1.0
    a = np.zeros(n, np.float32); b = np.zeros(n, np.float32)
    a[:10] = 1.0; b[20:] = 1.0
    assert ctx.dice(dev(torch, a), dev(torch, a)) == 1.0
    assert ctx.dice(dev(torch, a), dev(torch, b)) == 0.0
    assert ctx.dice(dev(torch, np.zeros(n)), dev(torch, np.zeros(n))) == 1.0
    half = np.full(n, 0.5, np.float32)
    assert ctx.dice(dev(torch, half), dev(torch, a)) == oracle.dice(half, a)


def test_kernels_only_context(env):
    """kernels_only = 1: the kernel-level calls give the same bits as a full
    context; solver-level calls return CLAIRE_ESTATE."""
    torch, claire = env
    n = (32, 40, 64)
    rng = np.random.default_rng(2)
    f = dev(torch, rng.standard_normal(n))
    v = dev(torch, synth.mode_velocity(n, seed=4, vmax=0.5))
    full = make_ctx(claire, torch, n)
    lean = make_ctx(claire, torch, n, kernels_only=1)
    outs = []
    for ctx in (full, lean):
        d = torch.empty((3,) + n, device="cuda")
        ctx.backtrace(v, d, 1)
        m = torch.empty(n, device="cuda")
        ctx.interp(f, d, m, 3)
        gr = torch.empty((3,) + n, device="cuda")
        ctx.fd8_grad(f, gr)
        torch.cuda.synchronize()
        outs.append((d.cpu(), m.cpu(), gr.cpu(), ctx.dot(f, f)))
    for a, b in zip(outs[0][:3], outs[1][:3]):
        assert torch.equal(a, b)
    assert outs[0][3] == outs[1][3]
    for call in (lambda: lean.set_images(f, f), lambda: lean.register(torch.zeros((3,) + n, device="cuda")),
                 lambda: lean.transport(v, f, f)):
        with pytest.raises(claire.ClaireError) as e:
            call()
        assert e.value.status == -8


@pytest.mark.parametrize("order", [3, 1])
def test_interp_integer_shift_bit_exact(env, order):
    torch, claire = env
    n = (16, 12, 20)
    rng = np.random.default_rng(0)
    f = f32(rng.standard_normal(n))
    d = np.zeros((3,) + n, np.float32)
    d[0] = 5; d[1] = -13; d[2] = 21
    ctx = make_ctx(claire, torch, n)
    out = torch.empty(n, device="cuda")
    ctx.interp(dev(torch, f), dev(torch, d), out, order)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), np.roll(f, (-5, 13, -21), axis=(0, 1, 2)))


def test_bspline_integer_shift_and_restrictions(env):
    """Cubic B-spline (interp 4): an integer shift returns the shifted grid
    values up to the FP32 prefilter round trip; 16-bit storage refuses it."""
    torch, claire = env
    n = (16, 12, 20)
    rng = np.random.default_rng(0)
    f = f32(rng.standard_normal(n))
    d = np.zeros((3,) + n, np.float32)
    d[0] = 5; d[1] = -13; d[2] = 21
    ctx = make_ctx(claire, torch, n, interp=4)
    out = torch.empty(n, device="cuda")
    ctx.interp(dev(torch, f), dev(torch, d), out, 4)
    torch.cuda.synchronize()
    assert rel_linf(host(out), np.roll(f, (-5, 13, -21), axis=(0, 1, 2)).astype(np.float64)) <= 1e-5
    with pytest.raises(claire.ClaireError):
        make_ctx(claire, torch, n, interp=4, storage=claire.STORAGE_F16)


def test_bspline_gradient_matvec_parity(env):
    torch, claire = env
    n = (32, 32, 32)
    m0, m1, vs, v, p = _problem(n)
    p.order = 4
    m1 = f32(oracle.transport(m0.astype(np.float64), vs.astype(np.float64), p))
    ctx = make_ctx(claire, torch, n, beta_v=p.beta_v, nt=p.nt, beta_w=p.beta_w, interp=4)
    ctx.set_images(dev(torch, m0), dev(torch, m1))
    g = torch.empty((3,) + n, device="cuda")
    J = ctx.gradient(dev(torch, v), g)
    st = oracle.State(v.astype(np.float64), m0.astype(np.float64), m1.astype(np.float64), p)
    assert abs(J - st.J) <= 1e-5 * abs(st.J)
    assert rel_l2(host(g), oracle.gradient(st)) <= 1e-4
    vt = f32(synth.mode_velocity(n, seed=33, vmax=0.3))
    Hv = torch.empty((3,) + n, device="cuda")
    ctx.hessian_matvec(dev(torch, vt), Hv)
    torch.cuda.synchronize()
    assert rel_l2(host(Hv), oracle.hessian_matvec(st, vt.astype(np.float64))) <= 1e-4
    lo, hi = ctx.detj(dev(torch, vs))
    ref = oracle.detj(vs.astype(np.float64), p)
    assert abs(lo - ref.min()) <= 1e-4 * abs(ref.min()) and abs(hi - ref.max()) <= 1e-4 * abs(ref.max())


@pytest.mark.parametrize("n", SHAPES)
@pytest.mark.parametrize("direction", [1, -1])
def test_backtrace_parity(env, n, direction):
    torch, claire = env
    v = f32(synth.mode_velocity(n, seed=4, vmax=1.0))
    for order in (3, 1, 4):
        ctx = make_ctx(claire, torch, n, nt=4, interp=order)
        d = torch.empty((3,) + n, device="cuda")
        ctx.backtrace(dev(torch, v), d, direction)
        torch.cuda.synchronize()
        ref = oracle.backtrace(v.astype(np.float64), 0.25, direction, order)
        assert rel_linf(host(d), ref) <= 1e-5


@pytest.mark.parametrize("n", SHAPES)
def test_fd8_parity(env, n):
    torch, claire = env
    f = f32(synth.blob_template(n, seed=5))
    v = f32(synth.mode_velocity(n, seed=6, vmax=1.0))
    ctx = make_ctx(claire, torch, n)
    g = torch.empty((3,) + n, device="cuda")
    dv = torch.empty(n, device="cuda")
    ctx.fd8_grad(dev(torch, f), g)
    ctx.fd8_div(dev(torch, v), dv)
    torch.cuda.synchronize()
    assert rel_linf(host(g), oracle.fd8_grad(f.astype(np.float64))) <= 1e-5
    assert rel_linf(host(dv), oracle.fd8_div(v.astype(np.float64))) <= 1e-5


@pytest.mark.parametrize("n", [(20, 8, 32), (36, 24, 96), (64, 16, 64)])
def test_fd8_grad_tiled_parity(env, n):
    """Grids whose (x2, x3) planes the 8 x 32 tiles cover take the tiled FD8
    gradient (halo planes in shared memory, x1 values in a register queue):
    x1 extents that leave a partial 16-plane slab, x2 = 8 (the halo wraps onto
    the tile itself) and several tiles per plane, against the oracle."""
    torch, claire = env
    f = f32(synth.blob_template(n, seed=15))
    ctx = make_ctx(claire, torch, n)
    g = torch.empty((3,) + n, device="cuda")
    ctx.fd8_grad(dev(torch, f), g)
    torch.cuda.synchronize()
    ref = oracle.fd8_grad(f.astype(np.float64))
    assert rel_linf(host(g), ref) <= 1e-5
    for c in range(3):
        assert rel_linf(host(g)[c], ref[c]) <= 1e-5


@pytest.mark.parametrize("n", SHAPES)
@pytest.mark.parametrize("reg", [1, 2])
def test_spectral_parity(env, n, reg):
    torch, claire = env
    rng = np.random.default_rng(7)
    x = f32(rng.standard_normal((3,) + n))
    p = oracle.Params(beta_v=3e-2, beta_w=2e-3, reg=reg)
    ctx = make_ctx(claire, torch, n, beta_v=p.beta_v, beta_w=p.beta_w, reg=reg)
    xd = dev(torch, x)
    x64 = x.astype(np.float64)
    for op, ref in ((claire.SPECTRAL_REG, oracle.reg_apply(x64, p)),
                    (claire.SPECTRAL_INV, oracle.reg_inverse(x64, p)),
                    (claire.SPECTRAL_K, oracle.project_K(x64, p))):
        out = torch.empty((3,) + n, device="cuda")
        ctx.spectral(xd, out, op)
        torch.cuda.synchronize()
        assert rel_l2(host(out), ref) <= 1e-5, op


def test_dot_parity(env):
    torch, claire = env
    n = (40, 36, 30)
    rng = np.random.default_rng(8)
    x = f32(rng.standard_normal(3 * int(np.prod(n))))
    y = f32(rng.standard_normal(3 * int(np.prod(n))))
    ctx = make_ctx(claire, torch, n)
    hv = float(np.prod(oracle.spacing(n)))
    ref = hv * float(np.dot(x.astype(np.float64), y.astype(np.float64)))
    got = ctx.dot(dev(torch, x), dev(torch, y))
    assert abs(got - ref) <= 1e-6 * hv * float(np.dot(np.abs(x), np.abs(y)))
    # misaligned start and odd length take the scalar path
    got2 = ctx.dot(dev(torch, x)[1:], dev(torch, y)[1:], x.size - 3)
    ref2 = hv * float(np.dot(x[1:-2].astype(np.float64), y[1:-2].astype(np.float64)))
    assert abs(got2 - ref2) <= 1e-6 * hv * float(np.dot(np.abs(x), np.abs(y)))


# ---------------------------------------------------------------------------
# solves and operators
# ---------------------------------------------------------------------------

def _problem(n, nt=4, seed=0, scale=0.5):
    m0 = f32(synth.blob_template(n, seed=seed))
    vs = f32(synth.mode_velocity(n, seed=seed + 10, vmax=0.5))
    p = oracle.Params(nt=nt, beta_v=1e-2, beta_w=1e-4)
    m1 = f32(oracle.transport(m0.astype(np.float64), vs.astype(np.float64), p))
    v = f32(scale * vs)
    return m0, m1, vs, v, p


@pytest.mark.parametrize("n", SHAPES)
@pytest.mark.parametrize("order", [3, 1, 4])
def test_transport_parity(env, n, order):
    torch, claire = env
    m0, _, vs, _, p = _problem(n)
    p.order = order
    ctx = make_ctx(claire, torch, n, nt=p.nt, interp=order)
    out = torch.empty(n, device="cuda")
    ctx.transport(dev(torch, vs), dev(torch, m0), out, claire.TRANSPORT_FWD)
    torch.cuda.synchronize()
    ref = oracle.transport(m0.astype(np.float64), vs.astype(np.float64), p)
    assert rel_l2(host(out), ref) <= 2e-4
    lam1 = f32(synth.blob_template(n, seed=9))
    ctx.transport(dev(torch, vs), dev(torch, lam1), out, claire.TRANSPORT_ADJ)
    torch.cuda.synchronize()
    ref = oracle.transport(lam1.astype(np.float64), vs.astype(np.float64), p, direction="adj")
    assert rel_l2(host(out), ref) <= 2e-4


@pytest.mark.parametrize("n", SHAPES)
@pytest.mark.parametrize("grad_form", [0, 1])
@pytest.mark.parametrize("lowmem", [0, 1])
def test_gradient_matvec_precond_parity(env, n, grad_form, lowmem):
    """lowmem = 1: the state gradients are computed by FD8 where they are used."""
    torch, claire = env
    m0, m1, vs, v, p = _problem(n)
    p.grad_form = grad_form
    ctx = make_ctx(claire, torch, n, beta_v=p.beta_v, nt=p.nt, beta_w=p.beta_w, grad_form=grad_form,
                   lowmem=lowmem)
    ctx.set_images(dev(torch, m0), dev(torch, m1))
    g = torch.empty((3,) + n, device="cuda")
    J = ctx.gradient(dev(torch, v), g)
    st = oracle.State(v.astype(np.float64), m0.astype(np.float64), m1.astype(np.float64), p)
    assert abs(J - st.J) <= 1e-5 * abs(st.J)
    vt = f32(synth.mode_velocity(n, seed=33, vmax=0.3))
    Hv = torch.empty((3,) + n, device="cuda")
    ctx.hessian_matvec(dev(torch, vt), Hv)
    torch.cuda.synchronize()
    g_ref, h_ref = oracle.gradient(st), oracle.hessian_matvec(st, vt.astype(np.float64))
    if grad_form == 0:
        # split S x + body: the body at 1e-4, S x within the FP32 transform bound
        sx = torch.empty((3,) + n, device="cuda")
        ctx.spectral(dev(torch, v), sx, claire.SPECTRAL_REG)
        torch.cuda.synchronize()
        split_check(host(g), host(sx), g_ref, st.reg_v, fft_roundoff_bound(n, p, v))
        ctx.spectral(dev(torch, vt), sx, claire.SPECTRAL_REG)
        torch.cuda.synchronize()
        split_check(host(Hv), host(sx), h_ref, oracle.reg_apply(vt.astype(np.float64), p),
                    fft_roundoff_bound(n, p, vt))
    else:
        # K (a contraction) of S x + body: 1e-4 of the result plus the transform bound
        for got, ref, x in ((host(g), g_ref, v), (host(Hv), h_ref, vt)):
            err = float(np.linalg.norm(got - ref))
            assert err <= 1e-4 * float(np.linalg.norm(ref)) + 2.0 * fft_roundoff_bound(n, p, x)
    z = torch.empty((3,) + n, device="cuda")
    ctx.precond(g, z)
    torch.cuda.synchronize()
    assert rel_l2(host(z), oracle.precond(host(g), p)) <= 1e-5
    Jo, mis = ctx.objective(dev(torch, v))
    assert abs(Jo - st.J) <= 1e-5 * abs(st.J) and abs(mis - st.mismatch) <= 1e-5 * st.mismatch


@pytest.mark.parametrize("order,storage", [(3, 0), (1, 0), (4, 0), (3, 1)])
def test_tile_bounds_table_path(env, order, storage):
    """On grids the tiles cover exactly, the gathers at the context's own
    characteristics take their boxes from the tile-bounds table that the
    backtrace wrote with them.  The states they produce are bit-identical to
    those of the in-kernel bounds path (the objective at the same velocity
    gathers at a scratch characteristic), and no tile leaves the box path
    (a point outside its table box would send the tile to global memory)."""
    torch, claire = env
    n = (64, 64, 64)
    m0, m1, vs, v, p = _problem(n)
    ctx = make_ctx(claire, torch, n, beta_v=p.beta_v, nt=p.nt, beta_w=p.beta_w, interp=order, storage=storage)
    ctx.set_images(dev(torch, m0), dev(torch, m1))
    claire.claire_gather_fallback_tiles(reset=True)
    g = torch.empty((3,) + n, device="cuda")
    J = ctx.gradient(dev(torch, v), g)
    vt = f32(synth.mode_velocity(n, seed=33, vmax=0.3))
    Hv = torch.empty((3,) + n, device="cuda")
    ctx.hessian_matvec(dev(torch, vt), Hv)
    torch.cuda.synchronize()
    assert claire.claire_gather_fallback_tiles(reset=True) == 0
    Jo, _ = ctx.objective(dev(torch, v))
    assert Jo == J
    assert np.all(np.isfinite(host(Hv)))


def test_gradient_nt1_linear_h2(env):
    """Degenerate and alternative settings: one time step, trilinear, H2."""
    torch, claire = env
    n = (16, 16, 16)
    m0, m1, vs, v, p = _problem(n, nt=1)
    p.order, p.reg = 1, 2
    ctx = make_ctx(claire, torch, n, beta_v=p.beta_v, nt=1, beta_w=p.beta_w, interp=1, reg=2)
    ctx.set_images(dev(torch, m0), dev(torch, m1))
    g = torch.empty((3,) + n, device="cuda")
    ctx.gradient(dev(torch, v), g)
    st = oracle.State(v.astype(np.float64), m0.astype(np.float64), m1.astype(np.float64), p)
    assert rel_l2(host(g), oracle.gradient(st)) <= 1e-4
    Hv = torch.empty((3,) + n, device="cuda")
    ctx.hessian_matvec(dev(torch, vs), Hv)
    torch.cuda.synchronize()
    assert rel_l2(host(Hv), oracle.hessian_matvec(st, vs.astype(np.float64))) <= 1e-4


@pytest.mark.parametrize("n", [(32, 32, 32), (40, 36, 30)])
def test_detj_parity(env, n):
    torch, claire = env
    vs = f32(synth.mode_velocity(n, seed=12, vmax=0.8))
    p = oracle.Params(nt=4)
    ctx = make_ctx(claire, torch, n, nt=4)
    lo, hi = ctx.detj(dev(torch, vs))
    ref = oracle.detj(vs.astype(np.float64), p)
    assert abs(lo - ref.min()) <= 1e-5 * abs(ref.min()) and abs(hi - ref.max()) <= 1e-5 * ref.max()
    assert ref.min() < 0.9 and ref.max() > 1.1  # a non-trivial map


def test_state_errors_and_failure_detection(env):
    torch, claire = env
    n = (16, 16, 16)
    m0, m1, vs, v, p = _problem(n)
    ctx = make_ctx(claire, torch, n)
    out = torch.empty((3,) + n, device="cuda")
    with pytest.raises(claire.ClaireError) as e:
        ctx.gradient(dev(torch, v), out)
    assert e.value.status == -8  # images not set
    ctx.set_images(dev(torch, m0), dev(torch, m1))
    with pytest.raises(claire.ClaireError) as e:
        ctx.hessian_matvec(dev(torch, v), out)
    assert e.value.status == -8  # no linearisation point
    bad = m1.copy()
    bad[3, 4, 5] = np.nan  # failure made on the host: a NaN in the reference image
    ctx.set_images(dev(torch, m0), dev(torch, bad))
    with pytest.raises(claire.ClaireError) as e:
        ctx.gradient(dev(torch, v), out)
    assert e.value.status == -5
    with pytest.raises(claire.ClaireError) as e:
        ctx.interp(np.zeros(n, np.float32), dev(torch, v), out[0])
    assert e.value.status == -1  # kernel-level entry points reject host pointers


def test_nonfinite_velocity_screened_before_any_gather(env):
    """A NaN or Inf in the velocity is rejected (CLAIRE_ENONFINITE) by the FP64
    max-norm screen before any backtrace or SL gather is launched (failure made
    on the host: the bad value is planted in the input array)."""
    torch, claire = env
    n = (16, 16, 16)
    m0, m1, vs, v, p = _problem(n)
    ctx = make_ctx(claire, torch, n)
    ctx.set_images(dev(torch, m0), dev(torch, m1))
    gathers = ("sl_interp", "sl_backtrace_rk2", "sl_adjoint_step", "sl_incremental_step",
               "sl_incremental_last", "sl_map_step")

    def launched():
        return {k["name"]: k["launches"] for k in ctx.kernel_stats() if k["name"] in gathers}

    out = torch.empty((3,) + n, device="cuda")
    for bad_value in (np.nan, np.inf, -np.inf):
        bad = v.copy()
        bad[1, 5, 6, 7] = bad_value
        before = launched()
        for call in (lambda: ctx.register(dev(torch, bad)),
                     lambda: ctx.gradient(dev(torch, bad), out),
                     lambda: ctx.objective(dev(torch, bad)),
                     lambda: ctx.transport(dev(torch, bad), dev(torch, m0), out[0]),
                     lambda: ctx.transport_vjp(dev(torch, bad), dev(torch, m0), dev(torch, m1), gm0=out[0]),
                     lambda: ctx.detj(dev(torch, bad)),
                     lambda: ctx.backtrace(dev(torch, bad), out, 1)):
            with pytest.raises(claire.ClaireError) as e:
                call()
            assert e.value.status == -5
        assert launched() == before
    # the context stays usable
    st, rep = ctx.register(torch.zeros((3,) + n, device="cuda"), check=False)
    assert st >= 0 and math.isfinite(rep["J"])


def test_misaligned_device_arrays(env):
    """Device arrays that start 4 bytes past a 16-byte boundary (a tensor view
    offset by one float): the tiled gathers stage such a field's box with
    4-byte copies instead of 16-byte chunks, the vector kernels take their
    scalar loops, so every call gives the bits of the aligned call;
    claire_resample, which hands its arrays to cuFFT, rejects them."""
    torch, claire = env
    n = (32, 32, 32)
    N = int(np.prod(n))
    m0, m1, vs, v, p = _problem(n)
    ctx = make_ctx(claire, torch, n)
    ctx.set_images(dev(torch, m0), dev(torch, m1))

    def shifted(a):
        buf = torch.zeros(a.numel() + 4, device="cuda")
        t = buf[1:1 + a.numel()].view(a.shape)
        t.copy_(a)
        assert t.data_ptr() % 16 == 4
        return t

    d = dev(torch, _disp(n, 3, 1.5))
    f = dev(torch, m0)
    f2 = torch.stack([f, dev(torch, m1)]).contiguous()
    vd = dev(torch, v)
    out_a, out_b = torch.empty(n, device="cuda"), shifted(torch.empty(n, device="cuda"))
    ctx.interp(f, d, out_a)
    ctx.interp(shifted(f), shifted(d), out_b)
    assert torch.equal(out_a, out_b)
    o2a, o2b = torch.empty_like(f2), torch.empty_like(f2)
    ctx.interp_fields(f2, 2, d, o2a)
    ctx.interp_fields(shifted(f2), 2, d, o2b)
    assert torch.equal(o2a, o2b)
    da, db = torch.empty((3,) + n, device="cuda"), torch.empty((3,) + n, device="cuda")
    ctx.backtrace(vd, da, 1)
    ctx.backtrace(shifted(vd), db, 1)
    assert torch.equal(da, db)
    # solver level: the arrays are used in place
    g_a, g_b = torch.empty((3,) + n, device="cuda"), torch.empty((3,) + n, device="cuda")
    J_a = ctx.gradient(vd, g_a)
    J_b = ctx.gradient(shifted(vd), shifted(g_b))
    assert J_a == J_b
    ctx.gradient(shifted(vd), g_b)
    assert torch.equal(g_a, g_b)
    ctx.transport(vd, f, out_a)
    ctx.transport(shifted(vd), shifted(f), out_b)
    assert torch.equal(out_a, out_b)
    with pytest.raises(claire.ClaireError) as e:
        claire.claire_resample(shifted(f), n, out_a, n)
    assert e.value.status == -1


def test_wall_clock_limit(env):
    torch, claire = env
    n = (32, 32, 32)
    m0, m1, vs, v, p = _problem(n)
    ctx = make_ctx(claire, torch, n, gtol=1e-9, wall_limit_s=1e-6, max_gn=20)
    ctx.set_images(dev(torch, m0), dev(torch, m1))
    vv = torch.zeros((3,) + n, device="cuda")
    with pytest.raises(claire.ClaireError) as e:
        ctx.register(vv)
    assert e.value.status == -7


# ---------------------------------------------------------------------------
# registration (Eq. (5)): 64^3 blob workload, 5 Gauss-Newton x 10 PCG
# ---------------------------------------------------------------------------

def _config1():
    n = (64, 64, 64)
    m0 = f32(synth.blob_template(n, seed=0))
    vs = synth.mode_velocity(n, seed=0, nmodes=6, kmax=4, vmax=0.5)
    p = oracle.Params(nt=4, beta_v=1e-2, beta_w=1e-4, gtol=0.0, max_gn=5, max_pcg=10,
                      pcg_fixed=True)
    m1 = f32(oracle.transport(m0.astype(np.float64), vs, p))
    return n, m0, m1, p


@pytest.fixture(scope="module")
def config1_oracle():
    n, m0, m1, p = _config1()
    v, rep = oracle.register(m0.astype(np.float64), m1.astype(np.float64), p)
    return n, m0, m1, p, v, rep


def test_registration_fixed_schedule_parity(env, config1_oracle):
    torch, claire = env
    n, m0, m1, p, v_ref, rep_ref = config1_oracle
    ctx = make_ctx(claire, torch, n, beta_v=p.beta_v, nt=p.nt, beta_w=p.beta_w, gtol=0.0,
                   max_gn=5, max_pcg=10, pcg_fixed=1)
    ctx.set_images(dev(torch, m0), dev(torch, m1))
    v = torch.zeros((3,) + n, device="cuda")
    st, rep = ctx.register(v)
    assert rep["gn_iters"] == rep_ref["gn_iters"] == 5
    assert rep["alpha"] == rep_ref["alpha"]
    assert rel_l2(host(v), v_ref) <= 1e-3
    assert abs(rep["r"] - rep_ref["r"]) <= 0.01 * rep_ref["r"]
    # the reported CFL of the returned velocity is the oracle's definition
    # (max |v(x)|_2 dt / min h) on the same FP32 values; the GPU takes h in FP32
    c_ref = oracle.cfl(host(v), p)
    assert abs(rep["cfl"] - c_ref) <= 1e-6 * c_ref


def test_registration_free_running_and_host_pointers(env):
    """gtol 5e-2 with the default forcing: same final mismatch within 1 %;
    the host-pointer call gives the same result as the device call."""
    torch, claire = env
    n, m0, m1, p = _config1()
    p.gtol, p.pcg_fixed, p.max_gn = 5e-2, False, 20
    v_ref, rep_ref = oracle.register(m0.astype(np.float64), m1.astype(np.float64), p)
    ctx = make_ctx(claire, torch, n, beta_v=p.beta_v, nt=p.nt, beta_w=p.beta_w, gtol=p.gtol,
                   max_gn=20, max_pcg=10)
    ctx.set_images(m0, m1)  # host arrays
    v_host = np.zeros((3,) + n, np.float32)
    st, rep = ctx.register(v_host)
    assert st == 0 and rep["gnorm_rel"] <= 5e-2
    assert abs(rep["r"] - rep_ref["r"]) <= 0.01 * rep_ref["r"]
    ctx.set_images(dev(torch, m0), dev(torch, m1))
    v_dev = torch.zeros((3,) + n, device="cuda")
    st2, rep2 = ctx.register(v_dev)
    assert np.array_equal(v_dev.cpu().numpy(), v_host)
    assert rep2["gn_iters"] == rep["gn_iters"]


# ---------------------------------------------------------------------------
# full size (256^3): sampled points and size-independent properties
# ---------------------------------------------------------------------------

def test_full_size_interp_sampled(env):
    torch, claire = env
    n = (256, 256, 256)
    m0 = f32(synth.label_template(n, seed=0))
    vs = synth.bandlimited_velocity(n, seed=0, kmax=8, vmax=1.0)
    ctx = make_ctx(claire, torch, n, nt=4)
    d = torch.empty((3,) + n, device="cuda")
    ctx.backtrace(dev(torch, vs), d, 1)
    out = torch.empty(n, device="cuda")
    f = dev(torch, m0)
    ctx.interp(f, d, out, 3)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    idx = rng.integers(0, m0.size, size=20000)
    dh = d.reshape(3, -1)[:, torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.float64)
    I, J, K = np.unravel_index(idx, n)
    y = np.stack([I + dh[0], J + dh[1], K + dh[2]])
    ref = oracle.interp_points(m0.astype(np.float64), y, 3)
    got = out.reshape(-1)[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(m0))
    # sampled backtrace: X = x - dt/2 (v(x) + v(x - dt v(x))) from the FP32 velocity
    h = oracle.spacing(n)
    v32 = f32(vs)
    u = np.stack([v32[c].reshape(-1)[idx].astype(np.float64) / h[c] for c in range(3)])
    ys = np.stack([I - 0.25 * u[0], J - 0.25 * u[1], K - 0.25 * u[2]])
    us = np.stack([oracle.interp_points(v32[c].astype(np.float64), ys, 3) / h[c] for c in range(3)])
    dref = -0.125 * (u + us)
    assert np.max(np.abs(dh - dref)) <= 1e-5 * np.max(np.abs(dref))


def test_full_size_transport_integer_shift_exact(env):
    """Constant velocity moving dt v / h = (1, -2, 3) cells per step: the 256^3
    transport is an exact periodic roll (interpolation weights are 0/1)."""
    torch, claire = env
    n = (256, 256, 256)
    m0 = f32(synth.label_template(n, seed=1))
    h = oracle.spacing(n)
    shift = (1, -2, 3)
    v = np.stack([np.full(n, s * h[c] * 4, np.float32) for c, s in enumerate(shift)])
    ctx = make_ctx(claire, torch, n, nt=4)
    out = torch.empty(n, device="cuda")
    ctx.transport(dev(torch, v), dev(torch, m0), out, claire.TRANSPORT_FWD)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), np.roll(m0, (4, -8, 12), axis=(0, 1, 2)))
