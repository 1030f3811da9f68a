"""Mixed precision (FP16 / BF16 storage of the scalar fields, FP32 arithmetic,
FP64 reductions) against the FP64 oracle.

Tolerances scale with the unit roundoff u of the storage type (2^-11 for
FP16, 2^-8 for BF16): every stored field (images, states m^j, their
gradients, adjoint levels, incremental fields, div v) adds a relative
rounding of u, and the adjoint's final condition m1 - m(1) amplifies it by
|m| / |m - m1| <= 10 on these inputs; 20 u bounds the gradient and the
Hessian matvec, and the Gauss-Newton iterate inherits it.
"""
import numpy as np
import pytest

import __graft_entry__ as entry
import oracle
from paper_2209_08189_gb300 import synth

pytestmark = pytest.mark.gpu
UNIT = {1: 2.0 ** -11, 2: 2.0 ** -8}


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
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _problem(n, seed=0):
    m0 = f32(synth.blob_template(n, seed=seed))
    vs = f32(synth.mode_velocity(n, seed=seed + 10, vmax=0.5))
    p = oracle.Params(nt=4, beta_v=1e-2, beta_w=1e-4)
    m1 = f32(oracle.transport(m0.astype(np.float64), vs.astype(np.float64), p))
    return m0, m1, vs, p


@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("n", [(32, 32, 32), (40, 36, 30)])
def test_mixed_gradient_and_matvec(env, storage, n):
    torch, claire = env
    m0, m1, vs, p = _problem(n)
    v = f32(0.5 * vs)
    ctx = claire.Context(n, p.beta_v, p.nt, beta_w=p.beta_w, storage=storage,
                         stream=torch.cuda.current_stream().cuda_stream)
    ctx.set_images(m0, m1)
    g = torch.empty((3,) + n, device="cuda")
    J = ctx.gradient(torch.from_numpy(v).cuda(), g)
    st = oracle.State(v.astype(np.float64), m0.astype(np.float64), m1.astype(np.float64), p)
    u = UNIT[storage]
    eg = rel_l2(g.cpu().numpy().astype(np.float64), oracle.gradient(st))
    assert eg <= 20 * u, eg
    assert abs(J - st.J) <= 20 * u * abs(st.J)
    vt = f32(synth.mode_velocity(n, seed=33, vmax=0.3))
    Hv = torch.empty((3,) + n, device="cuda")
    ctx.hessian_matvec(torch.from_numpy(vt).cuda(), Hv)
    torch.cuda.synchronize()
    eh = rel_l2(Hv.cpu().numpy().astype(np.float64), oracle.hessian_matvec(st, vt.astype(np.float64)))
    assert eh <= 20 * u, eh
    print("storage %d grid %s: gradient rel L2 %.2e, matvec rel L2 %.2e" % (storage, n, eg, eh))


@pytest.mark.parametrize("storage", [1, 2])
def test_mixed_registration_errors_vs_oracle(env, storage):
    """64^3 blob workload, 5 GN x 10 PCG (fixed schedule): final velocity,
    relative residual and det grad y against the FP64 oracle."""
    torch, claire = env
    n = (64, 64, 64)
    m0 = f32(synth.blob_template(n, seed=0))
    vs = synth.mode_velocity(n, seed=0, nmodes=6, kmax=4, vmax=0.5)
    p = oracle.Params(nt=4, beta_v=1e-2, beta_w=1e-4, gtol=0.0, max_gn=5, max_pcg=10, pcg_fixed=True)
    m1 = f32(oracle.transport(m0.astype(np.float64), vs, p))
    v_ref, rep_ref = oracle.register(m0.astype(np.float64), m1.astype(np.float64), p)
    ctx = claire.Context(n, p.beta_v, p.nt, beta_w=p.beta_w, gtol=0.0, max_gn=5, max_pcg=10, pcg_fixed=1,
                         storage=storage, stream=torch.cuda.current_stream().cuda_stream)
    ctx.set_images(m0, m1)
    v = torch.zeros((3,) + n, device="cuda")
    st, rep = ctx.register(v)
    u = UNIT[storage]
    ev = rel_l2(v.cpu().numpy().astype(np.float64), v_ref)
    er = abs(rep["r"] - rep_ref["r"]) / rep_ref["r"]
    dj = oracle.detj(v_ref, p)
    ej = max(abs(rep["detj_min"] - dj.min()) / dj.min(), abs(rep["detj_max"] - dj.max()) / dj.max())
    print("storage %d: v rel L2 %.2e, r rel %.2e, detJ rel %.2e" % (storage, ev, er, ej))
    assert ev <= 40 * u and er <= 40 * u and ej <= 40 * u
