"""GPU regularisation-parameter search and continuation (Sec. 3) against the
FP64 oracle's schedule on the same FP32 images: the same sequence of
(beta_v, beta_w, valid) decisions and the same selected weights, except
where the oracle's Jacobian extremes lie within 2 % of a bound (there FP32
and FP64 may legitimately decide differently)."""
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


def problem():
    n = (16, 16, 16)
    m0 = synth.blob_template(n, seed=3, sigma=0.6).astype(np.float32)
    vs = synth.mode_velocity(n, seed=4, kmax=2, vmax=1.2)
    p = oracle.Params(nt=4, beta_v=1e-2, beta_w=1e-4, gtol=5e-2, max_gn=10, max_pcg=10)
    m1 = oracle.transport(m0.astype(np.float64), vs, p).astype(np.float32)
    return n, m0, m1, p


def test_param_search_matches_oracle(env):
    torch, claire = env
    n, m0, m1, p = problem()
    ctx = claire.Context(n, 1.0, 4, stream=torch.cuda.current_stream().cuda_stream, gtol=5e-2, max_gn=10,
                         max_pcg=10)
    ctx.set_images(torch.from_numpy(m0).cuda(), torch.from_numpy(m1).cuda())
    v = torch.zeros((3,) + n, device="cuda")
    st, rep = ctx.param_search(v, jmin=0.5, max_solves=20)
    bv_o, bw_o, v_o, trace_o = oracle.param_search(m0.astype(np.float64), m1.astype(np.float64), p, jmin=0.5,
                                                   max_solves=20)
    print("GPU:", [(t["beta_v"], t["beta_w"], t["valid"]) for t in rep["trace"]], rep["beta_v"], rep["beta_w"])
    print("oracle:", trace_o, bv_o, bw_o)
    gpu = [(t["beta_v"], t["beta_w"], t["valid"]) for t in rep["trace"]]
    for (gb, gw, gok), (ob, ow, ook) in zip(gpu, trace_o):
        assert abs(gb - ob) <= 1e-12 * ob and abs(gw - ow) <= 1e-12 * max(ow, 1e-30)
        if gok != bool(ook):
            q = oracle.Params(**{**p.__dict__, "beta_v": ob, "beta_w": ow})
            vv, _ = oracle.register(m0.astype(np.float64), m1.astype(np.float64), q)
            dj = oracle.detj(vv, q)
            margin = min(abs(dj.min() - 0.5) / 0.5, abs(dj.max() - 2.0) / 2.0)
            assert margin < 0.02, "decision differs away from a bound"
            return
    assert len(gpu) == len(trace_o)
    assert abs(rep["beta_v"] - bv_o) <= 1e-12 * bv_o and abs(rep["beta_w"] - bw_o) <= 1e-12 * bw_o
    assert claire.claire_get_beta(ctx.handle) == pytest.approx((bv_o, bw_o), rel=1e-12)
    vg = v.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(vg - v_o) <= 1e-2 * np.linalg.norm(v_o)


def test_param_continuation(env):
    torch, claire = env
    n, m0, m1, p = problem()
    ctx = claire.Context(n, 1.0, 4, stream=torch.cuda.current_stream().cuda_stream, gtol=5e-2, max_gn=10,
                         max_pcg=10)
    ctx.set_images(torch.from_numpy(m0).cuda(), torch.from_numpy(m1).cuda())
    v = torch.zeros((3,) + n, device="cuda")
    st, rep = ctx.param_continuation(v, 0.03, 1e-7)
    steps = [(round(t["beta_v"], 12), round(t["beta_w"], 14)) for t in rep["trace"]]
    assert steps == [(1.0, 1e-5), (0.1, 1e-5), (0.03, 1e-5), (0.03, 1e-6), (0.03, 1e-7)]
    v_o, _ = oracle.param_continuation(m0.astype(np.float64), m1.astype(np.float64), p, 0.03, 1e-7)
    vg = v.cpu().numpy().astype(np.float64)
    err = np.linalg.norm(vg - v_o) / np.linalg.norm(v_o)
    print("continuation velocity rel L2 vs oracle %.2e" % err)
    assert err <= 1e-2
    with pytest.raises(claire.ClaireError):
        ctx.param_search(v, jmin=2.0)
