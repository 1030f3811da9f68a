"""claire_dot_noalloc: the inner product for callers that cannot allocate
device memory (a process whose device memory another allocator has fully
reserved, a loop that cannot take cudaMalloc's device-wide synchronisation,
or code without a claire context).  Its output must match claire_dot's on
the same inputs, on consecutive calls that reuse the shared static scratch,
and an FP64 sum on the host within the rounding of its FP32 products.

This file sorts last so that a run stopping at the first failure has already
run every other test.
"""
import numpy as np
import pytest

import __graft_entry__ as entry
import oracle

# x_i y_i is formed in FP32 and summed in groups of four in FP32 before the FP64
# accumulation: at most 4 roundings of 2^-24 relative to sum |x_i y_i|.
FP32_GROUP_BOUND = 4 * 2.0 ** -24
K_CHUNK = 256 * 32  # elements per partial sum of the kernel


def test_noalloc_rejects_oversized_input_before_any_launch():
    entry.build()
    from paper_2209_08189_gb300 import claire
    with pytest.raises(claire.ClaireError) as e:
        claire.claire_dot_noalloc(0, 0, (1 << 30) + 1, 1.0)
    assert e.value.status == -10  # CLAIRE_ETOOLARGE


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    entry.build()
    from paper_2209_08189_gb300 import claire
    return torch, claire


@pytest.mark.gpu
def test_noalloc_dot_matches_claire_dot_and_host_fp64_sum():
    torch, claire = _cuda()
    n = (40, 36, 30)
    hv = float(np.prod(oracle.spacing(n)))
    ctx = claire.Context(n, 1e-2, 4, stream=torch.cuda.current_stream().cuda_stream)
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(21)
    # calls in a row on the shared scratch: long, shorter with a ragged tail,
    # one element past a partial-sum boundary, and many partial sums plus a tail
    sizes = (3 * int(np.prod(n)), int(np.prod(n)) - 7, 40 * K_CHUNK + 1, (1 << 24) + K_CHUNK + 3)
    for size in sizes:
        xh = rng.standard_normal(size).astype(np.float32)
        yh = rng.standard_normal(size).astype(np.float32)
        x = torch.from_numpy(xh).cuda()
        y = torch.from_numpy(yh).cuda()
        st, got = claire.claire_dot_noalloc(x, y, size, hv, stream)
        assert st == 0
        prod = xh.astype(np.float64) * yh.astype(np.float64)
        exact = hv * float(np.sum(prod))
        bound = FP32_GROUP_BOUND * hv * float(np.sum(np.abs(prod))) + 1e-12 * abs(exact)
        assert abs(got - exact) <= bound, (size, got, exact, bound)
        if size <= 3 * int(np.prod(n)):
            ref = ctx.dot(x, y, size)
            assert abs(got - ref) <= 2 * bound
    ctx.close()


@pytest.mark.gpu
def test_noalloc_dot_at_the_size_limit_exact():
    """n = 2^30, the largest accepted size (all 2^17 partial-sum slots), on
    periodic small-integer inputs: every product and group sum is exact in FP32
    and the FP64 accumulation is exact, so the result equals the closed form."""
    torch, claire = _cuda()
    n = 1 << 30
    stream = torch.cuda.current_stream().cuda_stream
    i = torch.arange(n, device="cuda", dtype=torch.int64)
    x = ((i % 7) - 3).to(torch.float32)
    y = ((i % 5) - 2).to(torch.float32)
    del i
    # sum over one period of 35 and the remainder, in Python integers
    per = sum(((k % 7) - 3) * ((k % 5) - 2) for k in range(35))
    rem = sum(((k % 7) - 3) * ((k % 5) - 2) for k in range(n - (n // 35) * 35))
    exact = per * (n // 35) + rem
    for _ in range(2):
        st, got = claire.claire_dot_noalloc(x, y, n, 1.0, stream)
        assert st == 0 and got == float(exact)
