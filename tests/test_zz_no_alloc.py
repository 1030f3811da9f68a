"""claire_dot_noalloc: the inner product for callers that cannot allocate
device memory (a process whose device memory another allocator has fully
reserved, a loop that cannot take cudaMalloc's device-wide synchronisation,
or code without a claire context).  Its output must match claire_dot's on
the same inputs, on consecutive calls that reuse the shared static scratch.

This file sorts last so that a run stopping at the first failure has already
run every other test.
"""
import numpy as np
import pytest

import __graft_entry__ as entry
import oracle


def test_noalloc_rejects_oversized_input_before_any_launch():
    entry.build()
    from paper_2209_08189_gb300 import claire
    with pytest.raises(claire.ClaireError) as e:
        claire.claire_dot_noalloc(0, 0, (1 << 30) + 1, 1.0)
    assert e.value.status == -10  # CLAIRE_ETOOLARGE


@pytest.mark.gpu
def test_noalloc_dot_matches_claire_dot_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    entry.build()
    from paper_2209_08189_gb300 import claire
    n = (40, 36, 30)
    hv = float(np.prod(oracle.spacing(n)))
    ctx = claire.Context(n, 1e-2, 4, stream=torch.cuda.current_stream().cuda_stream)
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(21)
    sizes = (3 * int(np.prod(n)), int(np.prod(n)) - 7)  # second call: shorter, ragged tail
    for size in sizes:
        x = torch.from_numpy(rng.standard_normal(size).astype(np.float32)).cuda()
        y = torch.from_numpy(rng.standard_normal(size).astype(np.float32)).cuda()
        ref = ctx.dot(x, y, size)
        st, got = claire.claire_dot_noalloc(x, y, size, hv, stream)
        assert st == 0
        scale = hv * float(torch.dot(x.abs().double(), y.abs().double()))
        # same bound the dot-product parity test uses against the FP64 sum
        assert abs(got - ref) <= 1e-6 * scale
    ctx.close()
