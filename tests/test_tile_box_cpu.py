"""Box arithmetic of the tiled semi-Lagrangian gathers, checked on the host.

The gathers (RK2 backtrace and every SL step, Sec. 3's IP kernel) stage the
departure box of a tile in shared memory.  `tile_box_host.cu` compiles the
kernels' own __host__ __device__ split / bounds / box code for the CPU and runs
it over NaN, +-Inf, +-1e7, values at and below 2^20 cells and ordinary
displacements on a cubic, a ragged and two small grids: every fitting box must
hold all stencil nodes of its tile, and any tile with a non-finite or huge
displacement must be sent to the global-memory path.  Boxes taken from a
tile-bounds table (the backtrace's by-product) are checked against other
fields, NaN / Inf / huge values and arbitrary integer bounds: no point may
pass the in-box test with a stencil node outside the box.  No GPU is used.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "bin", "nvcc")):
            return os.path.join(cand, "bin", "nvcc")
    return shutil.which("nvcc")


def test_tile_box_host(tmp_path):
    nvcc = _nvcc()
    if not nvcc:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "tile_box_host")
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O1", "-std=c++17", "--expt-relaxed-constexpr",
           "-I" + os.path.join(ROOT, "include"), "-I" + os.path.join(ROOT, "paper_2209_08189_gb300", "csrc"),
           os.path.join(ROOT, "tests", "tile_box_host.cu"), "-o", exe]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stdout + res.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0 and run.stdout.strip().endswith("OK"), run.stdout + run.stderr
    # the realistic cases took the box path on the large grids, the bad ones did not
    assert "smooth                       order 3 es 4  tiles: 432 box, 0 global" in run.stdout
    assert "all NaN                      order 3 es 4  tiles: 0 box, 432 global (432 with bad" in run.stdout
    # tile-bounds tables: with their own field every point stays on the box
    # path; with another field some points fall outside and take the global path
    assert "table own field              order 3 es 4  box tiles 256, points in box 262144, out 0" in run.stdout
    assert "table NaN/Inf/huge field     order 3 es 4  box tiles 256" in run.stdout
