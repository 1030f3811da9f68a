"""Host-side checks of the C ABI that need no GPU: the library builds, loads,
exports every entry point include/claire.h declares, and its host logic
(option defaults, workspace sizing, argument validation) behaves."""
import ctypes
import os
import re

import pytest

import __graft_entry__ as entry

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def claire():
    entry.build()
    from paper_2209_08189_gb300 import claire as c
    return c


def _declared(header="claire.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(claire_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(claire):
    lib = claire.lib()
    declared = _declared()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name
    # the binding wraps exactly the declared entry points
    assert set(claire.exported_symbols()) == set(declared)


def test_every_network_symbol_is_exported(claire):
    """include/claire_net.h: exported by libclaire and bound by net.py with
    the same names; host-side validation rejects bad shapes without a GPU."""
    from paper_2209_08189_gb300 import net
    lib = net.lib()
    declared = _declared("claire_net.h")
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), name
    assert set(net._SIGS) == set(declared)
    chunks = ctypes.c_int()
    bad = (ctypes.c_int * 4)(1, 8, 8, 6)
    assert lib.claire_net_conv3d_wgrad_chunks(16, 16, bad, ctypes.byref(chunks)) == -1
    assert b"powers of two" in lib.claire_net_last_error()
    good = (ctypes.c_int * 4)(1, 8, 8, 8)
    assert lib.claire_net_conv3d_wgrad_chunks(24, 16, good, ctypes.byref(chunks)) == -1
    assert lib.claire_net_set_wgrad_tiling(24) == -1
    assert b"set_wgrad_tiling" in lib.claire_net_last_error()
    assert lib.claire_net_set_wgrad_tiling(0) == 0


def test_net_layer_table_has_the_stated_size(claire):
    from paper_2209_08189_gb300 import net
    layers = net.unet_layers((16, 32, 64, 128), 16)
    n = sum(co * 27 * ci + co for _, ci, co in layers) + 3 * 16 + 3
    assert 1.4e6 < n < 1.5e6
    assert [l[0] for l in layers][:2] == ["enc0a", "enc0b"] and layers[-1][0] == "dec0b"


def test_default_opts(claire):
    o = claire.claire_default_opts()
    assert o.interp == 3 and o.reg == 1 and abs(o.beta_w - 1e-4) < 1e-18
    assert abs(o.gtol - 5e-2) < 1e-18 and o.grad_form == 0 and o.timing == 0
    # the spectral preconditioner by default; the two-level one's defaults
    assert o.precond == claire.PRECOND_SPECTRAL and o.pc_coarse == 2
    assert abs(o.pc_tol - 1e-1) < 1e-18 and o.pc_maxit == 50


def test_two_level_options_are_validated(claire):
    """Invalid preconditioner options are rejected on the host (no GPU needed:
    validation precedes any device call)."""
    o = claire.claire_default_opts()
    o.precond = 2
    lib = claire.lib()
    ctx = ctypes.c_void_p()
    grid = (ctypes.c_int * 3)(16, 16, 16)
    assert lib.claire_create(ctypes.byref(ctx), grid, ctypes.c_double(1e-2), 4, ctypes.byref(o)) == -1
    o = claire.claire_default_opts()
    o.precond = claire.PRECOND_TWO_LEVEL
    o.pc_coarse = 3  # 16 / 3 is not whole
    assert lib.claire_create(ctypes.byref(ctx), grid, ctypes.c_double(1e-2), 4, ctypes.byref(o)) == -1
    o.pc_coarse = 8  # 16 / 8 = 2 < 4
    assert lib.claire_create(ctypes.byref(ctx), grid, ctypes.c_double(1e-2), 4, ctypes.byref(o)) == -1
    o.pc_coarse = 2
    o.pc_tol = -1.0
    assert lib.claire_create(ctypes.byref(ctx), grid, ctypes.c_double(1e-2), 4, ctypes.byref(o)) == -1


def test_query_workspace_scales_with_grid_and_nt(claire):
    b64 = claire.claire_query_workspace((64, 64, 64), 4)
    b128 = claire.claire_query_workspace((128, 128, 128), 4)
    assert 7.5 < b128 / b64 < 8.5
    assert claire.claire_query_workspace((64, 64, 64), 8) > b64
    # about 35 + 5 (nt+1) float fields per point (images, velocity, two
    # characteristics, nt+1 states, their gradients and adjoint levels, five
    # real and five Fourier-space vector buffers)
    assert 65 * 4 * 64 ** 3 < b64 < 75 * 4 * 64 ** 3
    # without stored state gradients: 3 (nt+1) = 15 fields fewer
    o = claire.claire_default_opts()
    o.lowmem = 1
    assert abs(b64 - claire.claire_query_workspace((64, 64, 64), 4, o) - 15 * 4 * 64 ** 3) < 64 * 1024


def test_reduced_storage_shrinks_workspace(claire):
    o32 = claire.claire_default_opts()
    o16 = claire.claire_default_opts()
    o16.storage = claire.STORAGE_F16
    ob = claire.claire_default_opts()
    ob.storage = claire.STORAGE_BF16
    b32 = claire.claire_query_workspace((64, 64, 64), 4, o32)
    b16 = claire.claire_query_workspace((64, 64, 64), 4, o16)
    assert claire.claire_query_workspace((64, 64, 64), 4, ob) == b16
    # 2 + 2 + 5 + 15 + 5 = 29 scalar fields per point (images, div v and its
    # value at X+, states, their gradients, adjoint levels) drop from 4 to 2 bytes
    assert abs((b32 - b16) - 29 * 2 * 64 ** 3) < 64 * 1024
    o16.storage = 3
    with pytest.raises(claire.ClaireError):
        claire.claire_query_workspace((64, 64, 64), 4, o16)


@pytest.mark.parametrize("grid", [(7, 8, 8), (8, 8, 9), (6, 8, 8), (0, 8, 8)])
def test_invalid_grids_rejected(claire, grid):
    with pytest.raises(claire.ClaireError) as e:
        claire.claire_query_workspace(grid, 4)
    assert e.value.status == -1
    with pytest.raises(claire.ClaireError) as e:
        claire.claire_create(grid, 1e-2, 4)
    assert e.value.status == -1


def test_invalid_parameters_rejected(claire):
    for beta, nt in ((0.0, 4), (-1.0, 4), (1e-2, 0)):
        with pytest.raises(claire.ClaireError) as e:
            claire.claire_create((8, 8, 8), beta, nt)
        assert e.value.status == -1
    o = claire.claire_default_opts()
    o.interp = 2
    with pytest.raises(claire.ClaireError) as e:
        claire.claire_create((8, 8, 8), 1e-2, 4, o)
    assert e.value.status == -1


def test_null_context_calls_fail_cleanly(claire):
    lib = claire.lib()
    assert lib.claire_destroy(None) == 0
    assert lib.claire_set_images(None, None, None) == -1
    assert lib.claire_register(None, None, None) == -1
    assert lib.claire_last_error(None) == b"null context"


@pytest.mark.skipif(bool(os.environ.get("CUDA_VISIBLE_DEVICES_FORCE")), reason="gpu forced")
def test_create_fails_loudly_without_gpu(claire):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(claire.ClaireError) as e:
        claire.claire_create((8, 8, 8), 1e-2, 4)
    assert e.value.status == -3


def test_wgrad_chunk_counts_are_consistent(claire):
    """Host-side tiling of the weight gradient (no GPU needed): every shape gets
    at least one chunk and no more chunks than bricks; a forced input-channel
    block that does not divide Cin leaves the shape to the mma.sync kernel (whose
    chunking differs); an invalid block is rejected."""
    from paper_2209_08189_gb300 import net
    lib = net.lib()
    shapes = [(16, 16, (4, 128, 128, 128)), (48, 16, (4, 128, 128, 128)), (96, 32, (4, 64, 64, 64)),
              (192, 64, (4, 32, 32, 32)), (128, 128, (4, 16, 16, 16)), (32, 48, (2, 4, 16, 16)),
              (32, 48, (2, 8, 8, 16))]
    for ci, co, vol in shapes:
        c = net.wgrad_chunks(ci, co, vol)
        B, D, H, W = vol
        bricks = B * D * (H // 16) * (W // 8) if H % 16 == 0 and W % 8 == 0 else B * D * H * W // 64
        assert 1 <= c <= max(1, bricks), (ci, co, vol, c)
    base = net.wgrad_chunks(96, 32, (4, 64, 64, 64))
    try:
        for nc in (16, 32, 48):
            net.set_wgrad_tiling(nc)
            assert net.wgrad_chunks(96, 32, (4, 64, 64, 64)) >= 1
        net.set_wgrad_tiling(64)  # 96 % 64 != 0: the mma.sync kernel's chunking
        assert net.wgrad_chunks(96, 32, (4, 64, 64, 64)) >= 1
    finally:
        net.set_wgrad_tiling(0)
    assert net.wgrad_chunks(96, 32, (4, 64, 64, 64)) == base
    assert lib.claire_net_set_wgrad_tiling(40) == -1
