"""The C-ABI library: builds, loads, exports every symbol include/gsfit.h
declares, and its host-side helpers behave (no GPU needed: nothing here
launches a kernel)."""
import ctypes
import re
from pathlib import Path

import numpy as np
import pytest

import oracle
import scenes
from paper_2601_22026_gb300 import _build
from paper_2601_22026_gb300 import gsfit as G

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return G.load()


def declared_functions():
    text = (ROOT / "include" / "gsfit.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gsfit_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(G.SIGNATURES), "binding and header disagree"


def test_abi_version_and_status_strings(lib):
    assert lib.gsfit_abi_version() == 10
    assert lib.gsfit_status_string(G.GSFIT_ERR_CAPACITY) == b"instance capacity exceeded"
    assert lib.gsfit_status_string(G.GSFIT_ERR_TIMEOUT) == b"bounded device wait ran out"


def test_num_planes(lib):
    for deg, expect in [(0, 4), (1, 6), (2, 10), (3, 15)]:
        assert lib.gsfit_num_planes(deg) == expect == G.num_planes(deg)
    assert lib.gsfit_num_planes(4) == G.GSFIT_ERR_INVALID_ARG


def test_camera_layout_matches_oracle_tiles(lib):
    cams = scenes.periphery_batch_cameras(7)
    table = G.camera_table(cams)
    assert table.total_tiles == oracle.total_tiles(cams, 16)
    assert table.total_pixels == scenes.num_pixels(cams)
    off = oracle.pixel_offsets(cams)
    toff = 0
    for v in range(table.n_views):
        c = table.host[v]
        assert c.pixel_offset == off[v]
        assert c.tile_offset == toff
        toff += (-(-c.width // 16)) * (-(-c.height // 16))


def test_pack_roundtrip_and_lr_table():
    for deg in range(4):
        gs = scenes.random_gaussians(37, deg, 3)
        P = G.pack_params(gs)
        assert P.shape == (G.num_planes(deg), 37, 4)
        back = G.unpack_params(P, deg)
        for k in gs:
            np.testing.assert_array_equal(back[k], gs[k])
        L = G.lr_table(deg, 1.0, 2.0, 3.0, 4.0, 5.0)
        assert L[0, 3] == 4.0 and L[2, 3] == 0.0 and L[1, 0] == 2.0
        K3 = 3 * (deg + 1) ** 2
        flat = L[3:].reshape(-1)
        assert np.all(flat[:3] == 5.0) and np.all(flat[3:K3] == 0.25) and np.all(flat[K3:] == 0)


def test_invalid_arguments_rejected_on_host(lib):
    g = G.Gaussians(None, 10, 0)
    p = G.Proj(None, None, None, None)
    assert lib.gsfit_project(ctypes.byref(g), None, 1, ctypes.byref(p), None) == G.GSFIT_ERR_INVALID_ARG
    g = G.Gaussians(16, 10, 7)  # bad degree
    fake = 256
    p = G.Proj(fake, fake, fake, fake)
    assert lib.gsfit_project(ctypes.byref(g), fake, 1, ctypes.byref(p), None) == G.GSFIT_ERR_INVALID_ARG
    g = G.Gaussians(fake, 10, 0)
    assert lib.gsfit_project(ctypes.byref(g), fake, 0, ctypes.byref(p), None) == G.GSFIT_ERR_INVALID_ARG
    assert lib.gsfit_project(ctypes.byref(g), fake, 257, ctypes.byref(p), None) == G.GSFIT_ERR_INVALID_ARG
    # capacity at or above 2^30 and undersized workspaces are refused before any launch
    assert lib.gsfit_bin_sort(ctypes.byref(p), fake, 1, 10, 4, fake, 1 << 40, fake, fake, 1 << 30, fake, fake,
                              None, fake, None) == G.GSFIT_ERR_INVALID_ARG
    need = lib.gsfit_bin_sort_workspace_size(10, 1000, 4)
    assert need > 0
    assert lib.gsfit_bin_sort(ctypes.byref(p), fake, 1, 10, 4, fake, need - 1, fake, fake, 1000, fake, fake,
                              None, fake, None) == G.GSFIT_ERR_INVALID_ARG
    assert lib.gsfit_adam_step(fake, fake, fake, fake, 10, 17, None, 0.9, 0.999, 1e-15, fake, None, 0,
                               None) == G.GSFIT_ERR_INVALID_ARG
    assert lib.gsfit_loss_workspace_size(None, 0) == 0


def test_loss_workspace_size_with_match_flags(lib):
    """With the host camera table the loss workspace holds the accumulators
    (3 floats per view, padded to 256 bytes) and one flag byte per 16 x 16
    block and channel; without it, the accumulators only."""
    import scenes
    cams = scenes.stack_cameras([scenes.make_camera((0, 0, 3), (0, 0, 0), w, h, fx=50.0)
                                 for w, h in [(45, 37), (1920, 1920), (7, 5), (513, 257)]])
    table = G.camera_table(cams)
    V = table.n_views
    blocks = sum(-(-int(w) // 16) * -(-int(h) // 16) for w, h in zip(cams["width"], cams["height"]))
    assert G.gsfit_loss_workspace_size(table) == ((12 * V + 255) // 256) * 256 + 3 * blocks
    assert G.gsfit_loss_workspace_size(V) == 12 * V
    assert lib.gsfit_loss_workspace_size(None, G.GSFIT_MAX_VIEWS + 1) == 0
    # the tile order: permutation, count, furthest contributors, the adjoint's order, count
    assert G.tile_order_words(table.total_tiles) == 3 * table.total_tiles + 2


def test_fused_adjoint_adam_arguments_rejected_on_host(lib):
    """The projection adjoint with Adam: missing moments, learning rates or
    step count, misaligned buffers and a 16-bit feature type without its copy
    are refused before any launch."""
    fake = 256
    g = G.Gaussians(fake, 10, 3)
    p = G.Proj(fake, fake, fake, fake)
    lr = (ctypes.c_float * 64)()
    call = lambda gg, grad2d, grads, m, v, lrp, step: lib.gsfit_project_bwd_adam(
        ctypes.byref(gg), ctypes.byref(p), fake, 2, grad2d, grads, m, v, lrp, 0.9, 0.999, 1e-15, step, None, None)
    for args in [(fake, None, None, fake, lr, fake), (fake, None, fake, None, lr, fake),
                 (fake, None, fake, fake, None, fake), (fake, None, fake, fake, lr, None),
                 (None, None, fake, fake, lr, fake), (fake + 4, None, fake, fake, lr, fake),
                 (fake, fake + 8, fake, fake, lr, fake), (fake, None, fake + 4, fake, lr, fake)]:
        assert call(g, *args) == G.GSFIT_ERR_INVALID_ARG
    half = G.Gaussians(fake, 10, 3, None, G.FEATURES["f16"], 0)
    assert call(half, fake, None, fake, fake, lr, fake) == G.GSFIT_ERR_INVALID_ARG
    assert lib.gsfit_project_bwd_adam(None, ctypes.byref(p), fake, 2, fake, None, fake, fake, lr, 0.9, 0.999,
                                      1e-15, fake, None, None) == G.GSFIT_ERR_INVALID_ARG


def test_reproject_alignment_rejected_on_host(lib):
    """zbuf takes 64-bit atomics and clip 16-byte stores: misaligned pointers
    are refused before any launch."""
    fake = 256
    m = (ctypes.c_float * 16)(*np.eye(4, dtype=np.float32).reshape(-1))
    pos = (ctypes.c_float * 3)(0, 0, 0)
    args = lambda clip, zbuf: (fake, fake, 8, 8, m, pos, m, 8, 8, clip, zbuf, fake, fake, None)
    assert lib.gsfit_reproject(*args(None, fake + 4)) == G.GSFIT_ERR_INVALID_ARG
    assert lib.gsfit_reproject(*args(fake + 8, fake)) == G.GSFIT_ERR_INVALID_ARG
    assert lib.gsfit_reproject(*args(None, None)) == G.GSFIT_ERR_INVALID_ARG


def test_workspace_size_grows_with_capacity(lib):
    a = lib.gsfit_bin_sort_workspace_size(1000, 10_000, 64)
    b = lib.gsfit_bin_sort_workspace_size(1000, 20_000, 64)
    c = lib.gsfit_bin_sort_workspace_size(1000, 20_000, 70_000)  # more tile bits: one more pass
    assert 0 < a < b < c
    assert b - a >= 10_000 * 12


def test_feature_storage_arguments_rejected_on_host(lib):
    fake = 256
    p = G.Proj(fake, fake, fake, fake)
    # unknown storage type, and a 16-bit type without its copy
    for dtype, feats in [(7, fake), (G.FEATURES["f16"], None), (G.FEATURES["bf16"], None), (G.FEATURES["f16"], 260)]:
        g = G.Gaussians(fake, 10, 0, feats, dtype, 0)
        assert lib.gsfit_project(ctypes.byref(g), fake, 1, ctypes.byref(p), None) == G.GSFIT_ERR_INVALID_ARG
    lr = (ctypes.c_float * 16)()
    assert lib.gsfit_adam_step(fake, fake, fake, fake, 10, 4, lr, 0.9, 0.999, 1e-15, fake, None,
                               G.FEATURES["f16"], None) == G.GSFIT_ERR_INVALID_ARG
    assert lib.gsfit_adam_step(fake, fake, fake, fake, 10, 4, lr, 0.9, 0.999, 1e-15, fake, fake, 5,
                               None) == G.GSFIT_ERR_INVALID_ARG
    assert lib.gsfit_features_refresh(fake, 10, 4, fake, G.FEATURES["f32"], None) == G.GSFIT_ERR_INVALID_ARG
    assert lib.gsfit_features_refresh(fake, 10, 3, fake, G.FEATURES["f16"], None) == G.GSFIT_ERR_INVALID_ARG


def test_camera_layout_tile_edges(lib):
    cams = scenes.periphery_batch_cameras(7)
    for tile in (8, 16):
        table = G.camera_table(cams, tile)
        assert table.total_tiles == oracle.total_tiles(cams, tile)
        assert all(table.host[v].tile == tile for v in range(table.n_views))
    with pytest.raises(RuntimeError):
        G.camera_table(cams, 12)


def test_render_options_rejected_on_host(lib):
    fake = 256
    p = G.Proj(fake, fake, fake, fake)
    for opts in [G.RenderOpts(8, 100), G.RenderOpts(32, 128), G.RenderOpts(12, 64), G.RenderOpts(16, 128, 2),
                 G.RenderOpts(16, 128, 0, 1), G.RenderOpts(16, 128, 0, 100), G.RenderOpts(16, 128, 0, 512)]:
        assert lib.gsfit_render_fwd(ctypes.byref(p), fake, 1, 10, 4, fake, fake, None, fake, fake, fake, fake, fake,
                                    ctypes.byref(opts), None, None) == G.GSFIT_ERR_INVALID_ARG
        assert lib.gsfit_blend_bwd(ctypes.byref(p), fake, 1, 10, 4, fake, fake, None, fake, fake, fake, fake, fake,
                                   fake, ctypes.byref(opts), None, None) == G.GSFIT_ERR_INVALID_ARG
    best = G.RenderOpts()
    assert lib.gsfit_render_autotune(ctypes.byref(p), fake, 1, 10, 4, fake, fake, None, fake, fake, fake, fake, fake,
                                     fake, fake, fake, 12, 3, ctypes.byref(best), None, None,
                                     None) == G.GSFIT_ERR_INVALID_ARG


def test_splat_power_selftest_arguments_rejected_on_host(lib):
    fake = 256
    assert lib.gsfit_selftest_splat_power(None, None, 1, None, None) == G.GSFIT_ERR_INVALID_ARG
    assert lib.gsfit_selftest_splat_power(fake, None, 1, fake, None) == G.GSFIT_ERR_INVALID_ARG
    assert lib.gsfit_selftest_splat_power(fake, fake, -1, fake, None) == G.GSFIT_ERR_INVALID_ARG
    assert lib.gsfit_selftest_splat_power(None, None, 0, None, None) == G.GSFIT_OK  # empty: nothing launched


def test_fit_stage_lists_name_state_methods():
    """The timed stage lists (the separate adjoint and Adam, and the fused
    pass) name FitState methods, which the graph capture and the bench call
    by name; the default list is the separate kernels'."""
    from paper_2601_22026_gb300.fit import FitState
    for stages in (FitState.TIMED_STAGES_SEPARATE, FitState.TIMED_STAGES_FUSED):
        for name in stages:
            assert callable(getattr(FitState, name, None)), name
    assert FitState.TIMED_STAGES == FitState.TIMED_STAGES_SEPARATE
    assert FitState.TIMED_STAGES_FUSED[-1] == "project_bwd_adam"
    assert set(FitState.STAGES) - {"render_bwd"} <= set(FitState.TIMED_STAGES_SEPARATE)
