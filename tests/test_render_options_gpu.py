"""The tunables of the batched launch against the FP64 oracle: every
(tile edge, forward batch depth, adjoint batch depth) variant of the
compositing kernels gives the same
keys, sorted lists and ranges as the oracle at that tile edge (bit for bit),
the same images (1e-4) and gradients (1e-3); a compositing call told a tile
edge the cameras were not laid out for reports it and does nothing; the
tuner returns a supported option and leaves the adjoint workspace zero."""
import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F = oracle.F
# (16, 128, 64) is the default, which the parity tests run
VARIANTS = [(8, 64, 64), (8, 128, 128), (8, 256, 256), (16, 64, 128), (16, 256, 256), (16, 128, 128),
            (16, 64, 64)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2601_22026_gb300 as pkg
    pkg.build()


def _state(gs, cams, bg, tile, batch, batch_bwd=64):
    from paper_2601_22026_gb300.fit import FitState
    return FitState(gs, cams, bg=bg, tile=tile, batch=batch, batch_bwd=batch_bwd, keep_keys=True)


@pytest.mark.parametrize("tile,batch,batch_bwd", VARIANTS)
def test_variant_matches_oracle(tile, batch, batch_bwd):
    from test_parity_gpu import (_case, _grad_check, _pairs_excluding, _pixel_tile_mask, _radius_flips,
                                 _rgb_to_pixels)
    gs, cams, bg = _case("sh3_uneven_views")
    st = _state(gs, cams, bg, tile, batch, batch_bwd)
    P = scenes.num_pixels(cams)
    w_rgb = scenes.cotangents(3 * P, 801, 1e-3)
    w_a = scenes.cotangents(P, 802, 1e-3)
    st.forward()
    torch.cuda.synchronize()
    assert st.check_status() == 0
    ref = oracle.render(gs, cams, bg, tile=tile)
    # keys and lists at this tile edge
    flips = _radius_flips(st, ref["proj"])
    n_inst = int(st.n_instances.item())
    keys = st.keys[:n_inst].cpu().numpy().view(np.uint64)
    vals = st.vals[:n_inst].cpu().numpy().view(np.uint32)
    gk, gv, bad_g = _pairs_excluding(keys, vals, ref["proj"], cams, st.n, flips)
    rk, rv, bad_o = _pairs_excluding(ref["keys"], ref["vals"], ref["proj"], cams, st.n, flips)
    np.testing.assert_array_equal(gk, rk)
    np.testing.assert_array_equal(gv, rv)
    if not (bad_g | bad_o):
        np.testing.assert_array_equal(st.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2), ref["ranges"])
    # images (the exclusion mask is built for 16-pixel tiles: widen it to the
    # 16-pixel tiles containing any excluded tile of this edge)
    bad16 = {t for t in (bad_g | bad_o)} if tile == 16 else _tiles16_of(cams, bad_g | bad_o, tile)
    ok = ~(ref["ambiguous"] | _pixel_tile_mask(cams, bad16))
    assert ok.mean() > 0.95
    rgb = _rgb_to_pixels(st.rgb.cpu().numpy().astype(np.float64), cams)
    assert np.abs(rgb - _rgb_to_pixels(ref["rgb"], cams))[ok].max() <= 1e-4
    np.testing.assert_array_equal(st.n_contrib.cpu().numpy()[ok], ref["n_contrib"][ok])
    # gradients
    st.dL_drgb.copy_(torch.from_numpy(w_rgb))
    st.dL_dalpha.copy_(torch.from_numpy(w_a))
    st.render_bwd()
    torch.cuda.synchronize()
    refg = oracle.render_bwd(gs, cams, bg, w_rgb.astype(np.float64), w_a.astype(np.float64), tile=tile)
    amb = refg["gauss_ambiguous"].any(axis=0) | (ref["proj"][:, :, F["near_boundary"]] > 0).any(axis=0)
    _grad_check(st.gradients(), refg["grads"], amb)
    assert float(st.grad2d.abs().max().item()) == 0.0


def _tiles16_of(cams, tiles, tile):
    """Global 16-pixel tile ids covering the given global tiles of edge `tile`."""
    out = set()
    off, off16 = 0, 0
    for W, H in zip(cams["width"], cams["height"]):
        W, H = int(W), int(H)
        txn, tyn = -(-W // tile), -(-H // tile)
        txn16, tyn16 = -(-W // 16), -(-H // 16)
        for t in tiles:
            if off <= t < off + txn * tyn:
                ty, tx = divmod(t - off, txn)
                out.add(off16 + (ty * tile // 16) * txn16 + tx * tile // 16)
        off += txn * tyn
        off16 += txn16 * tyn16
    return out


def test_tile_mismatch_is_reported_and_does_nothing():
    from paper_2601_22026_gb300 import gsfit as G
    from test_parity_gpu import _case
    gs, cams, bg = _case("sh1_ragged")
    st = _state(gs, cams, bg, 16, 128)
    st.forward()
    torch.cuda.synchronize()
    assert st.check_status() == 0
    st.rgb.fill_(-7.0)
    G.gsfit_render_fwd(st.proj, st.cams_dev, st.V, st.n, st.T, st.vals, st.ranges, st.bg, st.rgb, st.alpha,
                       st.T_final, st.n_contrib, None, st.tile_order, st.status, (8, 128))
    torch.cuda.synchronize()
    assert st.check_status() == G.GSFIT_ERR_INVALID_ARG
    assert float(st.rgb.max().item()) == -7.0


@pytest.mark.parametrize("tile", [8, 16])
def test_batch_tuner(tile):
    from test_parity_gpu import _case
    gs, cams, bg = _case("sh3_uneven_views")
    st = _state(gs, cams, bg, tile, 128)
    st.forward()
    torch.cuda.synchronize()
    rgb0 = st.rgb.clone()
    times = st.tune_batch(reps=2)
    assert st.check_status() == 0
    assert st.opts.tile == tile and st.opts.batch in (64, 128, 256) and st.opts.batch_bwd in (64, 128, 256)
    assert st.opts.batch == min(times, key=lambda d: times[d][0])
    assert st.opts.batch_bwd == min(times, key=lambda d: times[d][1])
    assert set(times) == {64, 128, 256} and all(f > 0 and b > 0 for f, b in times.values())
    assert float(st.grad2d.abs().max().item()) == 0.0
    # the forward result does not depend on the batch depth
    assert torch.equal(st.rgb, rgb0)
