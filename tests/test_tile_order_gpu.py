"""The tile order's use in the compositing launches. With an order, the CTAs
past its non-empty count leave before any setup (the forward pass after
writing the background into its tile); the forward pass records each
non-empty tile's furthest contributor, and the adjoint launches the
non-empty tiles sorted by it. What must hold: the forward outputs equal
those of the launch without an order, which composites every tile in full,
bit for bit (each pixel's sum runs in its own list order either way); the
adjoint's 2D gradients equal them up to the order of their float atomics;
an empty tile holds the background, alpha 0, T 1 and no contributor; the
recorded contributor is the tile's largest n_contrib; and the adjoint's
order is a permutation of the non-empty tiles in descending quarter octaves
of it."""
import numpy as np
import pytest

import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2601_22026_gb300 as pkg
    pkg.build()


def _state(gs, cams, bg, **kw):
    from paper_2601_22026_gb300.fit import FitState
    return FitState(gs, cams, bg=bg, **kw)


def _case(name):
    if name == "clustered":  # splats clustered to one side: most tiles empty
        gs = scenes.random_gaussians(2500, 2, 31, log_scale_mean=-2.6)
        gs["means"] = (gs["means"] * np.float32(0.1) + np.float32([0.6, 0.3, 0.0])).astype(np.float32)
        cams = scenes.stack_cameras([scenes.make_camera((0, 0, 3), (0, 0, 0), 333, 250, fx=260.0),
                                     scenes.make_camera((0.4, -2.8, 1.0), (0, 0, 0), 97, 61, fx=70.0),
                                     scenes.make_camera((2.5, 1.0, 1.0), (0, 0, 0), 200, 136, fx=150.0)])
        return gs, cams
    # the largest view count the calls accept, ragged 24 x 17 views
    return scenes.random_gaussians(400, 1, 15, log_scale_mean=-2.8), scenes.orbit_cameras(256, 24, 17, 60.0, 3.0, 16)


def _fwd_unordered(st):
    from paper_2601_22026_gb300 import gsfit as G
    out = [torch.empty_like(x) for x in (st.rgb, st.alpha, st.T_final, st.n_contrib)]
    G.gsfit_render_fwd(st.proj, st.cams_dev, st.V, st.n, st.T, st.vals, st.ranges, st.bg, *out,
                       None, None, st.status, st.opts)
    return out


@pytest.mark.parametrize("case", ["clustered", "max_views"])
@pytest.mark.parametrize("tile", [16, 8])
def test_forward_with_order_matches_unordered_launch(case, tile):
    gs, cams = _case(case)
    bg = scenes.backgrounds(len(cams["width"]), 5)
    st = _state(gs, cams, bg, tile=tile, batch=64 if tile == 8 else 128)
    st.project()
    st.bin_sort()
    st.render_fwd()
    ref = _fwd_unordered(st)
    torch.cuda.synchronize()
    assert st.check_status() == 0
    T = st.T
    words = st.tile_order.cpu().numpy().view(np.uint32).astype(np.int64)
    ranges = st.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2).astype(np.int64)
    lens = ranges[:, 1] - ranges[:, 0]
    n_work = int(words[T])
    assert n_work == int(np.count_nonzero(lens)) and 0 < n_work <= T
    if case == "clustered":
        assert n_work < T  # empty tiles too
    for a, b in zip((st.rgb, st.alpha, st.T_final, st.n_contrib), ref):
        np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
    # empty tiles: the background, alpha 0, T 1, no contributor
    empty = words[n_work:T]
    assert np.all(lens[empty] == 0)
    rgb, alpha, T_f, nc = (x.cpu().numpy() for x in (st.rgb, st.alpha, st.T_final, st.n_contrib))
    W_all, H_all = cams["width"].astype(np.int64), cams["height"].astype(np.int64)
    off = np.concatenate([[0], np.cumsum(W_all * H_all)])
    tiles_x, tiles_y = -(-W_all // tile), -(-H_all // tile)
    toff = np.concatenate([[0], np.cumsum(tiles_x * tiles_y)])
    for t in empty[:: max(1, len(empty) // 40)]:
        v = int(np.searchsorted(toff, t, side="right") - 1)
        W, H = int(W_all[v]), int(H_all[v])
        tx, ty = (t - toff[v]) % tiles_x[v], (t - toff[v]) // tiles_x[v]
        ys, xs = np.mgrid[ty * tile:min((ty + 1) * tile, H), tx * tile:min((tx + 1) * tile, W)]
        pix = off[v] + ys * W + xs
        assert np.all(alpha[pix] == 0) and np.all(T_f[pix] == 1) and np.all(nc[pix] == 0)
        for ch in range(3):
            assert np.all(rgb[3 * off[v] + ch * W * H + ys * W + xs] == np.float32(bg[v, ch]))


@pytest.mark.parametrize("tile", [16, 8])
def test_adjoint_with_order_matches_unordered_launch(tile):
    from paper_2601_22026_gb300 import gsfit as G
    gs, cams = _case("clustered")
    bg = scenes.backgrounds(len(cams["width"]), 6)
    st = _state(gs, cams, bg, tile=tile, batch=64 if tile == 8 else 128)
    st.forward()
    P = st.P
    st.dL_drgb.copy_(torch.from_numpy(scenes.cotangents(3 * P, 801, 1e-3)))
    st.dL_dalpha.copy_(torch.from_numpy(scenes.cotangents(P, 802, 1e-3)))
    st.grad2d.zero_()
    st.blend_bwd()
    torch.cuda.synchronize()
    got = st.grad2d.cpu().numpy().copy()
    _check_adjoint_order(st, cams, tile)
    st.grad2d.zero_()
    G.gsfit_blend_bwd(st.proj, st.cams_dev, st.V, st.n, st.T, st.vals, st.ranges, st.bg, st.T_final, st.n_contrib,
                      st.dL_drgb, st.dL_dalpha, st.grad2d, None, None, st.status, st.opts)
    torch.cuda.synchronize()
    assert st.check_status() == 0
    ref = st.grad2d.cpu().numpy()
    assert np.abs(ref).max() > 0
    np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-6 * np.abs(ref).max())


def _tile_max_contrib(st, cams, tile):
    """The largest n_contrib of each tile's pixels (host)."""
    nc = st.n_contrib.cpu().numpy().view(np.uint32).astype(np.int64)
    out, off = [], 0
    for W, H in zip(cams["width"].astype(np.int64), cams["height"].astype(np.int64)):
        tx, ty = -(-W // tile), -(-H // tile)
        pad = np.zeros((ty * tile, tx * tile), np.int64)
        pad[:H, :W] = nc[off:off + W * H].reshape(H, W)
        out.append(pad.reshape(ty, tile, tx, tile).max(axis=(1, 3)).reshape(-1))
        off += W * H
    return np.concatenate(out)


def _bucket(m):
    """Quarter octave of m + 1 (floor of 4 log2, from the two bits below the leading one)."""
    x = np.asarray(m, np.int64) + 1
    l = np.floor(np.log2(x)).astype(np.int64)
    f = np.where(l >= 2, (x >> np.maximum(l - 2, 0)) & 3, (x << np.maximum(2 - l, 0)) & 3)
    return 4 * l + f


def _check_adjoint_order(st, cams, tile):
    T = st.T
    words = st.tile_order.cpu().numpy().view(np.uint32).astype(np.int64)
    assert len(words) == 3 * T + 2
    n_work = int(words[T])
    key = words[T + 1:2 * T + 1]
    nonempty = words[:n_work]
    np.testing.assert_array_equal(key[nonempty], _tile_max_contrib(st, cams, tile)[nonempty])
    adj = words[2 * T + 1:2 * T + 1 + n_work]
    assert words[3 * T + 1] == n_work
    np.testing.assert_array_equal(np.sort(adj), np.sort(nonempty))
    assert np.all(np.diff(_bucket(key[adj])) <= 0)


def test_contributor_bucket_matches_its_definition():
    """The host restatement of the quarter-octave bucket used above, against
    4 floor(log2(m + 1)) + the two bits below the leading one, by brute force."""
    for m in list(range(0, 300)) + [1000, 4095, 4096, 65535, 10 ** 6]:
        x = m + 1
        l = x.bit_length() - 1
        f = (x >> (l - 2)) & 3 if l >= 2 else (x << (2 - l)) & 3
        assert _bucket(m) == 4 * l + f


def test_next_order_follows_the_recorded_contributors():
    """bin_sort of the next iteration orders the non-empty tiles by the
    furthest contributor the forward pass recorded (capped at the new list
    length; the length where none was recorded), the empty tiles last, and
    zeroes the recorded words for the next forward pass."""
    gs, cams = _case("clustered")
    bg = scenes.backgrounds(len(cams["width"]), 8)
    st = _state(gs, cams, bg)
    st.forward()
    torch.cuda.synchronize()
    T = st.T
    key = st.tile_order.cpu().numpy().view(np.uint32)[T + 1:2 * T + 1].astype(np.int64).copy()
    assert key.max() > 0
    gs2 = dict(gs)
    gs2["means"] = (gs["means"] + np.float32(0.01)).astype(np.float32)  # the next iteration's scene, moved a little
    from paper_2601_22026_gb300 import gsfit as G
    st.params.copy_(torch.from_numpy(G.pack_params(gs2)).to(st.params.device))
    st.project()
    st.bin_sort()
    torch.cuda.synchronize()
    words = st.tile_order.cpu().numpy().view(np.uint32).astype(np.int64)
    ranges = st.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2).astype(np.int64)
    lens = ranges[:, 1] - ranges[:, 0]
    order = words[:T]
    assert np.array_equal(np.sort(order), np.arange(T))
    work = np.where((key > 0) & (key < lens), key, lens)[order]
    buckets = np.where(lens[order] > 0, np.minimum(127, 1 + _bucket(work)), 0)
    assert np.all(np.diff(buckets) <= 0)
    assert words[T] == np.count_nonzero(lens)
    assert np.all(words[T + 1:2 * T + 1] == 0)
