"""Depth-guided reprojection (Section 4.3, Eqs. 2-4): the FP64 oracle pinned to
closed forms (CPU), and the GPU kernels against it (-m gpu)."""
import numpy as np
import pytest

import oracle
import scenes


def _cam(pos, target, W=24, H=20, fx=30.0):
    return scenes.stack_cameras([scenes.make_camera(pos, target, W, H, fx=fx)])


# Pixel positions are compared to 1e-5 px: the far-plane point sits 100 units
# out (near 0.2), and the depth mapping's conditioning lifts float64 rounding
# to ~1e-7 px; a convention error (half-pixel offset, transposed matrix,
# wrong far plane) moves pixels by whole fractions of a pixel.
PX = 1e-5


def _setup(cam, depth):
    pv = scenes.projection_view(cam, 0)
    return np.linalg.inv(pv), np.asarray(cam["campos"][0], np.float64), pv


def _ray_depth(cam, z0):
    """Linear depth of a fronto-parallel plane at camera-space z0, per pixel."""
    W, H = int(cam["width"][0]), int(cam["height"][0])
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    rx = (x - float(cam["cx"][0])) / float(cam["fx"][0])
    ry = (y - float(cam["cy"][0])) / float(cam["fy"][0])
    return (z0 * np.sqrt(rx * rx + ry * ry + 1.0)).reshape(-1)


def test_identity_motion_maps_every_pixel_to_itself():
    cam = _cam((0.3, -2.5, 1.0), (0, 0, 0))
    W, H = 24, 20
    g = scenes.rng(3)
    depth = g.uniform(1.0, 4.0, W * H)
    rgb = g.uniform(0, 1, (3, W * H))
    inv, pos, pv = _setup(cam, depth)
    r = oracle.reproject(rgb, depth, W, H, inv, pos, pv, W, H)
    c = r["clip"]
    y, x = np.divmod(np.arange(W * H), W)
    np.testing.assert_allclose((c[:, 0] / c[:, 3] + 1) * 0.5 * W - 0.5, x, rtol=0, atol=PX)
    np.testing.assert_allclose((c[:, 1] / c[:, 3] + 1) * 0.5 * H - 0.5, y, rtol=0, atol=PX)
    assert r["covered"].all()
    np.testing.assert_array_equal(r["out_rgb"], rgb)


def test_reconstructed_point_lies_on_the_pixel_ray_at_its_depth():
    cam = _cam((1.5, 2.0, -1.0), (0.1, 0, 0.2))
    W, H = 24, 20
    depth = scenes.rng(4).uniform(0.5, 5.0, W * H)
    inv, pos, pv = _setup(cam, depth)
    pw = oracle.reproject(np.zeros((3, W * H)), depth, W, H, inv, pos, pv, W, H)["p_world"]
    np.testing.assert_allclose(np.linalg.norm(pw - pos, axis=1), depth, rtol=1e-12)  # exact by construction
    # the pinhole camera sees the point at the pixel's centre
    vm = np.asarray(cam["viewmat"][0], np.float64).reshape(3, 4)
    pc = pw @ vm[:, :3].T + vm[:, 3]
    u = float(cam["fx"][0]) * pc[:, 0] / pc[:, 2] + float(cam["cx"][0])
    v = float(cam["fy"][0]) * pc[:, 1] / pc[:, 2] + float(cam["cy"][0])
    y, x = np.divmod(np.arange(W * H), W)
    np.testing.assert_allclose(u, x, rtol=0, atol=PX)
    np.testing.assert_allclose(v, y, rtol=0, atol=PX)


def test_sideways_move_shifts_a_plane_by_f_dx_over_z():
    z0, dx, fx = 3.0, 0.1, 30.0
    old = _cam((0, 0, -z0), (0, 0, 0), fx=fx)
    new = _cam((dx, 0, -z0), (dx, 0, 0), fx=fx)
    W, H = 24, 20
    depth = _ray_depth(old, z0)
    inv, pos, _ = _setup(old, depth)
    pv_new = scenes.projection_view(new, 0)
    c = oracle.reproject(np.zeros((3, W * H)), depth, W, H, inv, pos, pv_new, W, H)["clip"]
    y, x = np.divmod(np.arange(W * H), W)
    right = np.asarray(old["viewmat"][0], np.float64).reshape(3, 4)[0, :3]  # the camera's +x axis in world space
    shift = -fx * float(right @ np.array([dx, 0.0, 0.0])) / z0  # camera-space x drops by right . move
    assert abs(shift) == pytest.approx(1.0)
    np.testing.assert_allclose((c[:, 0] / c[:, 3] + 1) * 0.5 * W - 0.5, x + shift, rtol=0, atol=PX)
    np.testing.assert_allclose((c[:, 1] / c[:, 3] + 1) * 0.5 * H - 0.5, y, rtol=0, atol=PX)
    np.testing.assert_allclose(c[:, 3], z0, rtol=1e-9)  # w is the new camera's depth


def test_nearest_source_wins_and_ties_go_to_the_lower_index():
    cam = _cam((0, 0, -3), (0, 0, 0), W=2, H=1)
    inv, pos, _ = _setup(cam, None)
    # every point lands on the output centre; w = world z + 5 (source 1 nearer)
    pv_new = np.zeros((4, 4))
    pv_new[3] = [0, 0, 1, 5]
    rgb = np.array([[1.0, 2.0], [0, 0], [0, 0]])
    depth = np.array([3.5, 3.2])
    r = oracle.reproject(rgb, depth, 2, 1, inv, pos, pv_new, 1, 1)
    assert r["covered"][0] and r["out_rgb"][0, 0] == 2.0
    r = oracle.reproject(rgb, np.array([3.0, 3.0]) * _ray_depth(cam, 1.0), 2, 1, inv, pos, pv_new, 1, 1)
    assert r["out_rgb"][0, 0] == 1.0  # equal w: the lower source index


@pytest.mark.gpu
def test_gpu_matches_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2601_22026_gb300 as pkg
    from paper_2601_22026_gb300 import gsfit as G
    pkg.build()
    old = _cam((0.2, -2.8, 0.9), (0, 0, 0), W=200, H=150, fx=180.0)
    new = _cam((0.26, -2.75, 0.93), (0.02, 0.01, 0), W=180, H=160, fx=170.0)
    W, H, OW, OH = 200, 150, 180, 160
    g = scenes.rng(9)
    yy, xx = np.mgrid[0:H, 0:W]
    depth = (2.5 + 0.4 * np.sin(xx / 17.0) * np.cos(yy / 11.0) + (xx > 120) * 0.6).reshape(-1)  # with a step
    rgb = g.uniform(0, 1, (3, W * H)).astype(np.float32)
    inv, pos, _ = _setup(old, depth)
    pv_new = scenes.projection_view(new, 0)
    # the GPU gets float32 inputs; the oracle the same float32 values
    inv32, pos32, pv32 = inv.astype(np.float32), pos.astype(np.float32), pv_new.astype(np.float32)
    d32 = depth.astype(np.float32)
    ref = oracle.reproject(rgb, d32, W, H, inv32, pos32, pv32, OW, OH)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    clip = torch.zeros(W * H * 4, device="cuda")
    zbuf = torch.zeros(OW * OH, dtype=torch.int64, device="cuda")
    out = torch.zeros(3 * OW * OH, device="cuda")
    cov = torch.zeros(OW * OH, dtype=torch.uint8, device="cuda")
    G.gsfit_reproject(t(rgb.reshape(-1)), t(d32), W, H, inv32, pos32, pv32, OW, OH, clip, zbuf, out, cov)
    torch.cuda.synchronize()
    c = clip.cpu().numpy().reshape(-1, 4).astype(np.float64)
    scale = np.abs(ref["clip"]).max(axis=1, keepdims=True)
    assert np.all(np.abs(c - ref["clip"]) <= 2e-5 * scale + 1e-6)
    ok = ~ref["ambiguous"]
    assert ok.mean() > 0.97
    np.testing.assert_array_equal(cov.cpu().numpy().astype(bool)[ok], ref["covered"][ok])
    np.testing.assert_array_equal(out.cpu().numpy().reshape(3, -1)[:, ok], ref["out_rgb"][:, ok])
    assert 0.3 < ref["covered"].mean() < 1.0  # some pixels disoccluded or out of view
