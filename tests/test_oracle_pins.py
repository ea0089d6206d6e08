"""Pins of the FP64 oracle against facts fixed by the mathematics: closed
forms, library routines, invariants, brute force on tiny inputs and finite
differences. These run on the CPU (no GPU)."""
import math

import numpy as np
import pytest

import oracle
import scenes

F = oracle.F


def _camera_on_axis(W=128, H=128, fov=60.0, dist=3.0):
    """Camera at (0, 0, dist) looking at the origin: R = diag(1, -1, -1)."""
    fx = scenes.focal_for_fov(W, fov)
    return scenes.stack_cameras([scenes.make_camera((0, 0, dist), (0, 0, 0), W, H, fx=fx)])


def _gaussians(means, log_scales, quats=None, logits=None, rgb=None, K=1, dtype=np.float32):
    means = np.atleast_2d(np.asarray(means, dtype=np.float64))
    n = means.shape[0]
    ls = np.broadcast_to(np.asarray(log_scales, dtype=np.float64), (n, 3)).copy()
    q = np.tile([1.0, 0, 0, 0], (n, 1)) if quats is None else np.atleast_2d(np.asarray(quats, np.float64))
    lg = np.zeros(n) if logits is None else np.broadcast_to(np.asarray(logits, np.float64), (n,)).copy()
    col = np.full((n, 3), 0.5) if rgb is None else np.broadcast_to(np.asarray(rgb, np.float64), (n, 3))
    sh = np.zeros((n, K, 3))
    sh[:, 0, :] = (col - 0.5) / scenes.SH_C0
    return {"means": means.astype(dtype), "log_scales": ls.astype(dtype), "quats": q.astype(dtype),
            "opacity_logits": lg.astype(dtype), "sh": sh.astype(dtype)}


# ---------------------------------------------------------------------------
# projection: closed forms
# ---------------------------------------------------------------------------

def test_isotropic_on_axis_closed_form():
    """Isotropic s = 0.03 at the origin seen from distance 3 through a
    128 px, 60 degree camera: Sigma' = ((fx s / 3)^2 + 0.3) I = 1.52880 I."""
    cams = _camera_on_axis()
    fx = 128 / (2 * math.tan(math.radians(30)))
    assert abs(fx - 110.85125168) < 1e-6
    q = scenes.random_gaussians(1, 0, 5)["quats"]  # any rotation: isotropic
    gs = _gaussians([[0, 0, 0]], math.log(0.03), quats=q)
    p = oracle.project(gs, cams)[0, 0]
    s = float(np.float32(math.log(0.03)))
    sig2 = (fx * math.exp(s) / 3.0) ** 2 + 0.3
    assert abs(sig2 - 1.52880) < 1e-4
    assert p[F["cov_a"]] == pytest.approx(sig2, rel=1e-6)
    assert p[F["cov_c"]] == pytest.approx(sig2, rel=1e-6)
    assert abs(p[F["cov_b"]]) < 1e-6
    assert p[F["conic_a"]] == pytest.approx(1 / sig2, rel=1e-6)
    # lambda_max = mid + sqrt(max(0.1, mid^2 - det)) = sigma'^2 + sqrt(0.1) here
    assert p[F["radius"]] == math.ceil(3 * math.sqrt(sig2 + math.sqrt(0.1))) == 5
    assert p[F["u"]] == pytest.approx(63.5) and p[F["v"]] == pytest.approx(63.5)
    # rect from u = 63.5, r = 5, tile 16: x0 = floor(58.5/16) = 3, x1 = floor(83.5/16) = 5
    assert (p[F["rect_x0"]], p[F["rect_x1"]], p[F["rect_y0"]], p[F["rect_y1"]]) == (3, 5, 3, 5)
    assert p[F["tiles"]] == 4


def test_anisotropic_axes_and_quaternion_convention():
    """Identity rotation: Sigma' = diag((fx sx/3)^2, (fy sy/3)^2) + 0.3 I.
    A +90 degree rotation about z, q = (cos 45, 0, 0, sin 45), maps e_x to
    e_y and therefore swaps the two image-plane variances."""
    cams = _camera_on_axis()
    fx = float(cams["fx"][0])
    sx, sy, sz = 0.02, 0.05, 0.01
    ls = np.log([sx, sy, sz])
    c = math.sqrt(0.5)
    gs = _gaussians([[0, 0, 0], [0, 0, 0]], ls, quats=[[1, 0, 0, 0], [c, 0, 0, c]])
    p = oracle.project(gs, cams)[0]
    sxf, syf = np.exp(np.float32(ls[:2]).astype(np.float64))
    a_exp, c_exp = (fx * sxf / 3) ** 2 + 0.3, (fx * syf / 3) ** 2 + 0.3
    assert p[0, F["cov_a"]] == pytest.approx(a_exp, rel=1e-6)
    assert p[0, F["cov_c"]] == pytest.approx(c_exp, rel=1e-6)
    assert p[1, F["cov_a"]] == pytest.approx(c_exp, rel=1e-5)
    assert p[1, F["cov_c"]] == pytest.approx(a_exp, rel=1e-5)


def test_off_axis_centre_and_depth():
    """Camera at (0, 0, 3) looking at the origin has R = diag(1, -1, -1):
    t = (x, -y, 3 - z), u = fx x / (3 - z) + cx, v = -fy y / (3 - z) + cy."""
    cams = _camera_on_axis()
    fx = float(cams["fx"][0])
    pts = np.array([[0.3, -0.2, 0.5], [-0.7, 0.4, -0.9]])
    gs = _gaussians(pts, math.log(0.01))
    p = oracle.project(gs, cams)[0]
    for k, (x, y, z) in enumerate(pts.astype(np.float32).astype(np.float64)):
        assert p[k, F["u"]] == pytest.approx(fx * x / (3 - z) + 63.5, rel=1e-12)
        assert p[k, F["v"]] == pytest.approx(-fx * y / (3 - z) + 63.5, rel=1e-12)
        assert p[k, F["depth32"]] == pytest.approx(3 - z, rel=1e-6)


def test_depth_cull_at_near_plane():
    cams = _camera_on_axis(dist=1.0)
    gs = _gaussians([[0, 0, 0.85], [0, 0, 0.75], [0, 0, 1.5]], math.log(0.01))
    p = oracle.project(gs, cams)[0]
    assert p[0, F["visible"]] == 0  # depth 0.15 <= 0.2
    assert p[1, F["visible"]] == 1  # depth 0.25
    assert p[2, F["visible"]] == 0  # behind the camera


def test_covariance_symmetric_positive_definite():
    gs = scenes.random_gaussians(500, 0, 3)
    cams = scenes.orbit_cameras(2, 96, 80, 60.0, 3.0, 4)
    p = oracle.project(gs, cams)
    vis = p[:, :, F["visible"]] > 0
    a, b, c = p[:, :, F["cov_a"]][vis], p[:, :, F["cov_b"]][vis], p[:, :, F["cov_c"]][vis]
    assert np.all(a >= 0.3 - 1e-12) and np.all(c >= 0.3 - 1e-12)
    assert np.all(a * c - b * b >= 0.09 - 1e-9)
    # conic is the inverse of the covariance
    ca, cb, cc = p[:, :, F["conic_a"]][vis], p[:, :, F["conic_b"]][vis], p[:, :, F["conic_c"]][vis]
    np.testing.assert_allclose(a * ca + b * cb, 1.0, atol=1e-10)
    np.testing.assert_allclose(b * ca + c * cb, 0.0, atol=1e-10)
    np.testing.assert_allclose(b * cb + c * cc, 1.0, atol=1e-10)


# ---------------------------------------------------------------------------
# colour
# ---------------------------------------------------------------------------

def test_sh_basis_matches_scipy():
    """The oracle's real basis is sqrt(2) Re / sqrt(2) Im / Re of the complex
    spherical harmonics (Condon-Shortley phase) computed by scipy."""
    from scipy.special import sph_harm_y
    d = scenes.unit_sphere_points(40, 11)
    Y, _ = oracle.real_sh(3, d)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    k = 0
    for l in range(4):
        for m in range(-l, l + 1):
            ref = sph_harm_y(l, abs(m), theta, phi)
            if m > 0:
                expect = math.sqrt(2) * ref.real
            elif m < 0:
                expect = math.sqrt(2) * ref.imag
            else:
                expect = ref.real
            np.testing.assert_allclose(Y[:, k], expect, atol=1e-12, err_msg=f"l={l} m={m}")
            k += 1


def test_sh_orthonormal_by_quadrature():
    zs, wz = np.polynomial.legendre.leggauss(12)
    phis = np.arange(24) * 2 * np.pi / 24
    Z, PHI = np.meshgrid(zs, phis, indexing="ij")
    R = np.sqrt(1 - Z ** 2)
    d = np.stack([R * np.cos(PHI), R * np.sin(PHI), Z], -1).reshape(-1, 3)
    w = (wz[:, None] * np.full_like(PHI, 2 * np.pi / 24)).reshape(-1)
    Y, _ = oracle.real_sh(3, d)
    G = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_gradient_matches_finite_differences():
    d = scenes.unit_sphere_points(5, 12)
    Y, dY = oracle.real_sh(3, d)
    h = 1e-6
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        Yp, _ = oracle.real_sh(3, d + e)
        Ym, _ = oracle.real_sh(3, d - e)
        np.testing.assert_allclose((Yp - Ym) / (2 * h), dY[:, :, i], atol=1e-7)


def test_degree0_colour_is_affine_and_clamped():
    cams = _camera_on_axis()
    gs = _gaussians([[0, 0, 0]] * 3, math.log(0.01), rgb=[[0.25, 0.9, -0.3], [0.0, 1.0, 0.5], [0.5, 0.5, 0.5]])
    p = oracle.project(gs, cams)[0]
    C0 = 0.28209479177387814
    assert abs(C0 - 0.5 / math.sqrt(math.pi)) < 1e-15
    for k in range(3):
        for ch, name in enumerate("rgb"):
            raw = C0 * float(gs["sh"][k, 0, ch]) + 0.5
            assert p[k, F[name]] == pytest.approx(max(raw, 0.0), abs=1e-12)
            assert p[k, F["clamp_" + name]] == (1 if raw < 0 else 0)


# ---------------------------------------------------------------------------
# compositing
# ---------------------------------------------------------------------------

def test_single_gaussian_image_is_closed_form():
    """One isotropic Gaussian on the optical axis (where J J^T is isotropic)
    over a black background: every pixel equals
    c o exp(-d^2 / (2 sigma'^2)) where 1/255 <= alpha <= 0.99 and the pixel's
    tile lies in the rectangle, and exactly 0 elsewhere; alpha likewise."""
    cams = _camera_on_axis()
    s, o, col = 0.05, 0.8, (0.9, 0.4, 0.2)
    gs = _gaussians([[0, 0, 0]], math.log(s), logits=math.log(o / (1 - o)), rgb=col)
    bg = np.zeros((1, 3))
    r = oracle.render(gs, cams, bg)
    p = r["proj"][0, 0]
    fx = float(cams["fx"][0])
    sf = math.exp(float(gs["log_scales"][0, 0]))
    sig2 = (fx * sf / 3.0) ** 2 + 0.3
    of = 1 / (1 + math.exp(-float(gs["opacity_logits"][0])))
    ys, xs = np.mgrid[0:128, 0:128]
    d2 = (xs - p[F["u"]]) ** 2 + (ys - p[F["v"]]) ** 2
    a = of * np.exp(-0.5 * d2 / sig2)
    tx, ty = xs // 16, ys // 16
    inrect = (tx >= p[F["rect_x0"]]) & (tx < p[F["rect_x1"]]) & (ty >= p[F["rect_y0"]]) & (ty < p[F["rect_y1"]])
    a = np.where(inrect & (a >= 1 / 255), np.minimum(a, 0.99), 0.0)
    colf = (np.asarray(gs["sh"][0, 0], np.float64) * 0.28209479177387814 + 0.5)
    img = r["rgb"].reshape(3, 128, 128)
    amb = r["ambiguous"].reshape(128, 128)
    for ch in range(3):
        np.testing.assert_allclose(img[ch][~amb], (colf[ch] * a)[~amb], atol=1e-12)
    np.testing.assert_allclose(r["alpha"].reshape(128, 128)[~amb], a[~amb], atol=1e-12)
    # integrated footprint ~ c o 2 pi sigma'^2 (tails beyond the cut are < 1%)
    total = img[0].sum()
    assert total == pytest.approx(colf[0] * of * 2 * math.pi * sig2, rel=0.02)


def test_opaque_centre_hits_alpha_clamp():
    cams = _camera_on_axis()
    gs = _gaussians([[0, 0, 0]], math.log(0.05), logits=30.0, rgb=(1.0, 0.5, 0.25))
    bg = np.array([[0.2, 0.4, 0.6]])
    r = oracle.render(gs, cams, bg)
    pix = 63 * 128 + 63  # pixel (63, 63): the centre is at (63.5, 63.5): not exact
    gs2 = _gaussians([[0, 0, 0]], math.log(0.05), logits=30.0, rgb=(1.0, 0.5, 0.25))
    cams2 = _camera_on_axis(W=127, H=127)  # centre exactly on pixel (63, 63)
    r2 = oracle.render(gs2, cams2, bg)
    pix2 = 63 * 127 + 63
    assert r2["alpha"][pix2] == pytest.approx(0.99, abs=1e-15)
    assert r2["T_final"][pix2] == pytest.approx(0.01, abs=1e-15)
    colf = np.asarray(gs2["sh"][0, 0], np.float64) * 0.28209479177387814 + 0.5
    for ch in range(3):
        assert r2["rgb"][ch * 127 * 127 + pix2] == pytest.approx(0.99 * colf[ch] + 0.01 * bg[0, ch], abs=1e-14)
    assert r["alpha"].max() <= 0.99


def test_empty_tiles_are_background_exactly():
    cams = _camera_on_axis()
    gs = _gaussians([[-0.9, 0.9, 0]], math.log(0.01))  # top-left corner
    bg = np.array([[0.3, 0.6, 0.9]])
    r = oracle.render(gs, cams, bg)
    img = r["rgb"].reshape(3, 128, 128)
    far = np.zeros((128, 128), bool)
    far[64:, 64:] = True
    for ch in range(3):
        assert np.all(img[ch][far] == np.float64(bg[0, ch]))
    assert np.all(r["n_contrib"].reshape(128, 128)[far] == 0)
    assert np.all(r["T_final"].reshape(128, 128)[far] == 1.0)


def test_equal_depth_ties_follow_index_order():
    """Two identical footprints at the same depth: the lower index is in front."""
    cams = _camera_on_axis(W=127, H=127)
    o = 0.6
    lg = math.log(o / (1 - o))
    c0, c1 = (1.0, 0.0, 0.0), (0.0, 0.0, 1.0)
    bg = np.zeros((1, 3))
    for order in [(c0, c1), (c1, c0)]:
        gs = _gaussians([[0, 0, 0], [0, 0, 0]], math.log(0.05), logits=lg, rgb=list(order))
        r = oracle.render(gs, cams, bg)
        of = 1 / (1 + math.exp(-float(gs["opacity_logits"][0])))
        pix = 63 * 127 + 63
        front = np.maximum(np.asarray(gs["sh"][0, 0], np.float64) * 0.28209479177387814 + 0.5, 0.0)
        back = np.maximum(np.asarray(gs["sh"][1, 0], np.float64) * 0.28209479177387814 + 0.5, 0.0)
        for ch in range(3):
            expect = front[ch] * of + back[ch] * of * (1 - of)
            assert r["rgb"][ch * 127 * 127 + pix] == pytest.approx(expect, abs=1e-12)


def test_transmittance_bounds_and_monotone_in_list():
    """T_final in [1e-4, 1]; adding Gaussians behind never raises alpha; the
    early stop keeps T >= 1e-4 even under many opaque layers."""
    cams = _camera_on_axis(W=64, H=48)
    n = 60
    means = np.zeros((n, 3))
    means[:, 2] = np.linspace(0.5, -0.5, n)  # increasing depth with index
    gs = _gaussians(means, math.log(0.2), logits=2.0)
    r = oracle.render(gs, cams, np.zeros((1, 3)))
    T = r["T_final"]
    assert T.min() >= 1e-4 and T.max() <= 1.0
    assert T.min() < 1e-3  # the stop rule was exercised
    prev = None
    for m in (5, 20, 60):
        sub = {k: v[:m] for k, v in gs.items()}
        a = oracle.render(sub, cams, np.zeros((1, 3)))["alpha"]
        if prev is not None:
            assert np.all(a >= prev - 1e-15)
        prev = a


def test_brute_force_keys_and_order_on_tiny_input():
    gs = scenes.random_gaussians(30, 0, 21, log_scale_mean=-2.5)
    cams = scenes.stack_cameras([
        scenes.make_camera((0, 0.5, 3), (0, 0, 0), 40, 36, fx=50.0),
        scenes.make_camera((2.5, 0, 1), (0, 0, 0), 24, 50, fx=40.0)])
    tile = 8
    proj = oracle.project(gs, cams, tile)
    keys, vals, ranges = oracle.bin_tiles(proj, cams, tile)
    pairs = []
    toff = 0
    for v in range(2):
        W, H = int(cams["width"][v]), int(cams["height"][v])
        tx_n, ty_n = -(-W // tile), -(-H // tile)
        for ty in range(ty_n):
            for tx in range(tx_n):
                t = toff + ty * tx_n + tx
                for i in range(30):
                    p = proj[v, i]
                    if not p[F["visible"]]:
                        continue
                    if p[F["rect_x0"]] <= tx < p[F["rect_x1"]] and p[F["rect_y0"]] <= ty < p[F["rect_y1"]]:
                        bits = int(np.float32(p[F["depth32"]]).view(np.uint32))
                        pairs.append((t, bits, i))
        toff += tx_n * ty_n
    pairs.sort()
    assert len(pairs) == len(keys) > 0
    assert [((t << 32) | b) for t, b, _ in pairs] == [int(k) for k in keys]
    assert [i for _, _, i in pairs] == [int(x) for x in vals]
    for t in range(toff):
        idx = [j for j, (tt, _, _) in enumerate(pairs) if tt == t]
        if idx:
            assert tuple(ranges[t]) == (idx[0], idx[-1] + 1)
        else:
            assert tuple(ranges[t]) == (0, 0)


def test_views_render_independently():
    """Rendering two views in one batch equals rendering each alone."""
    gs = scenes.random_gaussians(300, 1, 31)
    cams = scenes.stack_cameras([
        scenes.make_camera((0, 0.5, 3), (0, 0, 0), 48, 40, fx=50.0),
        scenes.make_camera((2.5, 0, 1), (0, 0, 0), 32, 56, fx=40.0)])
    bg = scenes.backgrounds(2, 5)
    both = oracle.render(gs, cams, bg)
    off = oracle.pixel_offsets(cams)
    for v in range(2):
        one = oracle.render(gs, scenes.camera_subset(cams, [v]), bg[v:v + 1])
        np.testing.assert_array_equal(both["rgb"][3 * off[v]:3 * off[v + 1]], one["rgb"])
        np.testing.assert_array_equal(both["n_contrib"][off[v]:off[v + 1]], one["n_contrib"])


# ---------------------------------------------------------------------------
# adjoint: finite differences in smooth mode
# ---------------------------------------------------------------------------

def _fd_scene(seed=7, n=16, K=16):
    """Gaussians in front of two nearby cameras with well separated depths,
    opacity well below the clamp, colours well above the clamp, inside the
    frustum: the smooth-mode render is differentiable everywhere here."""
    g = scenes.rng(seed)
    means = np.zeros((n, 3))
    means[:, 0:2] = g.uniform(-0.35, 0.35, size=(n, 2))
    means[:, 2] = np.linspace(0.6, -0.6, n) + g.uniform(-0.01, 0.01, n)
    q = g.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    sh = np.zeros((n, K, 3))
    sh[:, 0, :] = (g.uniform(0.3, 0.7, size=(n, 3)) - 0.5) / scenes.SH_C0
    sh[:, 1:, :] = g.normal(0, 0.05, size=(n, K - 1, 3))
    gs = {"means": means, "log_scales": g.normal(-2.0, 0.3, size=(n, 3)), "quats": q,
          "opacity_logits": g.normal(-1.0, 0.5, size=n), "sh": sh}
    cams = scenes.stack_cameras([
        scenes.make_camera((0, 0, 3), (0, 0, 0), 40, 32, fx=55.0),
        scenes.make_camera((0.15, 0.1, 3), (0, 0, 0), 24, 36, fx=50.0)])
    return gs, cams


def _weighted(gs, cams, bg, w_rgb, w_a):
    r = oracle.render(gs, cams, bg, tile=8, smooth=True)
    return float(w_rgb @ r["rgb"] + w_a @ r["alpha"])


def test_adjoint_matches_central_differences_smooth_mode():
    gs, cams = _fd_scene()
    bg = np.array([[0.1, 0.5, 0.9], [0.7, 0.2, 0.4]])
    P = int(oracle.pixel_offsets(cams)[-1])
    g = scenes.rng(99)
    w_rgb, w_a = g.normal(size=3 * P), g.normal(size=P)
    an = oracle.render_bwd(gs, cams, bg, w_rgb, w_a, tile=8, smooth=True)["grads"]
    h = 1e-3

    def central(flat, j, step):
        old = flat[j]
        flat[j] = old + step
        fp = _weighted(gs, cams, bg, w_rgb, w_a)
        flat[j] = old - step
        fm = _weighted(gs, cams, bg, w_rgb, w_a)
        flat[j] = old
        return (fp - fm) / (2 * step)

    checked = 0
    for name in ["means", "log_scales", "quats", "opacity_logits", "sh"]:
        flat = gs[name].reshape(-1)
        idx = list(range(flat.size)) if name != "sh" else list(range(0, flat.size, 5))
        fd_h = np.array([central(flat, j, h) for j in idx])
        fd_h2 = np.array([central(flat, j, h / 2) for j in idx])
        a = an[name].reshape(-1)[idx]
        # plain central differences at h = 1e-3: O(h^2) truncation only
        err = np.linalg.norm(a - fd_h) / np.linalg.norm(fd_h)
        assert err < 2e-5, (name, err)
        # Richardson extrapolation removes the h^2 term: agreement to O(h^4)
        rich = (4 * fd_h2 - fd_h) / 3
        err_r = np.linalg.norm(a - rich) / np.linalg.norm(rich)
        assert err_r < 1e-8, (name, err_r)
        checked += len(idx)
    assert checked > 300


def _clamp_and_stop_scene(seed=123):
    """One 48 x 40 view (tile 8) with: a wide, nearly opaque Gaussian in
    front (o = 0.9999) whose o G exceeds the 0.99 clamp at about ten pixels
    around its centre; six wide layers (o ~ 0.86 - 0.92) behind it at well
    separated depths, under which about ninety pixels stop early (the next
    blend would take T below 1e-4); ten small Gaussians spread across the
    view at depths in between. SH degree 1."""
    cams = scenes.stack_cameras([scenes.make_camera((0, 0, 3), (0, 0, 0), 48, 40, fx=60.0)])
    g = scenes.rng(seed)
    means = [(0.2, 0.08, 0.8)]
    ls = [(math.log(0.5), math.log(0.42), math.log(0.46))]
    logit = [9.2]
    for k in range(6):
        means.append((g.uniform(-0.08, 0.08), g.uniform(-0.08, 0.08), 0.5 - 0.15 * k))
        ls.append(tuple(np.log(g.uniform(0.28, 0.4, 3))))
        logit.append(g.uniform(1.8, 2.4))
    n_small = 10
    means += [tuple(x) for x in np.c_[g.uniform(-0.55, 0.55, (n_small, 2)), np.linspace(0.65, -0.6, n_small) + 0.01]]
    ls += [tuple(x) for x in g.normal(-2.6, 0.25, (n_small, 3))]
    logit += list(g.normal(-0.5, 0.8, n_small))
    n, K = len(means), 4
    q = g.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    sh = np.zeros((n, K, 3))
    sh[:, 0, :] = (g.uniform(0.25, 0.75, (n, 3)) - 0.5) / scenes.SH_C0
    sh[:, 1:, :] = g.normal(0, 0.05, (n, K - 1, 3))
    gs = {"means": np.array(means, np.float64), "log_scales": np.array(ls, np.float64), "quats": q,
          "opacity_logits": np.array(logit, np.float64), "sh": sh}
    return gs, cams


def _splat_alpha_unclamped(proj_i, W, H):
    """o G at every pixel centre of a W x H view, from a projected record
    (the normal-mode float32 centre)."""
    yy, xx = np.mgrid[0:H, 0:W]
    dx, dy = xx - proj_i[F["u32"]], yy - proj_i[F["v32"]]
    pw = -0.5 * (proj_i[F["conic_a"]] * dx * dx + proj_i[F["conic_c"]] * dy * dy) - proj_i[F["conic_b"]] * dx * dy
    return (proj_i[F["opacity"]] * np.exp(pw)).reshape(-1)


def _stopped_pixels(r, W, H, tile):
    """Pixels whose front-to-back walk ended at the T stop (a later Gaussian
    would blend but take T below 1e-4), walked here from the oracle's own
    lists and records."""
    proj = r["proj"][0]
    tx_n = -(-W // tile)
    out = np.zeros(W * H, bool)
    for py in range(H):
        for px in range(W):
            t = (py // tile) * tx_n + px // tile
            s, e = r["ranges"][t]
            T = 1.0
            for gi in r["vals"][s:e]:
                p = proj[gi]
                dx, dy = px - p[F["u32"]], py - p[F["v32"]]
                pw = -0.5 * (p[F["conic_a"]] * dx * dx + p[F["conic_c"]] * dy * dy) - p[F["conic_b"]] * dx * dy
                if pw > 0:
                    continue
                a = min(0.99, p[F["opacity"]] * math.exp(pw))
                if a < 1 / 255:
                    continue
                if T * (1 - a) < 1e-4:
                    out[py * W + px] = True
                    break
                T *= 1 - a
    return out


def test_adjoint_matches_central_differences_normal_mode():
    """The analytic adjoint of the normal-mode render (1/255 skip, 0.99 clamp,
    T stop, tile lists) against central differences, h = 1e-4 in FP64, on a
    scene where the clamp is active at pixels of a Gaussian and pixels stop
    early. A parameter is compared wherever no decision of the render moves
    between theta - h and theta + h (same tile lists, contributor counts and
    blend counts; Gaussians with a near-threshold decision excluded): there
    the render is smooth, and the clamped alpha has zero derivative in o and
    in the exponent. Passing the gradient through the clamp (as 3DGS does)
    misses this check by a factor of about 50 in every geometric group."""
    gs, cams = _clamp_and_stop_scene()
    W, H, tile = 48, 40, 8
    bg = np.array([[0.2, 0.6, 0.4]])
    P = W * H
    g = scenes.rng(7)
    w_rgb, w_a = g.normal(size=3 * P), g.normal(size=P)

    def evaluate():
        r = oracle.render(gs, cams, bg, tile=tile)
        sig = (r["vals"].tobytes(), r["ranges"].tobytes(), r["n_contrib"].tobytes(), r["n_blended"].tobytes())
        return float(w_rgb @ r["rgb"] + w_a @ r["alpha"]), sig, r

    _, sig0, r0 = evaluate()
    # the scene exercises both branches
    clamped = _splat_alpha_unclamped(r0["proj"][0, 0], W, H) > 0.99
    assert clamped.sum() >= 5
    assert _stopped_pixels(r0, W, H, tile).sum() >= 50
    b = oracle.render_bwd(gs, cams, bg, w_rgb, w_a, tile=tile, fwd=r0)
    amb = b["gauss_ambiguous"].any(axis=0) | (r0["proj"][:, :, F["near_boundary"]] > 0).any(axis=0)
    assert not amb[0]
    h = 1e-4
    # The normal mode composites at the float32 splat centre, a staircase in
    # the mean with steps of about 2e-6 px against the 2.4e-3 px that h moves
    # the centre: the means' differences carry about 1e-3 relative noise.
    tol = {"means": 1e-3, "log_scales": 1e-6, "quats": 1e-6, "opacity_logits": 1e-6, "sh": 1e-6}
    total = checked = 0
    clamped_checked = 0
    for name in ["means", "log_scales", "quats", "opacity_logits", "sh"]:
        arr = gs[name]
        n = arr.shape[0]
        rows = arr.reshape(n, -1)
        fd, an = [], []
        for i in range(n):
            if amb[i]:
                continue
            for j in range(rows.shape[1]):
                total += 1
                old = rows[i, j]
                rows[i, j] = old + h
                fp, sp, _ = evaluate()
                rows[i, j] = old - h
                fm, sm, _ = evaluate()
                rows[i, j] = old
                if sp != sig0 or sm != sig0:
                    continue
                fd.append((fp - fm) / (2 * h))
                an.append(b["grads"][name].reshape(n, -1)[i, j])
                checked += 1
                clamped_checked += i == 0
        fd, an = np.array(fd), np.array(an)
        err = np.linalg.norm(an - fd) / np.linalg.norm(fd)
        assert err < tol[name], (name, err)
    assert checked >= 0.9 * total, (checked, total)
    assert clamped_checked >= 20  # most of the clamped Gaussian's 23 parameters


def _three_uneven_views():
    return scenes.stack_cameras([
        scenes.make_camera((0.2, 0.3, 3), (0, 0, 0), 53, 41, fx=45.0),
        scenes.make_camera((-2.0, 1.0, 2.0), (0, 0, 0), 37, 66, fx=40.0),
        scenes.make_camera((1.5, -1.5, 2.0), (0.05, 0, 0), 70, 29, fx=60.0)])


def test_sampled_entry_points_equal_full_render():
    """render_tiles (tiles composited on demand, one view at a time) and
    gaussian_grads (complete gradients of chosen Gaussians) give what the
    whole-batch render and adjoint give for the same tiles and Gaussians:
    three uneven views, tiles of the second and third view by their
    view-local ids (ragged edge tiles included), Gaussians seen in one, two
    or three views."""
    gs = scenes.random_gaussians(400, 2, 21, log_scale_mean=-2.6, extent=2.0)
    cams = _three_uneven_views()
    V, tile, B2 = 3, 16, 256
    bg = scenes.backgrounds(V, 22)
    full = oracle.render(gs, cams, bg, tile=tile)
    off = oracle.pixel_offsets(cams)
    Ws, Hs = [int(x) for x in cams["width"]], [int(x) for x in cams["height"]]
    txn = [-(-w // tile) for w in Ws]
    tyn = [-(-h // tile) for h in Hs]
    toff = np.concatenate([[0], np.cumsum([a * b for a, b in zip(txn, tyn)])])
    items = [(1, 0), (1, txn[1] * tyn[1] - 1), (1, txn[1] + 1), (2, 3), (2, txn[2] * tyn[2] - 1), (2, txn[2]),
             (0, 5)]
    got = oracle.render_tiles(gs, cams, bg, items, tile=tile)
    for k, (v, t) in enumerate(items):
        tx, ty = t % txn[v], t // txn[v]
        s, e = full["ranges"][toff[v] + t]
        np.testing.assert_array_equal(got["lists"][k], full["vals"][s:e])
        assert got["list_len"][k] == e - s
        plane = Ws[v] * Hs[v]
        for q in range(B2):
            px, py = tx * tile + q % tile, ty * tile + q // tile
            if px >= Ws[v] or py >= Hs[v]:
                assert got["n_contrib"][k, q] == -1
                continue
            pix = off[v] + py * Ws[v] + px
            for ch in range(3):
                ref = full["rgb"][3 * off[v] + ch * plane + py * Ws[v] + px]
                assert abs(got["rgb"][k, ch, q] - ref) <= 1e-12
            assert abs(got["alpha"][k, q] - full["alpha"][pix]) <= 1e-12
            assert abs(got["T_final"][k, q] - full["T_final"][pix]) <= 1e-12
            assert got["n_contrib"][k, q] == full["n_contrib"][pix]
            assert got["n_blended"][k, q] == full["n_blended"][pix]
            assert got["ambiguous"][k, q] == full["ambiguous"][pix]
    # gradients of chosen Gaussians
    P = int(off[-1])
    w_rgb = scenes.cotangents(3 * P, 23, 1.0).astype(np.float64)
    w_a = scenes.cotangents(P, 24, 1.0).astype(np.float64)
    b = oracle.render_bwd(gs, cams, bg, w_rgb, w_a, tile=tile, fwd=full)
    seen = (full["proj"][:, :, F["tiles"]] > 0).sum(axis=0)
    req = np.concatenate([np.flatnonzero(seen == c)[:4] for c in (0, 1, 2, 3)])
    assert {int(c) for c in seen[req]} == {0, 1, 2, 3}
    rows, amb = oracle.gaussian_grads(gs, cams, bg, w_rgb, w_a, req, tile=tile)
    ref = b["grads_flat"][req]
    scale = np.abs(b["grads_flat"]).max(axis=0)
    assert np.all(np.abs(rows - ref) <= 1e-12 * (np.abs(ref) + 1e-3 * scale))
    assert np.all(rows[seen[req] == 0] == 0)
    ref_amb = b["gauss_ambiguous"].any(axis=0) | (full["proj"][:, :, F["near_boundary"]] > 0).any(axis=0)
    np.testing.assert_array_equal(amb, ref_amb[req])


def test_projection_adjoint_entry_equals_the_second_half_of_render_bwd():
    """oracle.project_bwd (the projection adjoint alone, used to time the
    per-view share of an iteration) applied to render_bwd's 2D gradients
    gives render_bwd's parameter gradients."""
    gs = scenes.random_gaussians(300, 1, 31)
    cams = scenes.stack_cameras([
        scenes.make_camera((0, 0.5, 3), (0, 0, 0), 48, 40, fx=50.0),
        scenes.make_camera((2.5, 0, 1), (0, 0, 0), 32, 56, fx=40.0)])
    bg = scenes.backgrounds(2, 5)
    P = int(oracle.pixel_offsets(cams)[-1])
    g = scenes.rng(3)
    b = oracle.render_bwd(gs, cams, bg, g.normal(size=3 * P), g.normal(size=P))
    got = oracle.project_bwd(gs, cams, oracle.project(gs, cams), b["grad2d"])
    assert np.abs(b["grads_flat"]).max() > 0
    np.testing.assert_array_equal(got, b["grads_flat"])


def test_adjoint_sums_over_views():
    gs, cams = _fd_scene(seed=8)
    bg = np.array([[0.1, 0.5, 0.9], [0.7, 0.2, 0.4]])
    off = oracle.pixel_offsets(cams)
    P = int(off[-1])
    g = scenes.rng(5)
    w_rgb, w_a = g.normal(size=3 * P), g.normal(size=P)
    both = oracle.render_bwd(gs, cams, bg, w_rgb, w_a, tile=8)["grads_flat"]
    acc = np.zeros_like(both)
    for v in range(2):
        acc += oracle.render_bwd(gs, scenes.camera_subset(cams, [v]), bg[v:v + 1],
                                 w_rgb[3 * off[v]:3 * off[v + 1]], w_a[off[v]:off[v + 1]], tile=8)["grads_flat"]
    np.testing.assert_allclose(both, acc, rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------------------
# loss
# ---------------------------------------------------------------------------

def _images(cams, seed):
    g = scenes.rng(seed)
    P = int(oracle.pixel_offsets(cams)[-1])
    return g.uniform(0, 1, 3 * P), g.uniform(0, 1, P)


def _two_small_views():
    return scenes.stack_cameras([scenes.make_camera((0, 0, 3), (0, 0, 0), 17, 13, fx=20.0),
                                 scenes.make_camera((0, 0, 3), (0, 0, 0), 11, 19, fx=20.0)])


def test_loss_zero_at_identity():
    cams = _two_small_views()
    rgb, a = _images(cams, 1)
    bg = np.zeros((2, 3))
    L, grgb, ga, ssim = oracle.loss(rgb, a, rgb, a, bg, cams)
    assert L == pytest.approx(0.0, abs=1e-14)
    np.testing.assert_allclose(ssim, 1.0, atol=1e-14)
    assert np.abs(grgb).max() < 1e-13 and np.abs(ga).max() == 0.0


def test_ssim_matches_scipy_gaussian_filter():
    """Windowed moments from scipy.ndimage.gaussian_filter (sigma 1.5,
    radius 5, zero padding) give the same SSIM as the oracle."""
    from scipy.ndimage import gaussian_filter
    cams = _two_small_views()
    x, _ = _images(cams, 2)
    y, ya = _images(cams, 3)
    bg = np.zeros((2, 3))
    _, _, _, ssim = oracle.loss(x, np.zeros(len(ya)), y, np.ones(len(ya)), bg, cams)
    off = oracle.pixel_offsets(cams)
    for v in range(2):
        W, H = int(cams["width"][v]), int(cams["height"][v])
        s = 0.0
        for ch in range(3):
            sl = slice(3 * off[v] + ch * W * H, 3 * off[v] + (ch + 1) * W * H)
            X, Y = x[sl].reshape(H, W), y[sl].reshape(H, W)
            f = lambda im: gaussian_filter(im, 1.5, mode="constant", cval=0.0, truncate=5 / 1.5)
            mx, my = f(X), f(Y)
            sxx, syy, sxy = f(X * X) - mx * mx, f(Y * Y) - my * my, f(X * Y) - mx * my
            C1, C2 = 0.01 ** 2, 0.03 ** 2
            S = (2 * mx * my + C1) * (2 * sxy + C2) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
            s += S.mean()
        assert ssim[v] == pytest.approx(s / 3, abs=1e-12)


def test_loss_gradient_matches_central_differences():
    cams = _two_small_views()
    x, a = _images(cams, 4)
    y, ya = _images(cams, 5)
    bg = np.array([[0.2, 0.3, 0.4], [0.9, 0.1, 0.5]])
    L, gx, ga, _ = oracle.loss(x, a, y, ya, bg, cams)
    h = 1e-6
    g = scenes.rng(6)
    for j in g.choice(x.size, 40, replace=False):
        xp, xm = x.copy(), x.copy()
        xp[j] += h
        xm[j] -= h
        fd = (oracle.loss(xp, a, y, ya, bg, cams)[0] - oracle.loss(xm, a, y, ya, bg, cams)[0]) / (2 * h)
        assert fd == pytest.approx(gx[j], rel=1e-5, abs=1e-10)
    for j in g.choice(a.size, 10, replace=False):
        ap, am = a.copy(), a.copy()
        ap[j] += h
        am[j] -= h
        fd = (oracle.loss(x, ap, y, ya, bg, cams)[0] - oracle.loss(x, am, y, ya, bg, cams)[0]) / (2 * h)
        assert fd == pytest.approx(ga[j], rel=1e-5, abs=1e-10)


# ---------------------------------------------------------------------------
# Adam
# ---------------------------------------------------------------------------

def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    g = scenes.rng(8)
    p0 = g.normal(size=200)
    lr = np.where(np.arange(200) < 100, 1e-3, 5e-2)
    p, m, v = p0.copy(), np.zeros(200), np.zeros(200)
    tp = [torch.tensor(p0[:100].copy()), torch.tensor(p0[100:].copy())]
    for t in tp:
        t.requires_grad_(True)
    opt = torch.optim.Adam([{"params": [tp[0]], "lr": 1e-3}, {"params": [tp[1]], "lr": 5e-2}],
                           betas=(0.9, 0.999), eps=1e-15)
    for step in range(1, 4):
        grad = g.normal(size=200)
        oracle.adam(p, grad, m, v, lr, 0.9, 0.999, 1e-15, step)
        tp[0].grad = torch.tensor(grad[:100].copy())
        tp[1].grad = torch.tensor(grad[100:].copy())
        opt.step()
    np.testing.assert_allclose(p[:100], tp[0].detach().numpy(), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(p[100:], tp[1].detach().numpy(), rtol=1e-13, atol=1e-15)


def test_adam_first_step_moves_by_lr_sign():
    g = np.array([3.0, -1e-3, 0.0, 1e-9])
    p, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    oracle.adam(p, g, m, v, 1e-3, 0.9, 0.999, 1e-15, 1)
    np.testing.assert_allclose(p, -1e-3 * g / (np.abs(g) + 1e-15), rtol=1e-12, atol=0)


def test_threshold_margin_changes_flags_only():
    """Widening the near-threshold margin flags more pixels and changes no
    rendered value (it is a test aid for lower-precision forms)."""
    sc = scenes.plain_single_view(0)
    gs, cams, bg = sc["gaussians"], sc["cameras"], sc["bg"]
    a = oracle.render(gs, cams, bg)
    with oracle.threshold_margin(1e-2):
        b = oracle.render(gs, cams, bg)
    for k in ("rgb", "alpha", "T_final", "n_contrib", "n_blended"):
        np.testing.assert_array_equal(a[k], b[k])
    assert (b["ambiguous"] | ~a["ambiguous"]).all() and b["ambiguous"].sum() > a["ambiguous"].sum()
    assert oracle.lib().oracle_threshold_margin() == 2e-4
