"""Seeded synthetic inputs for the periphery fit step.

The paper's own data (CT scans rendered by a path tracer, Section 5.1) are not
available, so every input here is synthetic and seeded. This module is shared
by the GPU path, the oracle and the benchmarks; it holds no arithmetic of the
fit step itself (no projection, compositing, loss or optimiser math), only
random draws, the procedural CT volume of the CT-derived scenes, its transfer
function, and camera poses.

Every generator uses numpy's counter-based Philox bit generator keyed by the
caller's seed. Seeds follow one scheme: scene ``s``, target set ``s + 1``,
cameras ``s + 2``, backgrounds ``s + 3``.

Gaussian sets are returned as dicts of float32 arrays (float32 is the storage
precision of the fitted parameters):

    means (N, 3), log_scales (N, 3), quats (N, 4) as (w, x, y, z),
    opacity_logits (N,), sh (N, K, 3) with K = (degree + 1)**2

Cameras are returned as dicts of arrays over V views:

    viewmat (V, 3, 4) float32, world -> camera, rows are the camera's
        right (+x), down (+y) and forward (+z) axes, last column t = -R c
    campos (V, 3) float32, camera centre c in world coordinates
    fx, fy, cx, cy, near (V,) float32; width, height (V,) int32

The pixel-centre convention is the 3DGS one: the principal point of a
centred camera is (W/2 - 0.5, H/2 - 0.5) and pixel (px, py) samples the image
plane at integer coordinates (px, py).
"""
from __future__ import annotations

import math

import numpy as np

# Zeroth-band real spherical-harmonic constant 1/(2 sqrt(pi)): converts a
# target base colour into the DC coefficient of a Gaussian (colour = C0 k0 + 0.5).
SH_C0 = 0.5 / math.sqrt(math.pi)


def rng(seed: int) -> np.random.Generator:
    """Counter-based generator (Philox 4x64) keyed by ``seed``."""
    return np.random.Generator(np.random.Philox(key=int(seed)))


# ---------------------------------------------------------------------------
# Gaussian sets
# ---------------------------------------------------------------------------

def random_gaussians(n: int, sh_degree: int, seed: int, *,
                     extent: float = 1.0,
                     log_scale_mean: float = -3.5, log_scale_std: float = 0.5,
                     higher_band_std: float = 0.05) -> dict:
    """The uniform-cube Gaussian set of the plain single-view and
    differentiation scenes: means ~ U[-extent, extent]^3, log-scales
    ~ N(mean, std) per axis, rotations uniform on S^3 (normalised N(0, 1)^4),
    opacity logits ~ N(0, 1), base colours ~ U[0, 1] stored as DC
    coefficients, higher SH bands ~ N(0, higher_band_std)."""
    g = rng(seed)
    K = (sh_degree + 1) ** 2
    means = g.uniform(-extent, extent, size=(n, 3))
    log_scales = g.normal(log_scale_mean, log_scale_std, size=(n, 3))
    q = g.normal(0.0, 1.0, size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opacity_logits = g.normal(0.0, 1.0, size=(n,))
    rgb = g.uniform(0.0, 1.0, size=(n, 3))
    sh = np.zeros((n, K, 3))
    sh[:, 0, :] = (rgb - 0.5) / SH_C0
    if K > 1:
        sh[:, 1:, :] = g.normal(0.0, higher_band_std, size=(n, K - 1, 3))
    return {
        "means": means.astype(np.float32),
        "log_scales": log_scales.astype(np.float32),
        "quats": q.astype(np.float32),
        "opacity_logits": opacity_logits.astype(np.float32),
        "sh": sh.astype(np.float32),
    }


def sh_degree_of(gaussians: dict) -> int:
    K = gaussians["sh"].shape[1]
    d = int(round(math.sqrt(K))) - 1
    assert (d + 1) ** 2 == K, K
    return d


def num_gaussians(gaussians: dict) -> int:
    return int(gaussians["means"].shape[0])


# ---------------------------------------------------------------------------
# Cameras
# ---------------------------------------------------------------------------

def _look_rotation(forward: np.ndarray, up_hint: np.ndarray) -> np.ndarray:
    """Rows (right, down, forward) of a right-handed camera frame."""
    f = forward / np.linalg.norm(forward)
    if abs(float(np.dot(f, up_hint))) > 0.99 * np.linalg.norm(up_hint):
        up_hint = np.array([0.0, 1.0, 0.0]) if abs(f[1]) < 0.9 else np.array([1.0, 0.0, 0.0])
    down = -(up_hint - np.dot(up_hint, f) * f)
    down /= np.linalg.norm(down)
    right = np.cross(down, f)
    return np.stack([right, down, f])


def _rotate(v: np.ndarray, axis: np.ndarray, angle: float) -> np.ndarray:
    """Rodrigues rotation of v about a unit axis."""
    a = axis / np.linalg.norm(axis)
    return (v * math.cos(angle) + np.cross(a, v) * math.sin(angle)
            + a * np.dot(a, v) * (1.0 - math.cos(angle)))


def make_camera(position, target, width: int, height: int, *, fx: float,
                fy: float | None = None, forward=None, up=(0.0, 0.0, 1.0),
                near: float = 0.2) -> dict:
    """One centred pinhole camera. Looks at ``target`` unless an explicit
    ``forward`` direction is given."""
    c = np.asarray(position, dtype=np.float64)
    fwd = (np.asarray(target, dtype=np.float64) - c) if forward is None else np.asarray(forward, np.float64)
    R = _look_rotation(fwd, np.asarray(up, dtype=np.float64))
    t = -R @ c
    vm = np.concatenate([R, t[:, None]], axis=1)
    return {
        "viewmat": vm.astype(np.float32),
        "campos": c.astype(np.float32),
        "fx": np.float32(fx), "fy": np.float32(fx if fy is None else fy),
        "cx": np.float32(width / 2.0 - 0.5), "cy": np.float32(height / 2.0 - 0.5),
        "near": np.float32(near),
        "width": np.int32(width), "height": np.int32(height),
    }


def stack_cameras(cams: list) -> dict:
    """List of single cameras -> dict of arrays over views."""
    keys = ["viewmat", "campos", "fx", "fy", "cx", "cy", "near", "width", "height"]
    return {k: np.stack([np.asarray(c[k]) for c in cams]) for k in keys}


def focal_for_fov(width: int, fov_deg: float) -> float:
    """Focal length in pixels for a horizontal field of view."""
    return width / (2.0 * math.tan(math.radians(fov_deg) / 2.0))


def unit_sphere_points(n: int, seed: int) -> np.ndarray:
    g = rng(seed)
    p = g.normal(size=(n, 3))
    return p / np.linalg.norm(p, axis=1, keepdims=True)


def orbit_cameras(n_views: int, width: int, height: int, fov_deg: float,
                  distance: float, seed: int, near: float = 0.2) -> dict:
    """Cameras uniformly placed on a sphere, looking at the origin."""
    pts = unit_sphere_points(n_views, seed) * distance
    fx = focal_for_fov(width, fov_deg)
    return stack_cameras([make_camera(p, (0, 0, 0), width, height, fx=fx, near=near) for p in pts])


def periphery_batch_cameras(seed: int, *, n_crops: int = 14, periphery_size: int = 1920,
                            periphery_fov_deg: float = 100.0, baseline: float = 0.064,
                            distance: float = 3.0, crop_min: int = 256, crop_max: int = 768,
                            px_per_20deg: float = 512.0, max_gaze_deg: float = 20.0,
                            near: float = 0.2) -> dict:
    """The batched-views workload: two stereo periphery frames (eyes
    +-baseline/2 about a head at ``distance`` looking at the origin) plus
    foveal crops of uneven size at the foveal angular density of 512 px per
    20 degrees, whose gaze is offset by yaw/pitch ~ U[-20, 20] degrees and
    which are rendered from alternating eyes."""
    g = rng(seed)
    head = unit_sphere_points(1, seed)[0] * distance
    fwd = -head / np.linalg.norm(head)
    R = _look_rotation(fwd, np.array([0.0, 0.0, 1.0]))
    right, down = R[0], R[1]
    eyes = [head - right * baseline / 2, head + right * baseline / 2]
    fxp = focal_for_fov(periphery_size, periphery_fov_deg)
    cams = [make_camera(e, None, periphery_size, periphery_size, fx=fxp, forward=fwd,
                        up=-down, near=near) for e in eyes]
    fxf = (px_per_20deg / 2.0) / math.tan(math.radians(10.0))
    for k in range(n_crops):
        w = int(g.integers(crop_min, crop_max + 1))
        h = int(g.integers(crop_min, crop_max + 1))
        yaw = math.radians(g.uniform(-max_gaze_deg, max_gaze_deg))
        pitch = math.radians(g.uniform(-max_gaze_deg, max_gaze_deg))
        gaze = _rotate(_rotate(fwd, down, yaw), right, pitch)
        cams.append(make_camera(eyes[k % 2], None, w, h, fx=fxf, forward=gaze, up=-down, near=near))
    return stack_cameras(cams)


def foveal_crops(seed: int, n: int, stream_seed: int, *, periphery_size: int = 1920,
                 periphery_fov_deg: float = 100.0, baseline: float = 0.064, distance: float = 3.0,
                 crop_min: int = 256, crop_max: int = 768, px_per_20deg: float = 512.0,
                 max_gaze_deg: float = 20.0, near: float = 0.2) -> dict:
    """n further foveal crops for the head of periphery_batch_cameras(seed)
    (same eyes and angular density, new gaze directions and sizes), drawn
    from a stream seeded by stream_seed: the views a viewer keeps sending
    during continual refinement."""
    g = rng(stream_seed)
    head = unit_sphere_points(1, seed)[0] * distance
    fwd = -head / np.linalg.norm(head)
    R = _look_rotation(fwd, np.array([0.0, 0.0, 1.0]))
    right, down = R[0], R[1]
    eyes = [head - right * baseline / 2, head + right * baseline / 2]
    fxf = (px_per_20deg / 2.0) / math.tan(math.radians(10.0))
    cams = []
    for k in range(n):
        w = int(g.integers(crop_min, crop_max + 1))
        h = int(g.integers(crop_min, crop_max + 1))
        yaw = math.radians(g.uniform(-max_gaze_deg, max_gaze_deg))
        pitch = math.radians(g.uniform(-max_gaze_deg, max_gaze_deg))
        gaze = _rotate(_rotate(fwd, down, yaw), right, pitch)
        cams.append(make_camera(eyes[int(g.integers(0, 2))], None, w, h, fx=fxf, forward=gaze, up=-down, near=near))
    return stack_cameras(cams)


def projection_view(cams: dict, v: int, near: float = 0.2, far: float = 100.0) -> np.ndarray:
    """4x4 projection-view matrix (float64, acting on column vectors) of view
    v for the pixel convention of the cameras: a world point maps to
    ndc = ((u + 0.5) / W * 2 - 1, (v + 0.5) / H * 2 - 1) with u = fx x/z + cx,
    v = fy y/z + cy in camera space, and depth to [0, 1] with the far plane at
    z_ndc = 1."""
    W, H = float(cams["width"][v]), float(cams["height"][v])
    fx, fy, cx, cy = (float(cams[k][v]) for k in ("fx", "fy", "cx", "cy"))
    P = np.array([[2 * fx / W, 0.0, 2 * (cx + 0.5) / W - 1.0, 0.0],
                  [0.0, 2 * fy / H, 2 * (cy + 0.5) / H - 1.0, 0.0],
                  [0.0, 0.0, far / (far - near), -far * near / (far - near)],
                  [0.0, 0.0, 1.0, 0.0]])
    Vm = np.eye(4)
    Vm[:3, :] = np.asarray(cams["viewmat"][v], np.float64).reshape(3, 4)
    return P @ Vm


def concat_cameras(a: dict, b: dict) -> dict:
    return {k: np.concatenate([a[k], b[k]]) for k in a}


def camera_subset(cams: dict, idx) -> dict:
    return {k: v[idx] for k, v in cams.items()}


def num_pixels(cams: dict) -> int:
    return int(np.sum(cams["width"].astype(np.int64) * cams["height"].astype(np.int64)))


# ---------------------------------------------------------------------------
# Backgrounds, targets and cotangents
# ---------------------------------------------------------------------------

def backgrounds(n_views: int, seed: int, n_steps: int | None = None) -> np.ndarray:
    """Random per-view RGB backgrounds, U[0, 1]: (V, 3) or (steps, V, 3)."""
    g = rng(seed)
    shape = (n_views, 3) if n_steps is None else (n_steps, n_views, 3)
    return g.uniform(0.0, 1.0, size=shape).astype(np.float32)


def smooth_images(cams: dict, seed: int, channels: int = 4) -> np.ndarray:
    """Packed per-view planar images with smooth random content in [0, 1].

    Layout: view v occupies ``channels * W_v * H_v`` consecutive floats, one
    H x W plane per channel (the rgb planes followed by alpha when
    channels == 4). Used as target images where their content is irrelevant.
    """
    g = rng(seed)
    out = []
    for v in range(len(cams["width"])):
        W, H = int(cams["width"][v]), int(cams["height"][v])
        ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
        for _ in range(channels):
            a, b = g.uniform(0.5, 3.0, size=2) * 2 * math.pi
            ph = g.uniform(0, 2 * math.pi, size=2)
            plane = 0.5 + 0.25 * np.sin(a * xs / W + ph[0]) + 0.25 * np.cos(b * ys / H + ph[1])
            out.append(plane.reshape(-1))
    return np.concatenate(out).astype(np.float32)


def cotangents(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded N(0, scale^2) cotangent vector (upstream gradient)."""
    return (rng(seed).normal(0.0, scale, size=n)).astype(np.float32)


# ---------------------------------------------------------------------------
# Procedural CT volume and transfer-function seeding (CT-derived scenes)
# ---------------------------------------------------------------------------

# Piecewise-linear RGBA transfer function over HU: (HU, r, g, b, alpha).
TF_KNOTS = np.array([
    [200.0, 0.8, 0.1, 0.1, 0.0],
    [300.0, 0.8, 0.1, 0.1, 0.6],
    [1000.0, 0.9, 0.85, 0.75, 0.9],
    [1500.0, 1.0, 1.0, 1.0, 1.0],
])


def transfer_function(hu: np.ndarray) -> np.ndarray:
    """RGBA (n, 4) for HU values, linear between knots, clamped outside."""
    hu = np.asarray(hu, dtype=np.float64)
    return np.stack([np.interp(hu, TF_KNOTS[:, 0], TF_KNOTS[:, c]) for c in range(1, 5)], axis=1)


def ct_volume(shape=(256, 256, 256), seed: int = 0, *, semi_axes=(0.8, 0.6, 0.9),
              shell_voxels: int = 3, vessel_radius_voxels: float = 4.0,
              noise_hu: float = 20.0):
    """Procedural int16 CT volume in HU over x, y in [-1, 1] with isotropic
    voxels (voxel = 2 / shape[0]); z spans shape[2] voxels about 0.

    Air -1000; a soft-tissue ellipsoid (+40); a bone shell formed by the
    outermost ``shell_voxels`` voxels inside the ellipsoid, HU ~ U[1000, 1500];
    two straight vessel tubes of +300 through the interior along seeded
    directions; plus N(0, noise_hu) noise. Returns (volume[z, y, x], voxel).
    """
    g = rng(seed)
    nx, ny, nz = shape
    vox = 2.0 / nx
    ax, ay, az = semi_axes
    xs = (np.arange(nx) + 0.5) * vox - 1.0
    ys = (np.arange(ny) + 0.5) * vox - ny * vox / 2
    zs = (np.arange(nz) + 0.5) * vox - nz * vox / 2
    inner = (ax - shell_voxels * vox, ay - shell_voxels * vox, az - shell_voxels * vox)
    # vessel axes: points near the centre, random directions
    v_pts = g.uniform(-0.2, 0.2, size=(2, 3))
    v_dir = g.normal(size=(2, 3))
    v_dir /= np.linalg.norm(v_dir, axis=1, keepdims=True)
    vol = np.empty((nz, ny, nx), dtype=np.int16)
    X, Y = np.meshgrid(xs, ys)  # (ny, nx)
    for k, z in enumerate(zs):
        q = (X / ax) ** 2 + (Y / ay) ** 2 + (z / az) ** 2
        qi = (X / inner[0]) ** 2 + (Y / inner[1]) ** 2 + (z / inner[2]) ** 2
        inside = q <= 1.0
        shell = inside & (qi > 1.0)
        hu = np.full((ny, nx), -1000.0)
        hu[inside] = 40.0
        for p, d in zip(v_pts, v_dir):
            rx, ry, rz = X - p[0], Y - p[1], z - p[2]
            along = rx * d[0] + ry * d[1] + rz * d[2]
            dist2 = rx * rx + ry * ry + rz * rz - along * along
            tube = inside & ~shell & (dist2 <= (vessel_radius_voxels * vox) ** 2)
            hu[tube] = 300.0
        hu[shell] = g.uniform(1000.0, 1500.0, size=int(shell.sum()))
        hu += g.normal(0.0, noise_hu, size=hu.shape)
        vol[k] = np.clip(np.rint(hu), -32768, 32767).astype(np.int16)
    return vol, vox


def gaussians_from_volume(vol: np.ndarray, vox: float, n: int, seed: int, *,
                          threshold_hu: float = 200.0, sh_degree: int = 3) -> dict:
    """Seed ``n`` Gaussians at voxels above ``threshold_hu``, sampled without
    replacement: mean at the voxel centre, isotropic scale of one voxel,
    identity rotation, opacity and base colour from the transfer function
    (opacity logit = logit(clamp(alpha, 0.01, 0.99))), higher SH bands zero."""
    g = rng(seed)
    nz, ny, nx = vol.shape
    flat = np.flatnonzero(vol.reshape(-1) > threshold_hu)
    if flat.size < n:
        raise ValueError(f"only {flat.size} voxels above {threshold_hu} HU, need {n}")
    pick = np.sort(g.choice(flat.size, size=n, replace=False))
    idx = flat[pick]
    iz, rem = np.divmod(idx, ny * nx)
    iy, ix = np.divmod(rem, nx)
    means = np.stack([(ix + 0.5) * vox - 1.0,
                      (iy + 0.5) * vox - ny * vox / 2,
                      (iz + 0.5) * vox - nz * vox / 2], axis=1)
    rgba = transfer_function(vol.reshape(-1)[idx].astype(np.float64))
    a = np.clip(rgba[:, 3], 0.01, 0.99)
    K = (sh_degree + 1) ** 2
    sh = np.zeros((n, K, 3))
    sh[:, 0, :] = (rgba[:, :3] - 0.5) / SH_C0
    quats = np.zeros((n, 4))
    quats[:, 0] = 1.0
    return {
        "means": means.astype(np.float32),
        "log_scales": np.full((n, 3), math.log(vox), dtype=np.float32),
        "quats": quats.astype(np.float32),
        "opacity_logits": np.log(a / (1.0 - a)).astype(np.float32),
        "sh": sh.astype(np.float32),
    }


def perturb_gaussians(gs: dict, seed: int, *, mean_std: float = 0.0, log_scale_std: float = 0.2,
                      opacity_std: float = 0.5, dc_std: float = 0.3) -> dict:
    """A perturbed copy of a Gaussian set (an imperfect starting point)."""
    g = rng(seed)
    out = {k: v.copy() for k, v in gs.items()}
    n = out["means"].shape[0]
    out["means"] += g.normal(0.0, mean_std, size=(n, 3)).astype(np.float32)
    out["log_scales"] += g.normal(0.0, log_scale_std, size=(n, 3)).astype(np.float32)
    out["opacity_logits"] += g.normal(0.0, opacity_std, size=n).astype(np.float32)
    out["sh"][:, 0, :] += g.normal(0.0, dc_std, size=(n, 3)).astype(np.float32)
    return out


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

def plain_single_view(seed: int = 0) -> dict:
    """2,000 Gaussians, SH degree 0, one 128x128 view at 60 degrees FoV from
    distance 3 (position a seeded point of the sphere), tile 16, near 0.2."""
    cams = orbit_cameras(1, 128, 128, 60.0, 3.0, seed + 2)
    return {
        "gaussians": random_gaussians(2000, 0, seed),
        "target_gaussians": random_gaussians(2000, 0, seed + 1),
        "cameras": cams,
        "bg": backgrounds(1, seed + 3),
        "tile": 16,
        "lr": 1e-3,
    }


def differentiation_scene(seed: int = 0, n: int = 50_000, size: int = 512) -> dict:
    """50,000 Gaussians with SH degree 3 (DC uniform, bands 1-3 ~ N(0, 0.05)),
    one 512x512 view at 60 degrees FoV from distance 3."""
    cams = orbit_cameras(1, size, size, 60.0, 3.0, seed + 2)
    return {
        "gaussians": random_gaussians(n, 3, seed),
        "target_gaussians": random_gaussians(n, 3, seed + 1),
        "cameras": cams,
        "bg": backgrounds(1, seed + 3),
        "tile": 16,
    }


def ct_periphery_scene(seed: int = 0, n: int = 200_000, shape=(256, 256, 256),
                       n_views: int = 24, size: int = 1024) -> dict:
    """Gaussians seeded from the procedural 256^3 CT volume through the
    transfer function; 24 orbit views of 1024^2 at distance 3, 60 degrees."""
    vol, vox = ct_volume(shape, seed)
    return {
        "gaussians": gaussians_from_volume(vol, vox, n, seed),
        "target_gaussians": gaussians_from_volume(vol, vox, n, seed + 1),
        "cameras": orbit_cameras(n_views, size, size, 60.0, 3.0, seed + 2),
        "bg": backgrounds(n_views, seed + 3),
        "tile": 16,
    }


def batched_periphery_scene(seed: int = 0, n: int = 1_000_000, shape=(512, 512, 400),
                            n_crops: int = 14) -> dict:
    """1,000,000 Gaussians from the CT procedure on a 512x512x400 volume and
    a 16-view batch: 2 stereo 1920^2 periphery frames + 14 foveal crops."""
    vol, vox = ct_volume(shape, seed)
    cams = periphery_batch_cameras(seed + 2, n_crops=n_crops)
    return {
        "gaussians": gaussians_from_volume(vol, vox, n, seed),
        "target_gaussians": gaussians_from_volume(vol, vox, n, seed + 1),
        "cameras": cams,
        "bg": backgrounds(len(cams["width"]), seed + 3),
        "tile": 16,
    }
