"""FP64 CPU oracle of the periphery fit step (test infrastructure).

A plain, slow, obviously-correct implementation of what the GPU path
computes, used only by the tests, the benchmark's CPU-baseline leg and the
smoke check. The product path never imports it. It shares no code with the
CUDA kernels: the C++ sources under ``oracle/src`` are compiled here into
``oracle/_build/liboracle.so`` and called through ctypes.

Conventions (Section 4.2 fits a 3DGS model; the splatting details follow
standard 3DGS): see the header comments of each C++ file. Inputs are the
float32 scene dicts of :mod:`scenes`; everything is computed in float64
except the float32 values that decide integers (depth key, depth cull, tile
rectangle), which are reproduced in float32 with a fixed operation order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "src"
LIB = HERE / "_build" / "liboracle.so"

SMOOTH = 1

# Fields of the projected record (mirror of ProjField in src/oracle.h).
PROJ_FIELDS = [
    "visible", "depth32", "u", "v", "u32", "v32", "radius",
    "conic_a", "conic_b", "conic_c", "cov_a", "cov_b", "cov_c", "opacity",
    "r", "g", "b", "clamp_r", "clamp_g", "clamp_b",
    "rect_x0", "rect_y0", "rect_x1", "rect_y1", "tiles", "near_boundary",
]
F = {name: i for i, name in enumerate(PROJ_FIELDS)}

_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle (g++, OpenMP, no FP contraction)."""
    sources = sorted(str(p) for p in SRC.glob("*.cpp"))
    headers = sorted(SRC.glob("*.h"))
    if LIB.exists() and not force:
        newest = max(os.path.getmtime(p) for p in list(map(Path, sources)) + headers)
        if os.path.getmtime(LIB) >= newest:
            return LIB
    LIB.parent.mkdir(exist_ok=True)
    tmp = LIB.with_suffix(f".{os.getpid()}.tmp")
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", str(tmp)] + sources
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(LIB))
        P = ctypes.c_void_p
        i, d, ll = ctypes.c_int, ctypes.c_double, ctypes.c_longlong
        L.oracle_set_threshold_margin.argtypes = [d]
        L.oracle_threshold_margin.restype = d
        L.oracle_proj_stride.restype = i
        L.oracle_total_tiles.argtypes = [i, P, i]
        L.oracle_total_tiles.restype = i
        L.oracle_project.argtypes = [i, i, P, i, P, i, i, P]
        L.oracle_bin.argtypes = [i, i, P, i, P, P, P, ll, P]
        L.oracle_bin.restype = ll
        L.oracle_render_fwd.argtypes = [i, i, P, i, P, P, P, P, i, P, P, P, P, P, P, P]
        L.oracle_render_bwd.argtypes = [i, i, P, i, P, i, P, P, P, P, i, P, P, P, P, P]
        L.oracle_loss.argtypes = [i, P, P, P, P, P, P, P, d, P, P, P]
        L.oracle_loss.restype = d
        L.oracle_adam.argtypes = [ll, P, P, P, P, P, d, d, d, i]
        L.oracle_real_sh.argtypes = [i, P, P, P]
        L.oracle_tiles_fwd.argtypes = [i, i, P, i, P, i, i, P, P, P, P, P, P, P, P, P, i, P]
        L.oracle_gauss_bwd.argtypes = [i, i, P, i, P, i, P, P, P, i, P, P, P]
        L.oracle_project_bwd.argtypes = [i, i, P, i, P, i, P, P, P]
        L.oracle_set_threads.argtypes = [i]
        L.oracle_max_threads.restype = i
        assert L.oracle_proj_stride() == len(PROJ_FIELDS)
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "array must be contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(lib().oracle_max_threads())


# ---------------------------------------------------------------------------
# packing of the shared scene dicts
# ---------------------------------------------------------------------------

def pack_gaussians(gs: dict) -> np.ndarray:
    n = gs["means"].shape[0]
    K = gs["sh"].shape[1]
    out = np.empty((n, 11 + 3 * K), dtype=np.float64)
    out[:, 0:3] = gs["means"]
    out[:, 3:6] = gs["log_scales"]
    out[:, 6:10] = gs["quats"]
    out[:, 10] = gs["opacity_logits"]
    out[:, 11:] = gs["sh"].reshape(n, 3 * K)
    return out


def unpack_gaussians(flat: np.ndarray, K: int) -> dict:
    n = flat.shape[0]
    return {
        "means": flat[:, 0:3].copy(),
        "log_scales": flat[:, 3:6].copy(),
        "quats": flat[:, 6:10].copy(),
        "opacity_logits": flat[:, 10].copy(),
        "sh": flat[:, 11:].reshape(n, K, 3).copy(),
    }


def pack_cameras(cams: dict) -> np.ndarray:
    V = len(cams["width"])
    out = np.zeros((V, 24), dtype=np.float64)
    out[:, 0:12] = cams["viewmat"].reshape(V, 12)
    out[:, 12:15] = cams["campos"]
    for j, k in enumerate(["fx", "fy", "cx", "cy", "near"]):
        out[:, 15 + j] = cams[k]
    out[:, 20] = cams["width"]
    out[:, 21] = cams["height"]
    return out


def pixel_offsets(cams: dict) -> np.ndarray:
    P = cams["width"].astype(np.int64) * cams["height"].astype(np.int64)
    return np.concatenate([[0], np.cumsum(P)])


def total_tiles(cams: dict, tile: int) -> int:
    c = pack_cameras(cams)
    return int(lib().oracle_total_tiles(len(c), _p(c), tile))


# ---------------------------------------------------------------------------
# stages
# ---------------------------------------------------------------------------

def project(gs: dict, cams: dict, tile: int = 16, smooth: bool = False) -> np.ndarray:
    """(V, N, len(PROJ_FIELDS)) projected records."""
    g = pack_gaussians(gs)
    c = pack_cameras(cams)
    n, K, V = g.shape[0], gs["sh"].shape[1], c.shape[0]
    proj = np.zeros((V, n, len(PROJ_FIELDS)), dtype=np.float64)
    lib().oracle_project(n, K, _p(g), V, _p(c), tile, SMOOTH if smooth else 0, _p(proj))
    return proj


def project_bwd(gs: dict, cams: dict, proj: np.ndarray, grad2d: np.ndarray, tile: int = 16) -> np.ndarray:
    """The projection adjoint alone: parameter gradients (packed Gaussian
    rows, summed over views) of the per-(view, Gaussian) 2D gradients grad2d
    (V, N, 9: u, v, a', b', c', opacity, r, g, b) at the projected records."""
    g = pack_gaussians(gs)
    c = pack_cameras(cams)
    n, K, V = g.shape[0], gs["sh"].shape[1], c.shape[0]
    out = np.zeros_like(g)
    lib().oracle_project_bwd(n, K, _p(g), V, _p(c), tile, _p(np.ascontiguousarray(proj)),
                             _p(np.ascontiguousarray(grad2d, dtype=np.float64)), _p(out))
    return out


def bin_tiles(proj: np.ndarray, cams: dict, tile: int = 16):
    """Sorted keys (uint64), values (uint32 Gaussian index), ranges (T, 2)."""
    c = pack_cameras(cams)
    V, n = proj.shape[0], proj.shape[1]
    T = total_tiles(cams, tile)
    ranges = np.zeros((T, 2), dtype=np.uint32)
    cap = int(proj[:, :, F["tiles"]].sum())
    keys = np.zeros(max(cap, 1), dtype=np.uint64)
    vals = np.zeros(max(cap, 1), dtype=np.uint32)
    cnt = lib().oracle_bin(n, V, _p(c), tile, _p(np.ascontiguousarray(proj)), _p(keys), _p(vals), cap, _p(ranges))
    assert cnt == cap
    return keys[:cnt], vals[:cnt], ranges


class threshold_margin:
    """Context manager: widen (or narrow) the relative margin within which
    render / render_bwd flag a pixel or Gaussian as ambiguous (its alpha near
    1/255 or 0.99, or its T near 1e-4). Flags only; no value changes."""

    def __init__(self, margin: float):
        self.margin = float(margin)

    def __enter__(self):
        self.prev = lib().oracle_threshold_margin()
        lib().oracle_set_threshold_margin(self.margin)
        return self

    def __exit__(self, *exc):
        lib().oracle_set_threshold_margin(self.prev)
        return False


def render(gs: dict, cams: dict, bg: np.ndarray, tile: int = 16, smooth: bool = False) -> dict:
    """Forward render. Images are packed per view: rgb (3 planes of H x W per
    view), alpha / T_final / n_contrib / ambiguous (one plane per view)."""
    proj = project(gs, cams, tile, smooth)
    keys, vals, ranges = bin_tiles(proj, cams, tile)
    c = pack_cameras(cams)
    V, n = proj.shape[0], proj.shape[1]
    P = int(pixel_offsets(cams)[-1])
    rgb = np.zeros(3 * P)
    alpha = np.zeros(P)
    T = np.zeros(P)
    nc = np.zeros(P, dtype=np.int32)
    amb = np.zeros(P, dtype=np.uint8)
    nb = np.zeros(P, dtype=np.int32)
    bgd = np.ascontiguousarray(bg, dtype=np.float64).reshape(V, 3)
    vals_c = np.ascontiguousarray(vals) if vals.size else np.zeros(1, np.uint32)
    imp = np.zeros(n)
    lib().oracle_render_fwd(n, V, _p(c), tile, _p(proj), _p(vals_c), _p(ranges), _p(bgd),
                            SMOOTH if smooth else 0, _p(rgb), _p(alpha), _p(T), _p(nc), _p(amb), _p(nb), _p(imp))
    return {"rgb": rgb, "alpha": alpha, "T_final": T, "n_contrib": nc, "ambiguous": amb.astype(bool),
            "n_blended": nb, "proj": proj, "keys": keys, "vals": vals, "ranges": ranges, "importance": imp}


def render_bwd(gs: dict, cams: dict, bg: np.ndarray, dL_drgb: np.ndarray, dL_dalpha: np.ndarray,
               tile: int = 16, smooth: bool = False, fwd: dict | None = None) -> dict:
    """Adjoint of :func:`render`: gradients of sum(dL_drgb * rgb) +
    sum(dL_dalpha * alpha) w.r.t. every parameter group."""
    if fwd is None:
        fwd = render(gs, cams, bg, tile, smooth)
    proj = fwd["proj"]
    g = pack_gaussians(gs)
    c = pack_cameras(cams)
    V, n = proj.shape[0], proj.shape[1]
    K = gs["sh"].shape[1]
    grad2d = np.zeros((V, n, 9))
    grads = np.zeros_like(g)
    amb = np.zeros((V, n), dtype=np.uint8)
    bgd = np.ascontiguousarray(bg, dtype=np.float64).reshape(V, 3)
    vals_c = np.ascontiguousarray(fwd["vals"]) if fwd["vals"].size else np.zeros(1, np.uint32)
    lib().oracle_render_bwd(n, K, _p(g), V, _p(c), tile, _p(proj), _p(vals_c), _p(fwd["ranges"]), _p(bgd),
                            SMOOTH if smooth else 0,
                            _p(np.ascontiguousarray(dL_drgb, dtype=np.float64)),
                            _p(np.ascontiguousarray(dL_dalpha, dtype=np.float64)),
                            _p(grad2d), _p(grads), _p(amb))
    return {"grads": unpack_gaussians(grads, K), "grads_flat": grads, "grad2d": grad2d,
            "gauss_ambiguous": amb.astype(bool)}


def loss(rgb, alpha, target_rgb, target_alpha, bg, cams: dict, lam: float = 0.2):
    """(loss, dL/drgb, dL/dalpha, per-view SSIM) in the packed image layout."""
    V = len(cams["width"])
    W = np.ascontiguousarray(cams["width"], dtype=np.int32)
    H = np.ascontiguousarray(cams["height"], dtype=np.int32)
    f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    rgb, alpha, target_rgb, target_alpha = f64(rgb), f64(alpha), f64(target_rgb), f64(target_alpha)
    bgd = f64(bg).reshape(V, 3)
    g_rgb = np.zeros_like(rgb)
    g_a = np.zeros_like(alpha)
    ssim = np.zeros(V)
    L = lib().oracle_loss(V, _p(W), _p(H), _p(rgb), _p(alpha), _p(target_rgb), _p(target_alpha), _p(bgd),
                          float(lam), _p(g_rgb), _p(g_a), _p(ssim))
    return L, g_rgb, g_a, ssim


def adam(p, g, m, v, lr, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-15, step: int = 1):
    """In-place Adam step on float64 arrays; lr is per element (broadcast)."""
    n = p.size
    lr_full = np.ascontiguousarray(np.broadcast_to(np.asarray(lr, dtype=np.float64), p.shape)).reshape(-1)
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    gg = np.ascontiguousarray(g, dtype=np.float64)
    lib().oracle_adam(n, _p(p), _p(gg), _p(m), _p(v), _p(lr_full), b1, b2, eps, int(step))


def real_sh(deg: int, dirs: np.ndarray):
    """Real SH basis values (n, K) and gradients (n, K, 3) at directions."""
    dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    K = (deg + 1) ** 2
    Y = np.zeros((dirs.shape[0], K))
    dY = np.zeros((dirs.shape[0], K, 3))
    for i in range(dirs.shape[0]):
        y = np.zeros(K)
        dy = np.zeros(3 * K)
        lib().oracle_real_sh(deg, _p(dirs[i].copy()), _p(y), _p(dy))
        Y[i] = y
        dY[i] = dy.reshape(K, 3)
    return Y, dY


def grad_groups_flat(K: int) -> dict:
    """Column slices of the packed Gaussian record per parameter group."""
    return {"means": slice(0, 3), "log_scales": slice(3, 6), "quats": slice(6, 10),
            "opacity_logits": slice(10, 11), "sh": slice(11, 11 + 3 * K)}


def render_tiles(gs: dict, cams: dict, bg: np.ndarray, items, tile: int = 16, max_list: int = 20000) -> dict:
    """Composite only the given (view, local tile id) items, one view at a
    time; per item B x B pixels (row-major in the tile), their blend and
    clamp counts (n_blended, n_clamped), and its sorted Gaussian list."""
    g = pack_gaussians(gs)
    c = pack_cameras(cams)
    n, K, V = g.shape[0], gs["sh"].shape[1], c.shape[0]
    it = np.ascontiguousarray(np.asarray(items, dtype=np.int32).reshape(-1, 2))
    m, B2 = it.shape[0], tile * tile
    rgb = np.zeros((m, 3, B2))
    alpha = np.zeros((m, B2))
    T = np.zeros((m, B2))
    nc = np.zeros((m, B2), dtype=np.int32)
    amb = np.zeros((m, B2), dtype=np.uint8)
    ll = np.zeros(m, dtype=np.int32)
    lists = np.zeros((m, max_list), dtype=np.uint32)
    nb = np.zeros((m, B2, 2), dtype=np.int32)
    bgd = np.ascontiguousarray(bg, dtype=np.float64).reshape(V, 3)
    lib().oracle_tiles_fwd(n, K, _p(g), V, _p(c), tile, m, _p(it), _p(bgd), _p(rgb), _p(alpha), _p(T), _p(nc),
                           _p(amb), _p(ll), _p(lists), max_list, _p(nb))
    return {"rgb": rgb, "alpha": alpha, "T_final": T, "n_contrib": nc, "ambiguous": amb.astype(bool),
            "n_blended": nb[:, :, 0], "n_clamped": nb[:, :, 1],
            "list_len": ll, "lists": [lists[k, :min(ll[k], max_list)].copy() for k in range(m)]}


def gaussian_grads(gs: dict, cams: dict, bg: np.ndarray, dL_drgb, dL_dalpha, req, tile: int = 16):
    """Complete parameter gradients (rows in the packed Gaussian layout) of
    the requested Gaussians, and their ambiguity flags."""
    g = pack_gaussians(gs)
    c = pack_cameras(cams)
    n, K, V = g.shape[0], gs["sh"].shape[1], c.shape[0]
    r = np.ascontiguousarray(np.asarray(req, dtype=np.int32))
    out = np.zeros((r.size, 11 + 3 * K))
    amb = np.zeros(r.size, dtype=np.uint8)
    bgd = np.ascontiguousarray(bg, dtype=np.float64).reshape(V, 3)
    lib().oracle_gauss_bwd(n, K, _p(g), V, _p(c), tile, _p(bgd),
                           _p(np.ascontiguousarray(dL_drgb, dtype=np.float64)),
                           _p(np.ascontiguousarray(dL_dalpha, dtype=np.float64)), r.size, _p(r), _p(out), _p(amb))
    return out, amb.astype(bool)


def view_is_novel(pos_new, dir_new, pos_set, dir_set, delta_pos: float = 0.05, theta_deg: float = 5.0) -> bool:
    """Section 4.2, Eq. 1: a new view is added to the training set only if for
    every view C_i already in it, ||pos_new - pos_i|| > delta_pos or
    view_new . view_i < cos(theta_view) (view directions as unit vectors).
    The definition written out, in float64; an empty set accepts the view."""
    p = np.asarray(pos_new, np.float64)
    d = np.asarray(dir_new, np.float64)
    d = d / np.linalg.norm(d)
    c = np.cos(np.deg2rad(theta_deg))
    for pi, di in zip(np.asarray(pos_set, np.float64).reshape(-1, 3), np.asarray(dir_set, np.float64).reshape(-1, 3)):
        di = di / np.linalg.norm(di)
        if not (np.linalg.norm(p - pi) > delta_pos or float(d @ di) < c):
            return False
    return True


def reproject(rgb, depth, W: int, H: int, inv_pv_old, pos_old, pv_new, out_w: int, out_h: int) -> dict:
    """Section 4.3, Eqs. 2-4, in float64: per source pixel (x, y) with
    uv = ((x + 0.5) / W, (y + 0.5) / H) and linear depth d,
      p_far = (P_old V_old)^-1 (2uv - 1, 1, 1) / w,
      p_world = pos_old + d (p_far - pos_old) / |p_far - pos_old|,
      p'_clip = P_new V_new p_world;
    then each source pixel is carried to the output pixel nearest its
    projected centre (w > 0), the smallest w winning, ties to the lower index.
    Returns clip (W*H, 4), out_rgb (3, out_w*out_h), covered, and `ambiguous`
    output pixels whose winner could differ in float32: a source landing within
    1e-3 px of a rounding boundary next to them, or a runner-up w within 1e-5."""
    rgb = np.asarray(rgb, np.float64).reshape(3, -1)
    d = np.asarray(depth, np.float64).reshape(-1)
    n = W * H
    y, x = np.divmod(np.arange(n), W)
    ndc = np.stack([2 * (x + 0.5) / W - 1, 2 * (y + 0.5) / H - 1, np.ones(n), np.ones(n)])
    h = np.asarray(inv_pv_old, np.float64) @ ndc
    p_far = h[:3] / h[3]
    pos = np.asarray(pos_old, np.float64).reshape(3, 1)
    ray = p_far - pos
    p_world = pos + ray / np.linalg.norm(ray, axis=0) * d
    clip = np.asarray(pv_new, np.float64) @ np.vstack([p_world, np.ones(n)])
    ok = (d > 0) & np.isfinite(d)
    clip[:, ~ok] = 0.0
    out_rgb = np.zeros((3, out_w * out_h))
    covered = np.zeros(out_w * out_h, bool)
    ambiguous = np.zeros(out_w * out_h, bool)
    best_w = np.full(out_w * out_h, np.inf)
    second_w = np.full(out_w * out_h, np.inf)
    best_src = np.full(out_w * out_h, -1)
    for k in range(n):  # plain per-source loop (small images only)
        c = clip[:, k]
        if not ok[k] or not c[3] > 0:
            continue
        px = (c[0] / c[3] + 1) * 0.5 * out_w - 0.5
        py = (c[1] / c[3] + 1) * 0.5 * out_h - 0.5
        rx, ry = np.floor(px + 0.5), np.floor(py + 0.5)
        near_x = abs((px + 0.5) - np.round(px + 0.5)) < 1e-3
        near_y = abs((py + 0.5) - np.round(py + 0.5)) < 1e-3
        if near_x or near_y:  # flag every output pixel it could land on
            for ax in ([rx - 1, rx] if near_x else [rx]):
                for ay in ([ry - 1, ry] if near_y else [ry]):
                    if 0 <= ax < out_w and 0 <= ay < out_h:
                        ambiguous[int(ay) * out_w + int(ax)] = True
        if not (0 <= rx < out_w and 0 <= ry < out_h):
            continue
        t = int(ry) * out_w + int(rx)
        w = c[3]
        if w < best_w[t] or (w == best_w[t] and k < best_src[t]):
            second_w[t] = best_w[t]
            best_w[t], best_src[t] = w, k
        elif w < second_w[t]:
            second_w[t] = w
    has = best_src >= 0
    covered[has] = True
    out_rgb[:, has] = rgb[:, best_src[has]]
    with np.errstate(invalid="ignore"):  # inf - inf where a pixel has no runner-up
        close = has & np.isfinite(second_w) & (np.abs(second_w - best_w) <= 1e-5 * np.abs(best_w))
    ambiguous |= close
    return {"clip": clip.T.copy(), "out_rgb": out_rgb, "covered": covered, "ambiguous": ambiguous,
            "p_world": p_world.T.copy()}


def simplify(gs: dict, importance, keep: int) -> tuple[dict, np.ndarray]:
    """Simplification by importance: keep the Gaussians whose importance is at
    least the keep-th largest (all of them when there are at most keep; ties
    at the threshold all kept), in index order. Importance compared as float32
    values, as stored on the GPU. Returns (kept set, kept indices)."""
    imp = np.asarray(importance, np.float32)
    imp = np.where(np.isfinite(imp) & (imp > 0), imp, np.float32(0.0))
    if imp.size <= keep:
        idx = np.arange(imp.size)
    else:
        thr = np.sort(imp)[::-1][keep - 1]
        idx = np.flatnonzero(imp >= thr)
    return {k: np.asarray(v)[idx] for k, v in gs.items()}, idx


def first_hit(vol, origin, voxel: float, knots, cams: dict, rays_x: int, rays_y: int, step: float,
              alpha_min: float) -> dict:
    """Section 4.1 first-hit seeding, in float64: per view a rays_x x rays_y
    grid of rays from the camera centre through pixel ((i + 0.5) W / rays_x -
    0.5, (j + 0.5) H / rays_y - 0.5); clipped to the volume's box; samples at
    t0 + k step (k = 0 .. floor((t1 - t0) / step)); the first sample whose
    transfer-function opacity of the trilinear HU field (voxel centres at
    origin + (i + 0.5) voxel, indices clamped at the faces) reaches alpha_min
    is refined by bisection against the previous sample (or the entry point).
    Returns points (R, 4: x, y, z, hit), colour (R, 4) and `ambiguous` rays
    whose float32 march could decide differently (a sample's opacity within
    1e-4 of alpha_min, or a sample count within rounding of the exit)."""
    vol = np.asarray(vol)
    nz, ny, nx = vol.shape
    kn = np.asarray(knots, np.float64)
    org = np.asarray(origin, np.float64)
    lo, hi = org, org + voxel * np.array([nx, ny, nz], np.float64)

    def hu_at(p):  # p (R, 3) -> trilinear HU
        c = (p - org) / voxel - 0.5
        f = np.floor(c)
        t = c - f
        i0 = f.astype(np.int64)
        out = np.zeros(len(p))
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    w = (t[:, 0] if dx else 1 - t[:, 0]) * (t[:, 1] if dy else 1 - t[:, 1]) * \
                        (t[:, 2] if dz else 1 - t[:, 2])
                    ix = np.clip(i0[:, 0] + dx, 0, nx - 1)
                    iy = np.clip(i0[:, 1] + dy, 0, ny - 1)
                    iz = np.clip(i0[:, 2] + dz, 0, nz - 1)
                    out += w * vol[iz, iy, ix]
        return out

    def tf(hu, c):
        return np.interp(hu, kn[:, 0], kn[:, c])

    pts, cols, amb = [], [], []
    for v in range(len(cams["width"])):
        W, H = float(cams["width"][v]), float(cams["height"][v])
        R = np.asarray(cams["viewmat"][v], np.float64).reshape(3, 4)[:, :3]
        j, i = np.divmod(np.arange(rays_x * rays_y), rays_x)
        u = (i + 0.5) * W / rays_x - 0.5
        w = (j + 0.5) * H / rays_y - 0.5
        dc = np.stack([(u - float(cams["cx"][v])) / float(cams["fx"][v]),
                       (w - float(cams["cy"][v])) / float(cams["fy"][v]), np.ones_like(u)], 1)
        d = dc @ R
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        o = np.asarray(cams["campos"][v], np.float64)
        with np.errstate(divide="ignore", invalid="ignore"):
            ta = (lo - o) / d
            tb = (hi - o) / d
        t0 = np.maximum(np.nanmax(np.where(d != 0, np.minimum(ta, tb), -np.inf), axis=1), 0.0)
        t1 = np.nanmin(np.where(d != 0, np.maximum(ta, tb), np.inf), axis=1)
        inside_par = np.all(np.where(d == 0, (o >= lo) & (o <= hi), True), axis=1)
        live = inside_par & (t0 <= t1)
        n_s = np.where(live, np.floor((t1 - t0) / step) + 1, 0).astype(np.int64)
        frac = (t1 - t0) / step
        a_flag = live & (np.abs(frac - np.round(frac)) < 1e-4)
        n = len(u)
        hit_t = np.full(n, np.nan)
        prev_t = t0.copy()
        done = ~live
        for k in range(int(n_s.max()) if n > 0 else 0):
            act = ~done & (k < n_s)
            if not act.any():
                break
            t = t0 + k * step
            a = tf(hu_at(o + t[act, None] * d[act]), 4)
            a_flag[np.flatnonzero(act)[np.abs(a - alpha_min) < 1e-4]] = True
            idx = np.flatnonzero(act)
            got = idx[a >= alpha_min]
            hit_t[got] = t[got]
            done[got] = True
            prev_t[idx[a < alpha_min]] = t[idx[a < alpha_min]]
            done |= ~done & (k + 1 >= n_s)
        hit = ~np.isnan(hit_t)
        a_lo, b_hi = prev_t[hit], hit_t[hit]
        for _ in range(50):
            m = 0.5 * (a_lo + b_hi)
            up = tf(hu_at(o + m[:, None] * d[hit]), 4) >= alpha_min
            b_hi = np.where(up, m, b_hi)
            a_lo = np.where(up, a_lo, m)
        p = np.zeros((n, 4))
        c = np.zeros((n, 4))
        hp = o + b_hi[:, None] * d[hit]
        p[hit, :3], p[hit, 3] = hp, 1.0
        hu_h = hu_at(hp)
        c[hit] = np.stack([tf(hu_h, 1), tf(hu_h, 2), tf(hu_h, 3), tf(hu_h, 4)], 1)
        pts.append(p)
        cols.append(c)
        amb.append(a_flag)
    return {"points": np.concatenate(pts), "colour": np.concatenate(cols), "ambiguous": np.concatenate(amb)}
