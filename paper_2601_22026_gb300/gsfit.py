"""Thin Python binding of libgsfit.so (the C ABI in include/gsfit.h).

Argument marshalling only: every function here passes device pointers of
torch tensors, sizes and torch's current CUDA stream to the C entry point of
the same name and raises on a non-zero return. All computation happens in the
CUDA kernels of the library. Importing this module does not need a GPU;
calling a function needs the built library and a CUDA device.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _build

GSFIT_OK = 0
GSFIT_ERR_INVALID_ARG = -1
GSFIT_ERR_CAPACITY = -2
GSFIT_ERR_CUDA = -3
GSFIT_ERR_TIMEOUT = -4
GSFIT_ERR_NONFINITE = -5
GSFIT_TILE = 16
GSFIT_MAX_VIEWS = 256


def tile_order_words(total_tiles: int) -> int:
    """GSFIT_TILE_ORDER_WORDS: the heavy-first permutation, the number of
    non-empty tiles, each tile's furthest contributor, the adjoint's launch
    order and the count again."""
    return 3 * int(total_tiles) + 2


_P = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_f32 = ctypes.c_float
_size = ctypes.c_size_t


class Gaussians(ctypes.Structure):
    _fields_ = [("params", _P), ("n", _i32), ("sh_degree", _i32), ("features", _P), ("feature_dtype", _i32),
                ("reserved", _i32)]


ABI_VERSION = 10  # GSFIT_ABI_VERSION of include/gsfit.h

# gsfit_gaussians.feature_dtype values (GSFIT_FEATURES_*)
FEATURES = {"f32": 0, "f16": 1, "bf16": 2}


class Proj(ctypes.Structure):
    _fields_ = [("xyd", _P), ("conic", _P), ("rgb", _P), ("tiles", _P)]


class Camera(ctypes.Structure):
    _fields_ = [("viewmat", _f32 * 12), ("campos", _f32 * 3), ("fx", _f32), ("fy", _f32), ("cx", _f32),
                ("cy", _f32), ("near_plane", _f32), ("width", _i32), ("height", _i32), ("tile_offset", _i32),
                ("pixel_offset", _i32), ("tile", _i32), ("reserved", _i32 * 7)]


class RenderOpts(ctypes.Structure):
    """gsfit_render_opts: tile edge (8 or 16), the forward passes' batch depth
    (64, 128, 256), the half2-exponent switch (0 or 1) and the adjoint's batch
    depth (64, 128, 256); 0 selects a field's default."""
    _fields_ = [("tile", _i32), ("batch", _i32), ("exp_half2", _i32), ("batch_bwd", _i32)]


assert ctypes.sizeof(Camera) == 128

# (name, restype, argtypes) of every exported symbol
SIGNATURES = {
    "gsfit_abi_version": (ctypes.c_int, []),
    "gsfit_num_planes": (ctypes.c_int, [ctypes.c_int]),
    "gsfit_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "gsfit_camera_layout": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P]),
    "gsfit_project": (ctypes.c_int, [_P, _P, _i32, _P, _P]),
    "gsfit_bin_sort_workspace_size": (_size, [_i64, _i64, _i32]),
    "gsfit_bin_sort": (ctypes.c_int, [_P, _P, _i32, _i32, _i32, _P, _size, _P, _P, _i64, _P, _P, _P, _P, _P]),
    "gsfit_render_fwd": (ctypes.c_int, [_P, _P, _i32, _i32, _i32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "gsfit_loss_workspace_size": (_size, [_P, _i32]),
    "gsfit_loss": (ctypes.c_int, [_P, _i32, _P, _P, _P, _P, _P, _f32, _P, _P, _P, _P, _size, _P]),
    "gsfit_loss_noalloc": (ctypes.c_int, [_P, _i32, _P, _P, _P, _P, _P, _f32, _P, _P, _P, _P]),
    "gsfit_render_bwd": (ctypes.c_int, [_P, _P, _P, _i32, _i32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                        _P]),
    "gsfit_blend_bwd": (ctypes.c_int, [_P, _P, _i32, _i32, _i32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "gsfit_project_bwd": (ctypes.c_int, [_P, _P, _P, _i32, _P, _P, _P]),
    "gsfit_project_bwd_adam": (ctypes.c_int, [_P, _P, _P, _i32, _P, _P, _P, _P, _P, _f32, _f32, _f32, _P, _P,
                                              _P]),
    "gsfit_render_count": (ctypes.c_int, [_P, _P, _i32, _i32, _i32, _P, _P, _P, _P, _P, _P, _P]),
    "gsfit_render_autotune": (ctypes.c_int, [_P, _P, _i32, _i32, _i32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                             _i32, _i32, _P, _P, _P, _P]),
    "gsfit_adam_step": (ctypes.c_int, [_P, _P, _P, _P, _i32, _i32, _P, _f32, _f32, _f32, _P, _P, _i32, _P]),
    "gsfit_features_refresh": (ctypes.c_int, [_P, _i32, _i32, _P, _i32, _P]),
    "gsfit_view_is_novel": (ctypes.c_int, [_P, _P, _P, _P, _i32, _f32, _f32]),
    "gsfit_render_importance": (ctypes.c_int, [_P, _P, _i32, _i32, _i32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                               _P, _P]),
    "gsfit_simplify_workspace_size": (_size, [_i32]),
    "gsfit_simplify": (ctypes.c_int, [_P, _i32, _i32, _P, _i32, _P, _P, _P, _size, _P]),
    "gsfit_first_hit": (ctypes.c_int, [_P, _i32, _i32, _i32, _P, _f32, _P, _i32, _P, _i32, _i32, _i32, _f32, _f32,
                                       _P, _P, _P]),
    "gsfit_selftest_wait_timeout": (ctypes.c_int, [ctypes.c_int64, _P, _P]),
    "gsfit_selftest_lookback_timeout": (ctypes.c_int, [_P, _i32, _P, _P]),
    "gsfit_selftest_splat_power": (ctypes.c_int, [_P, _P, _i32, _P, _P]),
    "gsfit_selftest_alu_rate": (ctypes.c_int, [_i32, _i32, _i32, _P, _P]),
    "gsfit_reproject": (ctypes.c_int, [_P, _P, _i32, _i32, _P, _P, _P, _i32, _i32, _P, _P, _P, _P, _P]),
}

_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libgsfit.so; raises if it is missing (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not _build.LIB.exists():
        raise RuntimeError(f"libgsfit.so not built ({_build.LIB}); run paper_2601_22026_gb300.build()")
    lib = ctypes.CDLL(str(_build.LIB))
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if lib.gsfit_abi_version() != ABI_VERSION:
        raise RuntimeError("libgsfit.so ABI version mismatch")
    _lib = lib
    return lib


def _check(rc: int, what: str) -> None:
    if rc != GSFIT_OK:
        msg = load().gsfit_status_string(rc).decode()
        raise RuntimeError(f"{what} failed: {msg} ({rc})")


def _ptr(t) -> int:
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return t.data_ptr()


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------------------
# host-side layout helpers
# ---------------------------------------------------------------------------

def num_planes(sh_degree: int) -> int:
    K = (sh_degree + 1) ** 2
    return 3 + (3 * K + 3) // 4


def pack_params(gs: dict) -> np.ndarray:
    """Scene dict -> (n_planes, n, 4) float32 planes (the gsfit layout)."""
    n = gs["means"].shape[0]
    K = gs["sh"].shape[1]
    deg = int(round(K ** 0.5)) - 1
    P = np.zeros((num_planes(deg), n, 4), dtype=np.float32)
    P[0, :, 0:3] = gs["means"]
    P[0, :, 3] = gs["opacity_logits"]
    P[1] = gs["quats"]
    P[2, :, 0:3] = gs["log_scales"]
    flat = np.zeros((n, 4 * (P.shape[0] - 3)), dtype=np.float32)
    flat[:, :3 * K] = gs["sh"].reshape(n, 3 * K)
    P[3:] = flat.reshape(n, P.shape[0] - 3, 4).transpose(1, 0, 2)
    return P


def unpack_params(P: np.ndarray, sh_degree: int) -> dict:
    """(n_planes, n, 4) planes -> scene dict (also used for gradients)."""
    n = P.shape[1]
    K = (sh_degree + 1) ** 2
    flat = P[3:].transpose(1, 0, 2).reshape(n, -1)
    return {
        "means": P[0, :, 0:3].copy(),
        "opacity_logits": P[0, :, 3].copy(),
        "quats": P[1].copy(),
        "log_scales": P[2, :, 0:3].copy(),
        "sh": flat[:, :3 * K].reshape(n, K, 3).copy(),
    }


def lr_table(sh_degree: int, lr_means: float, lr_quats: float, lr_scales: float, lr_opacity: float,
             lr_sh_dc: float, lr_sh_rest: float | None = None) -> np.ndarray:
    """Per-(plane, component) learning rates in the plane layout; pads get 0."""
    K = (sh_degree + 1) ** 2
    L = np.zeros((num_planes(sh_degree), 4), dtype=np.float32)
    L[0, 0:3] = lr_means
    L[0, 3] = lr_opacity
    L[1, :] = lr_quats
    L[2, 0:3] = lr_scales
    flat = np.zeros(4 * (L.shape[0] - 3), dtype=np.float32)
    flat[0:3] = lr_sh_dc
    flat[3:3 * K] = lr_sh_dc / 20.0 if lr_sh_rest is None else lr_sh_rest
    L[3:] = flat.reshape(-1, 4)
    return L


@dataclass
class CameraTable:
    host: ctypes.Array          # Camera * V, with offsets filled in
    n_views: int
    total_tiles: int
    total_pixels: int

    def as_bytes(self) -> bytes:
        return ctypes.string_at(ctypes.addressof(self.host), ctypes.sizeof(self.host))


def camera_table(cams: dict, tile: int = GSFIT_TILE) -> CameraTable:
    """Scene camera dict -> gsfit_camera records laid out for tile edge `tile` (host)."""
    V = len(cams["width"])
    arr = (Camera * V)()
    for v in range(V):
        c = arr[v]
        vm = np.asarray(cams["viewmat"][v], dtype=np.float32).reshape(12)
        for k in range(12):
            c.viewmat[k] = float(vm[k])
        for k in range(3):
            c.campos[k] = float(cams["campos"][v][k])
        c.fx, c.fy, c.cx, c.cy = (float(cams[k][v]) for k in ("fx", "fy", "cx", "cy"))
        c.near_plane = float(cams["near"][v])
        c.width, c.height = int(cams["width"][v]), int(cams["height"][v])
    tt = ctypes.c_int32()
    tp = ctypes.c_int64()
    _check(load().gsfit_camera_layout(arr, V, int(tile), ctypes.byref(tt), ctypes.byref(tp)), "gsfit_camera_layout")
    return CameraTable(arr, V, int(tt.value), int(tp.value))


def cameras_to_device(table: CameraTable, device="cuda"):
    import torch
    buf = np.frombuffer(table.as_bytes(), dtype=np.uint8).copy()
    return torch.from_numpy(buf).to(device)


# ---------------------------------------------------------------------------
# the C entry points (same names)
# ---------------------------------------------------------------------------

@dataclass
class ProjBuffers:
    xyd: object      # float32 (V*n, 4)
    conic: object    # float32 (V*n, 4)
    rgb: object      # float32 (V*n, 4)
    tiles: object    # int32 (V*n,), read as uint32

    def struct(self) -> Proj:
        return Proj(_ptr(self.xyd), _ptr(self.conic), _ptr(self.rgb), _ptr(self.tiles))

    @staticmethod
    def allocate(n_records: int, device="cuda") -> "ProjBuffers":
        import torch
        f = lambda: torch.empty((n_records, 4), dtype=torch.float32, device=device)
        return ProjBuffers(f(), f(), f(), torch.empty(n_records, dtype=torch.int32, device=device))


def gaussians_struct(params, n: int, sh_degree: int, features=None, feature_dtype: int = 0) -> Gaussians:
    return Gaussians(_ptr(params), n, sh_degree, _ptr(features), int(feature_dtype), 0)


def gsfit_project(params, n, sh_degree, cams_dev, n_views, proj: ProjBuffers, stream=None, features=None,
                  feature_dtype=0):
    g = gaussians_struct(params, n, sh_degree, features, feature_dtype)
    p = proj.struct()
    _check(load().gsfit_project(ctypes.byref(g), _ptr(cams_dev), n_views, ctypes.byref(p), _stream(stream)),
           "gsfit_project")


def gsfit_bin_sort_workspace_size(n_records, capacity, total_tiles) -> int:
    return int(load().gsfit_bin_sort_workspace_size(n_records, capacity, total_tiles))


def gsfit_bin_sort(proj: ProjBuffers, cams_dev, n_views, n, total_tiles, ws, keys, vals, capacity, n_instances,
                   ranges, status, stream=None, tile_order=None):
    p = proj.struct()
    _check(load().gsfit_bin_sort(ctypes.byref(p), _ptr(cams_dev), n_views, n, total_tiles, _ptr(ws),
                                 ws.numel() * ws.element_size(), _ptr(keys), _ptr(vals), capacity,
                                 _ptr(n_instances), _ptr(ranges), _ptr(tile_order), _ptr(status), _stream(stream)),
           "gsfit_bin_sort")


def _opts(opts):
    """None, a RenderOpts, or a (tile, batch[, exp_half2[, batch_bwd]]) tuple -> a pointer argument."""
    if opts is None:
        return None
    if not isinstance(opts, RenderOpts):
        opts = RenderOpts(*[int(x) for x in opts])
    return ctypes.byref(opts)


def gsfit_render_fwd(proj: ProjBuffers, cams_dev, n_views, n, total_tiles, vals, ranges, bg, rgb, alpha, T_final,
                     n_contrib, stream=None, tile_order=None, status=None, opts=None):
    p = proj.struct()
    _check(load().gsfit_render_fwd(ctypes.byref(p), _ptr(cams_dev), n_views, n, total_tiles, _ptr(vals),
                                   _ptr(ranges), _ptr(tile_order), _ptr(bg), _ptr(rgb), _ptr(alpha), _ptr(T_final),
                                   _ptr(n_contrib), _opts(opts), _ptr(status), _stream(stream)),
           "gsfit_render_fwd")


def gsfit_loss_workspace_size(table) -> int:
    """Workspace bytes of gsfit_loss for a camera table (with the match flags),
    or, given a view count, for the accumulators only."""
    if isinstance(table, CameraTable):
        return int(load().gsfit_loss_workspace_size(ctypes.cast(table.host, _P), table.n_views))
    return int(load().gsfit_loss_workspace_size(None, int(table)))


def gsfit_loss(cams_dev, n_views, rgb, alpha, target_rgb, target_alpha, bg, lam, dL_drgb, dL_dalpha, loss_out, ws,
               stream=None):
    _check(load().gsfit_loss(_ptr(cams_dev), n_views, _ptr(rgb), _ptr(alpha), _ptr(target_rgb),
                             _ptr(target_alpha), _ptr(bg), float(lam), _ptr(dL_drgb), _ptr(dL_dalpha),
                             _ptr(loss_out), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)),
           "gsfit_loss")


def gsfit_loss_noalloc(cams_dev, n_views, rgb, alpha, target_rgb, target_alpha, bg, lam, dL_drgb, dL_dalpha,
                       loss_out, stream=None):
    """gsfit_loss without a workspace, for callers that cannot allocate device
    memory; its accumulators live in a fixed array inside the library (make
    the first call on a device before any stream capture; overlapping calls
    race on the shared array)."""
    _check(load().gsfit_loss_noalloc(_ptr(cams_dev), n_views, _ptr(rgb), _ptr(alpha), _ptr(target_rgb),
                                     _ptr(target_alpha), _ptr(bg), float(lam), _ptr(dL_drgb), _ptr(dL_dalpha),
                                     _ptr(loss_out), _stream(stream)),
           "gsfit_loss_noalloc")


def gsfit_render_bwd(params, n, sh_degree, proj: ProjBuffers, cams_dev, n_views, total_tiles, vals, ranges, bg,
                     T_final, n_contrib, dL_drgb, dL_dalpha, grad2d, grads, stream=None, tile_order=None,
                     status=None, features=None, feature_dtype=0, opts=None):
    g = gaussians_struct(params, n, sh_degree, features, feature_dtype)
    p = proj.struct()
    _check(load().gsfit_render_bwd(ctypes.byref(g), ctypes.byref(p), _ptr(cams_dev), n_views, total_tiles,
                                   _ptr(vals), _ptr(ranges), _ptr(tile_order), _ptr(bg), _ptr(T_final), _ptr(n_contrib),
                                   _ptr(dL_drgb), _ptr(dL_dalpha), _ptr(grad2d), _ptr(grads), _opts(opts),
                                   _ptr(status), _stream(stream)),
           "gsfit_render_bwd")


def gsfit_blend_bwd(proj: ProjBuffers, cams_dev, n_views, n, total_tiles, vals, ranges, bg, T_final, n_contrib,
                    dL_drgb, dL_dalpha, grad2d, stream=None, tile_order=None, status=None, opts=None):
    p = proj.struct()
    _check(load().gsfit_blend_bwd(ctypes.byref(p), _ptr(cams_dev), n_views, n, total_tiles, _ptr(vals), _ptr(ranges),
                                  _ptr(tile_order), _ptr(bg), _ptr(T_final), _ptr(n_contrib), _ptr(dL_drgb), _ptr(dL_dalpha),
                                  _ptr(grad2d), _opts(opts), _ptr(status), _stream(stream)),
           "gsfit_blend_bwd")


def gsfit_project_bwd(params, n, sh_degree, proj: ProjBuffers, cams_dev, n_views, grad2d, grads, stream=None,
                      features=None, feature_dtype=0):
    g = gaussians_struct(params, n, sh_degree, features, feature_dtype)
    p = proj.struct()
    _check(load().gsfit_project_bwd(ctypes.byref(g), ctypes.byref(p), _ptr(cams_dev), n_views, _ptr(grad2d),
                                    _ptr(grads), _stream(stream)),
           "gsfit_project_bwd")


def gsfit_project_bwd_adam(params, n, sh_degree, proj: ProjBuffers, cams_dev, n_views, grad2d, grads, m, v,
                           lr: np.ndarray, beta1, beta2, eps, step, stream=None, features=None, feature_dtype=0,
                           status=None):
    """The projection adjoint and Adam in one pass; params (and features)
    are updated in place; grads may be None (the gradient is then not
    written)."""
    lr = np.ascontiguousarray(lr, dtype=np.float32).reshape(-1)
    assert lr.size == 4 * num_planes(sh_degree)
    g = gaussians_struct(params, n, sh_degree, features, feature_dtype)
    p = proj.struct()
    _check(load().gsfit_project_bwd_adam(ctypes.byref(g), ctypes.byref(p), _ptr(cams_dev), n_views, _ptr(grad2d),
                                         _ptr(grads), _ptr(m), _ptr(v), lr.ctypes.data_as(_P), float(beta1),
                                         float(beta2), float(eps), _ptr(step), _ptr(status), _stream(stream)),
           "gsfit_project_bwd_adam")


def gsfit_render_count(proj: ProjBuffers, cams_dev, n_views, n, total_tiles, vals, ranges, n_contrib, count,
                       stream=None, tile_order=None, opts=None):
    p = proj.struct()
    _check(load().gsfit_render_count(ctypes.byref(p), _ptr(cams_dev), n_views, n, total_tiles, _ptr(vals),
                                     _ptr(ranges), _ptr(tile_order), _ptr(n_contrib), _ptr(count), _opts(opts),
                                     _stream(stream)),
           "gsfit_render_count")


BATCH_DEPTHS = (64, 128, 256)  # the depths gsfit_render_autotune measures, in its order


def gsfit_render_autotune(proj: ProjBuffers, cams_dev, n_views, n, total_tiles, vals, ranges, tile_order, bg, rgb,
                          alpha, T_final, n_contrib, dL_drgb, dL_dalpha, grad2d, tile, reps=3, stream=None,
                          status=None):
    """Measures every batch depth for this tile edge; returns (best RenderOpts,
    {depth: (forward ms, adjoint ms)}). Synchronises the stream."""
    p = proj.struct()
    best = RenderOpts()
    times = (ctypes.c_float * (2 * len(BATCH_DEPTHS)))()
    _check(load().gsfit_render_autotune(ctypes.byref(p), _ptr(cams_dev), n_views, n, total_tiles, _ptr(vals),
                                        _ptr(ranges), _ptr(tile_order), _ptr(bg), _ptr(rgb), _ptr(alpha),
                                        _ptr(T_final), _ptr(n_contrib), _ptr(dL_drgb), _ptr(dL_dalpha), _ptr(grad2d),
                                        int(tile), int(reps), ctypes.byref(best), times, _ptr(status),
                                        _stream(stream)),
           "gsfit_render_autotune")
    return best, {d: (times[2 * k], times[2 * k + 1]) for k, d in enumerate(BATCH_DEPTHS)}


def gsfit_adam_step(params, grads, m, v, n, n_planes, lr: np.ndarray, beta1, beta2, eps, step, stream=None,
                    features=None, feature_dtype=0):
    lr = np.ascontiguousarray(lr, dtype=np.float32).reshape(-1)
    assert lr.size == 4 * n_planes
    _check(load().gsfit_adam_step(_ptr(params), _ptr(grads), _ptr(m), _ptr(v), n, n_planes,
                                  lr.ctypes.data_as(_P), float(beta1), float(beta2), float(eps), _ptr(step),
                                  _ptr(features), int(feature_dtype), _stream(stream)),
           "gsfit_adam_step")


def gsfit_features_refresh(params, n, n_planes, features, feature_dtype, stream=None):
    _check(load().gsfit_features_refresh(_ptr(params), n, n_planes, _ptr(features), int(feature_dtype),
                                         _stream(stream)),
           "gsfit_features_refresh")


def gsfit_view_is_novel(pos_new, dir_new, pos_set, dir_set, delta_pos=0.05, theta_deg=5.0) -> bool:
    """Eq. 1 view selection (host): True if the new view is novel w.r.t. every view of the set."""
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32).reshape(-1)
    pn, dn, ps, ds = f(pos_new), f(dir_new), f(pos_set), f(dir_set)
    n = ps.size // 3
    rc = load().gsfit_view_is_novel(pn.ctypes.data_as(_P), dn.ctypes.data_as(_P), ps.ctypes.data_as(_P) if n else None,
                                    ds.ctypes.data_as(_P) if n else None, n, float(delta_pos),
                                    float(np.cos(np.deg2rad(theta_deg))))
    _check(min(rc, 0), "gsfit_view_is_novel")
    return rc == 1


def gsfit_reproject(rgb, depth, width, height, inv_pv_old, pos_old, pv_new, out_w, out_h, clip, zbuf, out_rgb,
                    covered, stream=None):
    """Depth-guided reprojection (Eqs. 2-4); matrices and pos_old are host arrays."""
    m0 = np.ascontiguousarray(inv_pv_old, dtype=np.float32).reshape(16)
    m1 = np.ascontiguousarray(pv_new, dtype=np.float32).reshape(16)
    p0 = np.ascontiguousarray(pos_old, dtype=np.float32).reshape(3)
    _check(load().gsfit_reproject(_ptr(rgb), _ptr(depth), int(width), int(height), m0.ctypes.data_as(_P),
                                  p0.ctypes.data_as(_P), m1.ctypes.data_as(_P), int(out_w), int(out_h), _ptr(clip),
                                  _ptr(zbuf), _ptr(out_rgb), _ptr(covered), _stream(stream)),
           "gsfit_reproject")


def gsfit_render_importance(proj: ProjBuffers, cams_dev, n_views, n, total_tiles, vals, ranges, bg, rgb, alpha,
                            T_final, n_contrib, importance, stream=None, tile_order=None, status=None, opts=None):
    p = proj.struct()
    _check(load().gsfit_render_importance(ctypes.byref(p), _ptr(cams_dev), n_views, n, total_tiles, _ptr(vals),
                                          _ptr(ranges), _ptr(tile_order), _ptr(bg), _ptr(rgb), _ptr(alpha),
                                          _ptr(T_final), _ptr(n_contrib), _ptr(importance), _opts(opts),
                                          _ptr(status), _stream(stream)),
           "gsfit_render_importance")


def gsfit_simplify_workspace_size(n) -> int:
    return int(load().gsfit_simplify_workspace_size(n))


def gsfit_simplify(params, n, n_planes, importance, keep, params_out, n_out, ws, stream=None):
    _check(load().gsfit_simplify(_ptr(params), n, n_planes, _ptr(importance), int(keep), _ptr(params_out),
                                 _ptr(n_out), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)),
           "gsfit_simplify")


def gsfit_first_hit(hu, nx, ny, nz, origin, voxel, tf_knots, cams_dev, n_views, rays_x, rays_y, step, alpha_min,
                    points, colour, stream=None):
    """First-hit seeding rays (Section 4.1); origin and tf_knots are host arrays."""
    o = np.ascontiguousarray(origin, dtype=np.float32).reshape(3)
    k = np.ascontiguousarray(tf_knots, dtype=np.float32).reshape(-1, 5)
    _check(load().gsfit_first_hit(_ptr(hu), int(nx), int(ny), int(nz), o.ctypes.data_as(_P), float(voxel),
                                  k.ctypes.data_as(_P), int(k.shape[0]), _ptr(cams_dev), int(n_views), int(rays_x),
                                  int(rays_y), float(step), float(alpha_min), _ptr(points), _ptr(colour),
                                  _stream(stream)),
           "gsfit_first_hit")


def gsfit_selftest_wait_timeout(limit_cycles, status, stream=None):
    _check(load().gsfit_selftest_wait_timeout(int(limit_cycles), _ptr(status), _stream(stream)),
           "gsfit_selftest_wait_timeout")


def gsfit_selftest_lookback_timeout(word, polls, status, stream=None):
    _check(load().gsfit_selftest_lookback_timeout(_ptr(word), int(polls), _ptr(status), _stream(stream)),
           "gsfit_selftest_lookback_timeout")


def gsfit_selftest_splat_power(conic, pix, n, out, stream=None):
    _check(load().gsfit_selftest_splat_power(_ptr(conic), _ptr(pix), int(n), _ptr(out), _stream(stream)),
           "gsfit_selftest_splat_power")


def gsfit_selftest_alu_rate(kind: int, blocks: int, iters: int, sink, stream=None) -> None:
    _check(load().gsfit_selftest_alu_rate(int(kind), int(blocks), int(iters), _ptr(sink), _stream(stream)),
           "gsfit_selftest_alu_rate")
