"""Child process of tests/test_zz_no_alloc.py (run by it, not collected by
pytest): calls gsfit_loss and gsfit_loss_noalloc through the C ABI on two
inputs, resets the device (cudaDeviceReset ends this process's context; the
next CUDA call creates a new one, into which the library's module is loaded
again), and calls both again. Prints one JSON line with the largest
differences between the two entry points in each call.

It uses no PyTorch: device buffers come from the CUDA runtime that
libgsfit.so itself links (the same shared-library instance), so the reset
and the library's calls see the same contexts."""
import ctypes
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import scenes  # noqa: E402
from paper_2601_22026_gb300 import gsfit as G  # noqa: E402

H2D, D2H = 1, 2


def loss_inputs(cams, seed):
    """Seeded render / target images in the packed layout (rgb planes,
    alpha, target rgb planes, target alpha), float32."""
    P = (np.asarray(cams["width"], np.int64) * np.asarray(cams["height"], np.int64))
    off = np.concatenate([[0], np.cumsum(P)])
    g = scenes.rng(seed)
    img = scenes.smooth_images(cams, seed + 1, channels=4)
    tgt = scenes.smooth_images(cams, seed + 2, channels=4)
    rgb, alpha, trgb, talpha = [], [], [], []
    for v in range(len(cams["width"])):
        n = int(P[v])
        a = img[4 * off[v]:4 * off[v + 1]]
        b = tgt[4 * off[v]:4 * off[v + 1]]
        rgb.append(a[:3 * n] + g.normal(0, 0.05, 3 * n).astype(np.float32))
        alpha.append(a[3 * n:])
        trgb.append(b[:3 * n])
        talpha.append(b[3 * n:])
    return [np.concatenate(x).astype(np.float32) for x in (rgb, alpha, trgb, talpha)]


def main() -> None:
    lib = G.load()
    rt = ctypes.CDLL("libcudart.so.13")  # already loaded by libgsfit.so: the same instance
    rt.cudaMalloc.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t]
    rt.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
    rt.cudaFree.argtypes = [ctypes.c_void_p]
    ok = lambda rc, what: (_ for _ in ()).throw(RuntimeError(f"{what}: cuda error {rc}")) if rc != 0 else None

    def dev(nbytes):
        p = ctypes.c_void_p()
        ok(rt.cudaMalloc(ctypes.byref(p), max(int(nbytes), 4)), "cudaMalloc")
        return p

    def put(arr):
        a = np.ascontiguousarray(arr)
        p = dev(a.nbytes)
        ok(rt.cudaMemcpy(p, a.ctypes.data, a.nbytes, H2D), "cudaMemcpy H2D")
        return p

    def get(p, n):
        a = np.empty(n, np.float32)
        ok(rt.cudaMemcpy(a.ctypes.data, p, a.nbytes, D2H), "cudaMemcpy D2H")
        return a

    cams = scenes.stack_cameras([scenes.make_camera((0, 0, 3), (0, 0, 0), w, h, fx=50.0)
                                 for w, h in [(70, 45), (33, 64), (129, 97)]])
    V = len(cams["width"])
    table = G.camera_table(cams)
    P = table.total_pixels
    out = []
    for phase in range(2):
        if phase == 1:
            ok(rt.cudaDeviceReset(), "cudaDeviceReset")
        cams_dev = put(np.frombuffer(table.as_bytes(), np.uint8))
        for seed in (101, 202):
            rgb, alpha, trgb, talpha = (put(np.asarray(x, np.float32)) for x in loss_inputs(cams, seed))
            bg = put(np.asarray(scenes.backgrounds(V, seed + 3), np.float32))
            ws = put(np.zeros(G.gsfit_loss_workspace_size(V) // 4, np.float32))
            g_ref, a_ref, L_ref = dev(12 * P), dev(4 * P), dev(4)
            g_na, a_na, L_na = dev(12 * P), dev(4 * P), dev(4)
            rc1 = lib.gsfit_loss(cams_dev, V, rgb, alpha, trgb, talpha, bg, 0.2, g_ref, a_ref, L_ref, ws,
                                 G.gsfit_loss_workspace_size(V), None)
            rc2 = lib.gsfit_loss_noalloc(cams_dev, V, rgb, alpha, trgb, talpha, bg, 0.2, g_na, a_na, L_na, None)
            ok(rt.cudaDeviceSynchronize(), "cudaDeviceSynchronize")
            Lr, Ln = float(get(L_ref, 1)[0]), float(get(L_na, 1)[0])
            gr, gn = get(g_ref, 3 * P), get(g_na, 3 * P)
            ar, an = get(a_ref, P), get(a_na, P)
            out.append({"phase": phase, "seed": seed, "rc": [int(rc1), int(rc2)], "loss": [Lr, Ln],
                        "grad_rgb_maxdiff": float(np.abs(gr - gn).max()), "grad_rgb_max": float(np.abs(gr).max()),
                        "grad_alpha_maxdiff": float(np.abs(ar - an).max())})
            for p in (rgb, alpha, trgb, talpha, bg, ws, g_ref, a_ref, L_ref, g_na, a_na, L_na):
                rt.cudaFree(p)
        rt.cudaFree(cams_dev)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
