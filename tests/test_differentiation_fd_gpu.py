"""The differentiation workload (50,000 Gaussians, SH degree 3, one 512^2
view): the GPU adjoint, called through the autograd function, against
central finite differences of the FP64 oracle's render on 64 seeded
Gaussians.

The differences are of the function the GPU computes (the normal mode: 1/255
skip, 0.99 clamp, T stop, tile lists), so they are taken only where none of
its decisions moves between theta - h and theta + h: the same tile lists,
contributor counts, blend counts and clamp counts at every pixel of the
Gaussian's tiles and a one-tile margin around them (the oracle's sampled
render of those tiles, on the Gaussians whose tiles reach them: the other
Gaussians cannot change these pixels). The loss is <w, image> for a fixed
random cotangent w. h = 1e-3 for every parameter but the means: the normal
mode composites at the float32 splat centre, a staircase in the mean, and
h = 1e-4 keeps a mean's step within a splat's smooth range while moving the
centre by ~0.015 px, 500 float32 steps (so the difference carries ~2e-3
relative noise, the means' tolerance)."""
import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F = oracle.F
# (group, index within the Gaussian's row of that group)
PARAMS = [("means", (0,)), ("means", (1,)), ("means", (2,)),
          ("log_scales", (0,)), ("log_scales", (1,)), ("log_scales", (2,)),
          ("quats", (0,)), ("quats", (1,)), ("quats", (2,)), ("quats", (3,)),
          ("opacity_logits", ()), ("sh", (0, 0)), ("sh", (0, 1)), ("sh", (3, 2))]
TOL = {"means": 5e-3, "log_scales": 1e-3, "quats": 1e-3, "opacity_logits": 1e-3, "sh": 1e-3}


def test_autograd_gradient_matches_central_differences_on_64_gaussians():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2601_22026_gb300 as pkg
    from paper_2601_22026_gb300 import gsfit as G
    from paper_2601_22026_gb300.fit import FitState, render
    pkg.build()
    sc = scenes.differentiation_scene(0)
    gs, cams, bg = sc["gaussians"], sc["cameras"], sc["bg"]
    W, H = int(cams["width"][0]), int(cams["height"][0])
    P, txn, tyn = W * H, -(-W // 16), -(-H // 16)
    w_rgb = scenes.cotangents(3 * P, 811, 1e-3)
    w_a = scenes.cotangents(P, 812, 1e-3)
    # GPU: the autograd function's gradient of <w, image>
    st = FitState(gs, cams, bg=bg)
    params = st.params.clone().requires_grad_(True)
    rgb, alpha = render(params, st)
    (rgb * torch.from_numpy(w_rgb).cuda()).sum().add_((alpha * torch.from_numpy(w_a).cuda()).sum()).backward()
    gpu = G.unpack_params(params.grad.cpu().numpy(), 3)
    # the 64 Gaussians: seeded among those whose gradient is above the median
    # (most of this dense scene lies behind opaque splats and has none), whose
    # tiles span at most 3 x 3, and without a near-threshold decision
    w64, wa64 = w_rgb.astype(np.float64), w_a.astype(np.float64)
    ref = oracle.render_bwd(gs, cams, bg, w64, wa64)
    proj = oracle.project(gs, cams)[0]
    amb = ref["gauss_ambiguous"][0] | (proj[:, F["near_boundary"]] > 0)
    gn = np.linalg.norm(ref["grads_flat"], axis=1)
    cand = np.flatnonzero((proj[:, F["tiles"]] > 0) & (proj[:, F["tiles"]] <= 9) & ~amb)
    cand = cand[gn[cand] > np.median(gn[cand])]
    req = scenes.rng(813).choice(cand, 64, replace=False)
    g64 = {k: np.asarray(v, np.float64) for k, v in gs.items()}
    fd, an_gpu, an_ref = {k: [] for k in TOL}, {k: [] for k in TOL}, {k: [] for k in TOL}
    checked = total = 0
    for i in req:
        x0, y0, x1, y1 = (int(proj[i, F[k]]) for k in ("rect_x0", "rect_y0", "rect_x1", "rect_y1"))
        rx0, ry0, rx1, ry1 = max(0, x0 - 1), max(0, y0 - 1), min(txn, x1 + 1), min(tyn, y1 + 1)
        sel = np.flatnonzero((proj[:, F["tiles"]] > 0) & (proj[:, F["rect_x0"]] < rx1) &
                             (proj[:, F["rect_x1"]] > rx0) & (proj[:, F["rect_y0"]] < ry1) &
                             (proj[:, F["rect_y1"]] > ry0))
        k = int(np.flatnonzero(sel == i)[0])
        sub = {name: v[sel].copy() for name, v in g64.items()}
        items = [(0, ty * txn + tx) for ty in range(ry0, ry1) for tx in range(rx0, rx1)]
        pix = np.array([[(t // txn * 16 + q // 16) * W + t % txn * 16 + q % 16 for q in range(256)]
                        for _, t in items])
        inside = (pix % W < W) & (pix // W < H)

        def f():
            r = oracle.render_tiles(sub, cams, bg, items)
            val = 0.0
            for m in range(len(items)):
                ok = inside[m] & (r["n_contrib"][m] >= 0)
                for ch in range(3):
                    val += w64[ch * P + pix[m][ok]] @ r["rgb"][m, ch][ok]
                val += wa64[pix[m][ok]] @ r["alpha"][m][ok]
            sig = (r["n_contrib"].tobytes(), r["n_blended"].tobytes(), r["n_clamped"].tobytes(),
                   b"".join(x.tobytes() for x in r["lists"]))
            return val, sig

        _, sig0 = f()
        for name, idx in PARAMS:
            total += 1
            h = 1e-4 if name == "means" else 1e-3
            at = (k,) + idx
            old = sub[name][at]
            sub[name][at] = old + h
            fp, sp = f()
            sub[name][at] = old - h
            fm, sm = f()
            sub[name][at] = old
            if sp != sig0 or sm != sig0:
                continue  # a decision moved within +-h: not differentiable there
            checked += 1
            fd[name].append((fp - fm) / (2 * h))
            an_gpu[name].append(float(np.asarray(gpu[name])[(i,) + idx]))
            an_ref[name].append(float(np.asarray(ref["grads"][name])[(i,) + idx]))
    print(f"\nfinite differences on 64 Gaussians: {checked} of {total} parameters checked")
    for name, tol in TOL.items():
        a, b, o = np.array(an_gpu[name]), np.array(fd[name]), np.array(an_ref[name])
        share = 0.25 if name == "means" else 0.5
        assert len(b) >= share * 64 * sum(1 for n, _ in PARAMS if n == name), (name, len(b))
        err = np.linalg.norm(a - b) / np.linalg.norm(b)
        err_o = np.linalg.norm(o - b) / np.linalg.norm(b)
        print(f"  {name:15s} n={len(b):4d}  GPU vs FD {err:.2e}  oracle vs FD {err_o:.2e}")
        assert err <= tol, (name, err)
    assert checked >= 0.6 * total
