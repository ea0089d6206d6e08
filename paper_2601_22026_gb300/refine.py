"""Continuous refinement during viewing (Section 4.2).

After the initial model, the fit keeps running on the foveal views the
viewer streams in. A new view joins the training set only when Eq. 1 calls
it novel (gsfit_view_is_novel: farther than delta_pos = 0.05 from, or turned
more than 5 degrees against, every view already in the set). The paper
simplifies continual training to periodic restarts that reload the current
Gaussians and discard the optimiser state (ContinuousRefinement.restart).

The loop keeps a fixed-size batch of V views (the periphery frames plus
foveal crops); every `replace_every` iterations the oldest `n_replace` crops
are replaced by newly streamed views that pass Eq. 1, their targets are
rendered from the target set, and the iteration is captured again as a CUDA
graph. Every arithmetic step runs in the library's kernels; this module only
moves views and buffers around.
"""
from __future__ import annotations

import numpy as np

from . import gsfit as G


SH_Y00 = 0.28209479177387814  # 1 / (2 sqrt(pi)), the constant SH basis function


def first_hit_points(vol: np.ndarray, origin, voxel: float, tf_knots, cams: dict, rays_x: int, rays_y: int,
                     step: float | None = None, alpha_min: float = 0.3):
    """First-hit seeding rays (Section 4.1) through gsfit_first_hit: the
    volume vol[z][y][x] (int16 HU) seen from the given cameras. Returns host
    (points (R, 4), colour (R, 4)) and the kernel's time in ms."""
    import torch
    nz, ny, nx = vol.shape
    table = G.camera_table(cams)
    cams_dev = G.cameras_to_device(table)
    hu = torch.from_numpy(np.ascontiguousarray(vol, dtype=np.int16).reshape(-1)).cuda()
    n = table.n_views * rays_x * rays_y
    pts = torch.empty(4 * n, device="cuda")
    col = torch.empty(4 * n, device="cuda")
    step = 0.5 * voxel if step is None else step
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    G.gsfit_first_hit(hu, nx, ny, nz, origin, voxel, tf_knots, cams_dev, table.n_views, rays_x, rays_y, step,
                      alpha_min, pts, col)
    b.record()
    torch.cuda.synchronize()
    return pts.cpu().numpy().reshape(-1, 4), col.cpu().numpy().reshape(-1, 4), a.elapsed_time(b)


def gaussians_from_hits(points: np.ndarray, colour: np.ndarray, voxel: float, sh_degree: int = 3) -> dict:
    """One Gaussian per hit: mean at the hit, isotropic scale of one voxel,
    identity rotation, opacity and base colour from the transfer function at
    the hit (opacity logit = logit(clamp(alpha, 0.01, 0.99))), higher SH bands
    zero -- the starting point the optimisation refines."""
    hit = points[:, 3] > 0
    n = int(hit.sum())
    rgba = colour[hit].astype(np.float64)
    a = np.clip(rgba[:, 3], 0.01, 0.99)
    K = (sh_degree + 1) ** 2
    sh = np.zeros((n, K, 3), np.float32)
    sh[:, 0, :] = (rgba[:, :3] - 0.5) / SH_Y00
    return {"means": points[hit, :3].astype(np.float32),
            "quats": np.tile(np.array([1.0, 0.0, 0.0, 0.0], np.float32), (n, 1)),
            "log_scales": np.full((n, 3), np.log(voxel), np.float32),
            "opacity_logits": np.log(a / (1.0 - a)).astype(np.float32),
            "sh": sh}


def camera_forward(cams: dict, v: int) -> np.ndarray:
    """World-space viewing direction of view v (third row of the rotation)."""
    return np.asarray(cams["viewmat"][v], np.float64).reshape(3, 4)[2, :3].copy()


class ViewSet:
    """The training views of continual refinement, grown by Eq. 1."""

    def __init__(self, delta_pos: float = 0.05, theta_deg: float = 5.0):
        self.delta_pos = float(delta_pos)
        self.theta_deg = float(theta_deg)
        self.pos: list[np.ndarray] = []
        self.dir: list[np.ndarray] = []

    def __len__(self) -> int:
        return len(self.pos)

    def add(self, pos, direction) -> None:
        self.pos.append(np.asarray(pos, np.float64))
        self.dir.append(np.asarray(direction, np.float64))

    def offer(self, pos, direction) -> bool:
        """Adds the view if it is novel w.r.t. every view of the set (Eq. 1)."""
        ps = np.array(self.pos).reshape(-1, 3)
        ds = np.array(self.dir).reshape(-1, 3)
        novel = G.gsfit_view_is_novel(pos, direction, ps, ds, self.delta_pos, self.theta_deg)
        if novel:
            self.add(pos, direction)
        return novel


def share_parameters(dst, src) -> None:
    """Makes FitState dst render src's Gaussians (parameters, 16-bit copy,
    optimiser state) on its own views."""
    dst.params, dst.grads, dst.m, dst.v = src.params, src.grads, src.m, src.v
    dst.step_count, dst.lr = src.step_count, src.lr
    dst.features, dst.feature_dtype = src.features, src.feature_dtype
    dst.graph = None


def view_state(src, cams: dict, bg=None, **kw):
    """A FitState on other views that renders (and, if stepped, fits) src's
    Gaussians: built around a one-Gaussian placeholder, then sharing src's
    parameters, 16-bit copy and optimiser state."""
    from .fit import FitState
    st = FitState(src.gaussians_first(), cams, bg=bg, capacity=16, tile=src.tile, batch=int(src.opts.batch),
                  batch_bwd=int(src.opts.batch_bwd), **kw)
    st.n = src.n
    share_parameters(st, src)
    st.set_cameras(cams, bg=bg)
    st.capacity = 0
    st.ensure_capacity()
    return st


def psnr(eval_state, masked: bool = True) -> float:
    """PSNR (dB) of eval_state's render against its targets over its view
    batch (a measurement; not part of the fit step). masked: the paper's
    masked PSNR (Section 5), only pixels whose alpha is non-zero in the target
    or the render; otherwise every pixel."""
    import torch
    eval_state.forward()
    if not masked:
        mse = torch.mean((eval_state.rgb - eval_state.target_rgb) ** 2).item()
        return float(10.0 * np.log10(1.0 / max(mse, 1e-20)))
    se, count = 0.0, 0
    off = 0
    for v in range(eval_state.V):
        c = eval_state.table.host[v]
        P = int(c.width) * int(c.height)
        m = (eval_state.alpha[off:off + P] > 0) | (eval_state.target_alpha[off:off + P] > 0)
        d = (eval_state.rgb[3 * off:3 * (off + P)] - eval_state.target_rgb[3 * off:3 * (off + P)]).view(3, P)
        se += float((d[:, m] ** 2).sum().item())
        count += 3 * int(m.sum().item())
        off += P
    return float(10.0 * np.log10(count / max(se, 1e-20))) if count else float("inf")


class ContinuousRefinement:
    """Streams foveal views into a FitState's batch.

    state: the FitState being fitted (its batch: n_fixed periphery frames,
    then crops); target_state: a FitState of the target Gaussians used to
    render the targets of new views (over a zero background, premultiplied);
    crop_stream: an iterator of single-view camera dicts; backgrounds:
    (steps, V, 3) random per-view backgrounds, one row per iteration."""

    def __init__(self, state, target_state, cams: dict, crop_stream, backgrounds: np.ndarray, *, n_fixed: int = 2,
                 replace_every: int = 10, n_replace: int = 4, view_set: ViewSet | None = None):
        import torch
        self.st, self.tgt = state, target_state
        self.cams = {k: np.array(v) for k, v in cams.items()}
        self.V = len(self.cams["width"])
        self.crops = crop_stream
        self.bg = torch.as_tensor(np.asarray(backgrounds, np.float32)).to(state.device)
        self.n_fixed, self.replace_every, self.n_replace = int(n_fixed), int(replace_every), int(n_replace)
        self.views = view_set if view_set is not None else ViewSet()
        for v in range(self.V):  # the starting batch is the starting training set
            self.views.add(self.cams["campos"][v], camera_forward(self.cams, v))
        self.next_slot = self.n_fixed
        self.it = 0
        self.offered = 0
        self.accepted = 0
        self.replacements = 0

    def _render_targets(self) -> None:
        self.tgt.set_cameras(self.cams, bg=np.zeros((self.V, 3), np.float32))
        self.tgt.ensure_capacity()
        self.tgt.forward()
        self.st.target_rgb.copy_(self.tgt.rgb)
        self.st.target_alpha.copy_(self.tgt.alpha)

    def replace_crops(self, max_offers: int = 64) -> int:
        """Replaces up to n_replace of the oldest crops by streamed views that
        pass Eq. 1; returns how many were replaced."""
        new = []
        while len(new) < self.n_replace and self.offered < 10**9 and max_offers > 0:
            c = next(self.crops)
            self.offered += 1
            max_offers -= 1
            if self.views.offer(c["campos"][0], camera_forward(c, 0)):
                self.accepted += 1
                new.append(c)
        for c in new:
            slot = self.next_slot
            for k in self.cams:
                self.cams[k][slot] = c[k][0]
            self.next_slot = self.n_fixed + (slot - self.n_fixed + 1) % (self.V - self.n_fixed)
        if new:
            self.st.set_cameras(self.cams, bg=np.zeros((self.V, 3), np.float32))
            self.st.ensure_capacity()
            self._render_targets()
            self.replacements += 1
        return len(new)

    def step(self) -> None:
        """One fit iteration (no host synchronisation unless views change)."""
        if self.it > 0 and self.it % self.replace_every == 0:
            self.replace_crops()
        self.st.bg.copy_(self.bg[self.it % self.bg.shape[0]])
        if self.st.graph is None:
            self.st.capture(warmup=0)
        self.st.replay()
        self.it += 1

    def restart(self) -> None:
        """Periodic restart: keep the Gaussians, discard the optimiser state."""
        self.st.reset_optimizer()


def regenerate(gaussians: dict, cams: dict, target_rgb, target_alpha, backgrounds: np.ndarray, *, iters: int = 700,
               simplify_at: int = 95, keep: int = 10_000, lr: dict | None = None, **state_kw) -> tuple:
    """The abbreviated initial regeneration of Section 4.2: fit the seeded
    Gaussians to the view batch with the raised learning rates, no
    densification, simplify to the `keep` most important Gaussians after
    `simplify_at` steps, and continue (fresh optimiser state) to `iters`
    steps. backgrounds: (steps, V, 3) random per-view backgrounds. Returns
    (final FitState, {"wall_s", "simplify_s", "n_before", "n_after"});
    wall time from the first step to the last one's completion, including the
    simplification and the rebuilt state's first capture."""
    import time
    import torch
    from .fit import FitState, boosted_lr
    lr = lr if lr is not None else boosted_lr()
    bgt = torch.as_tensor(np.asarray(backgrounds, np.float32)).cuda()
    V = len(cams["width"])
    regrown = 0

    def run(st, first, last):
        # splats grow at the raised rates: the pair capacity starts at 4x the
        # initial count and is checked every `check_every` steps; a step that
        # overflowed it (its sort emits nothing, so it renders the background)
        # is followed by a regrow to the counted need and a new capture
        nonlocal regrown
        for it in range(first, last):
            st.bg.copy_(bgt[it % bgt.shape[0]])
            st.replay()
            if (it + 1 - first) % check_every == 0 or it + 1 == last:
                s = st.check_status()
                if s == G.GSFIT_ERR_CAPACITY:
                    st.ensure_capacity(int(int(st.n_instances.item()) * 1.5) + 1024)
                    st.capture(warmup=0)
                    regrown += 1
                elif s != 0:
                    raise RuntimeError(f"device status {s} during the regeneration")

    check_every = 50
    st = FitState(gaussians, cams, bg=np.zeros((V, 3), np.float32), lr=lr, **state_kw)
    st.ensure_capacity(4 * st.count_instances())
    st.target_rgb.copy_(torch.as_tensor(target_rgb).reshape(-1))
    st.target_alpha.copy_(torch.as_tensor(target_alpha).reshape(-1))
    n_before = st.n
    st.capture(warmup=0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run(st, 0, min(simplify_at, iters))
    t1 = time.perf_counter()
    if iters > simplify_at:
        kept = st.simplified_params(keep)
        st2 = FitState.from_params(kept, st.sh_degree, cams, bg=np.zeros((V, 3), np.float32), lr=lr, **state_kw)
        st2.ensure_capacity(4 * st2.count_instances())
        st2.target_rgb.copy_(st.target_rgb)
        st2.target_alpha.copy_(st.target_alpha)
        del st
        st = st2
        st.capture(warmup=0)
        t2 = time.perf_counter()
        run(st, simplify_at, iters)
    else:
        t2 = t1
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    return st, {"wall_s": t3 - t0, "simplify_s": t2 - t1, "n_before": n_before, "n_after": st.n,
                "capacity_regrows": regrown}
