"""Fit-step runner: device buffers for one Gaussian set and one view batch,
the iteration project -> bin/sort -> render -> loss -> adjoint -> Adam as
calls into libgsfit, CUDA-graph capture of the whole iteration, and a
torch.autograd.Function around render.

PyTorch provides device memory, streams and graphs only; every arithmetic
step runs in the library's kernels.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import gsfit as G

# 3DGS learning rates; the paper raises scale, opacity and colour by ~50% for
# its abbreviated regeneration run (Section 4.2).
DEFAULT_LR = dict(lr_means=1.6e-4, lr_quats=1e-3, lr_scales=5e-3, lr_opacity=5e-2, lr_sh_dc=2.5e-3)


def boosted_lr(scale: float = 1.5) -> dict:
    lr = dict(DEFAULT_LR)
    for k in ("lr_scales", "lr_opacity", "lr_sh_dc"):
        lr[k] *= scale
    return lr


class StageMarks:
    """Timing events that a captured CUDA graph records as event-record
    nodes, so that every replay timestamps the boundaries between its stages
    (cudaEventRecordExternal; through PyTorch where its events support it,
    else through the CUDA runtime PyTorch and the library share)."""

    def __init__(self, count: int):
        try:
            self._ev = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(count)]
            self._rt = None
        except TypeError:
            import ctypes
            self._rt = ctypes.CDLL("libcudart.so.13")
            self._rt.cudaEventRecordWithFlags.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint]
            self._rt.cudaEventElapsedTime.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.c_void_p,
                                                      ctypes.c_void_p]
            self._ev = []
            for _ in range(count):
                e = ctypes.c_void_p()
                if self._rt.cudaEventCreate(ctypes.byref(e)) != 0:
                    raise RuntimeError("cudaEventCreate failed")
                self._ev.append(e)

    def record(self, k: int, stream=None) -> None:
        s = torch.cuda.current_stream() if stream is None else stream
        if self._rt is None:
            self._ev[k].record(s)
        elif self._rt.cudaEventRecordWithFlags(self._ev[k], s.cuda_stream, 1) != 0:  # 1: cudaEventRecordExternal
            raise RuntimeError("cudaEventRecordWithFlags failed")

    def elapsed(self, a: int, b: int) -> float:
        if self._rt is None:
            return self._ev[a].elapsed_time(self._ev[b])
        import ctypes
        ms = ctypes.c_float()
        if self._rt.cudaEventElapsedTime(ctypes.byref(ms), self._ev[a], self._ev[b]) != 0:
            raise RuntimeError("cudaEventElapsedTime failed")
        return float(ms.value)


class FitState:
    """All device buffers of the fit step for one scene and one view batch."""

    def __init__(self, gaussians: dict, cams: dict, *, target_rgb=None, target_alpha=None, bg=None,
                 capacity: int | None = None, lr: dict | None = None, eps: float = 1e-15,
                 lam: float = 0.2, features: str = "f32", tile: int = 16, batch: int = 128,
                 batch_bwd: int = 64, exp_half2: bool = False, keep_keys: bool = False, fuse_adam: bool = False,
                 keep_grads: bool = False, device: str = "cuda"):
        """features: "f32", or "f16" / "bf16" for the mixed-precision form
        (16-bit copy of the SH coefficients read by the projection, kept
        current by Adam; float32 master parameters and moments).
        tile (8 or 16), batch and batch_bwd (64, 128, 256 records per
        shared-memory slot of the forward and the adjoint compositing): the
        compositing options; see tune.py for choosing them.
        exp_half2: evaluate the compositing exponent in packed half precision
        (the half2 option of the mixed-precision form).
        keep_keys: also write the sorted (tile, depth) keys to self.keys; the
        fit needs only the lists and ranges, which the sort then produces
        with 32-bit tile keys.
        fuse_adam: step() runs the projection adjoint and Adam as one pass
        (gsfit_project_bwd_adam), which passes each Gaussian's gradient
        straight into its update and needs no gradient buffer; on GB300 the
        two separate kernels are faster (the fused pass runs at the register
        budget of the projection adjoint, too few warps for Adam's stream),
        so it is off by default. keep_grads: that pass also writes the
        gradient to self.grads (render_bwd() and project_bwd() always do)."""
        self.device = device
        self.keep_keys = bool(keep_keys)
        self.fuse_adam = bool(fuse_adam)
        self.keep_grads = bool(keep_grads)
        self.TIMED_STAGES = self.TIMED_STAGES_FUSED if self.fuse_adam else self.TIMED_STAGES_SEPARATE
        self.tile = int(tile)
        self.exp_half2 = bool(exp_half2)
        self.opts = G.RenderOpts(self.tile, int(batch), int(self.exp_half2), int(batch_bwd))
        self.n = int(gaussians["means"].shape[0])
        self.sh_degree = int(round(gaussians["sh"].shape[1] ** 0.5)) - 1
        self.n_planes = G.num_planes(self.sh_degree)
        self.params = torch.from_numpy(G.pack_params(gaussians)).to(device).contiguous()
        self.feature_name = features
        self.feature_dtype = G.FEATURES[features]
        self.features = None
        if self.feature_dtype != 0:
            tdt = torch.float16 if features == "f16" else torch.bfloat16
            self.features = torch.empty((self.n_planes - 3, self.n, 4), dtype=tdt, device=device)
            self.refresh_features()
        self.grads = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step_count = torch.zeros(1, dtype=torch.int32, device=device)
        self.lam = float(lam)
        self.eps = float(eps)
        self.lr = G.lr_table(self.sh_degree, **(lr or DEFAULT_LR))
        self.loss_out = torch.zeros(1, dtype=torch.float32, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self.n_instances = torch.zeros(1, dtype=torch.int32, device=device)
        self.set_cameras(cams, bg=bg)
        if target_rgb is not None:
            self.set_targets(target_rgb, target_alpha)
        self.capacity = 0
        self.ensure_capacity(capacity)
        self.graph = None
        self.marks = None

    @classmethod
    def from_params(cls, params, sh_degree: int, cams: dict, **kw):
        """A state around device parameters (n_planes, n, 4) float32 (e.g. a
        simplified set): fresh gradients and optimiser state."""
        import torch
        first = G.unpack_params(params[:, :1].cpu().numpy(), sh_degree)
        st = cls(first, cams, capacity=16, **{k: v for k, v in kw.items() if k != "capacity"})
        st.n = int(params.shape[1])
        st.params = params.contiguous()
        st.grads = torch.zeros_like(st.params)
        st.m = torch.zeros_like(st.params)
        st.v = torch.zeros_like(st.params)
        if st.feature_dtype != 0:
            st.features = torch.empty((st.n_planes - 3, st.n, 4), dtype=st.features.dtype, device=st.device)
            st.refresh_features()
        st.set_cameras(cams, bg=kw.get("bg"))
        st.capacity = 0
        st.ensure_capacity(kw.get("capacity"))
        return st

    def save(self, path) -> None:
        """Checkpoint: parameters, Adam moments and step count as raw arrays
        (numpy .npz; syncs)."""
        np.savez(path, params=self.params.cpu().numpy(), m=self.m.cpu().numpy(), v=self.v.cpu().numpy(),
                 step=self.step_count.cpu().numpy(), sh_degree=np.int32(self.sh_degree))

    @classmethod
    def resume(cls, path, cams: dict, *, reset_optimizer: bool = False, **kw):
        """A state from a checkpoint on the given views. reset_optimizer:
        reload the Gaussians but discard the optimiser state, as the paper's
        periodic restarts do (Section 4.2)."""
        import torch
        d = np.load(path)
        st = cls.from_params(torch.from_numpy(d["params"]).to(kw.get("device", "cuda")), int(d["sh_degree"]), cams,
                             **kw)
        if not reset_optimizer:
            st.m.copy_(torch.from_numpy(d["m"]))
            st.v.copy_(torch.from_numpy(d["v"]))
            st.step_count.copy_(torch.from_numpy(d["step"]))
        return st

    def importance(self):
        """Per-Gaussian blend-weight importance over the current view batch
        (one forward pass with gsfit_render_importance; no synchronisation)."""
        import torch
        imp = torch.zeros(self.n, dtype=torch.float32, device=self.device)
        self.project()
        self.bin_sort()
        G.gsfit_render_importance(self.proj, self.cams_dev, self.V, self.n, self.T, self.vals, self.ranges, self.bg,
                                  self.rgb, self.alpha, self.T_final, self.n_contrib, imp, None, self.tile_order,
                                  self.status, self.opts)
        return imp

    def simplified_params(self, keep: int):
        """The `keep` most important Gaussians' parameters (gsfit_simplify over
        this batch's importance); synchronises to read the count."""
        import torch
        imp = self.importance()
        out = torch.empty_like(self.params)
        n_out = torch.zeros(1, dtype=torch.int32, device=self.device)
        ws = torch.empty(G.gsfit_simplify_workspace_size(self.n), dtype=torch.uint8, device=self.device)
        G.gsfit_simplify(self.params, self.n, self.n_planes, imp, int(keep), out, n_out, ws)
        m = int(n_out.item())
        return out[:, :m].contiguous()

    # -- view batch -----------------------------------------------------
    def set_cameras(self, cams: dict, bg=None) -> None:
        self.table = G.camera_table(cams, self.tile)
        self.V = self.table.n_views
        self.T = self.table.total_tiles
        self.P = self.table.total_pixels
        self.cams_dev = G.cameras_to_device(self.table, self.device)
        dev, f32 = self.device, torch.float32
        self.proj = G.ProjBuffers.allocate(self.V * self.n, dev)
        self.rgb = torch.zeros(3 * self.P, dtype=f32, device=dev)
        self.alpha = torch.zeros(self.P, dtype=f32, device=dev)
        self.T_final = torch.zeros(self.P, dtype=f32, device=dev)
        self.n_contrib = torch.zeros(self.P, dtype=torch.int32, device=dev)
        self.dL_drgb = torch.zeros(3 * self.P, dtype=f32, device=dev)
        self.dL_dalpha = torch.zeros(self.P, dtype=f32, device=dev)
        self.target_rgb = torch.zeros(3 * self.P, dtype=f32, device=dev)
        self.target_alpha = torch.zeros(self.P, dtype=f32, device=dev)
        self.ranges = torch.zeros(2 * self.T, dtype=torch.int32, device=dev)
        # the heavy-first tile permutation, the number of non-empty tiles, each
        # tile's furthest contributor and the adjoint's launch order
        self.tile_order = torch.zeros(G.tile_order_words(self.T), dtype=torch.int32, device=dev)
        self.grad2d = torch.zeros(self.V * self.n * 16, dtype=f32, device=dev)
        self.loss_ws = torch.zeros(G.gsfit_loss_workspace_size(self.table) // 4 + 1, dtype=f32, device=dev)
        bgv = np.zeros((self.V, 3), np.float32) if bg is None else np.asarray(bg, np.float32).reshape(self.V, 3)
        self.bg = torch.from_numpy(bgv.copy()).to(dev)
        self.graph = None

    def set_targets(self, target_rgb, target_alpha) -> None:
        self.target_rgb.copy_(torch.as_tensor(np.asarray(target_rgb, np.float32)).reshape(-1))
        self.target_alpha.copy_(torch.as_tensor(np.asarray(target_alpha, np.float32)).reshape(-1))

    def set_bg(self, bg) -> None:
        self.bg.copy_(torch.as_tensor(np.asarray(bg, np.float32)).reshape(self.V, 3))

    def refresh_features(self, stream=None) -> None:
        """Rewrites the 16-bit feature copy from the float32 parameters."""
        if self.feature_dtype != 0:
            G.gsfit_features_refresh(self.params, self.n, self.n_planes, self.features, self.feature_dtype, stream)

    # -- capacity -------------------------------------------------------
    def count_instances(self) -> int:
        """Pairs the current parameters produce (projects once; syncs)."""
        self.project()
        return int(self.proj.tiles.to(torch.int64).sum().item())

    def ensure_capacity(self, capacity: int | None = None, slack: float = 1.5) -> None:
        need = capacity if capacity is not None else max(1024, int(math.ceil(self.count_instances() * slack)))
        if need <= self.capacity:
            return
        self.capacity = int(need)
        dev = self.device
        self.keys = torch.empty(self.capacity, dtype=torch.int64, device=dev) if self.keep_keys else None
        self.vals = torch.empty(self.capacity, dtype=torch.int32, device=dev)
        ws_bytes = G.gsfit_bin_sort_workspace_size(self.V * self.n, self.capacity, self.T)
        self.sort_ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        self.graph = None

    def check_status(self) -> int:
        """Reads (and clears) the device status word; syncs."""
        s = int(self.status.item())
        if s != 0:
            self.status.zero_()
        return s

    # -- stages ---------------------------------------------------------
    def project(self, stream=None):
        G.gsfit_project(self.params, self.n, self.sh_degree, self.cams_dev, self.V, self.proj, stream,
                        self.features, self.feature_dtype)

    def bin_sort(self, stream=None):
        G.gsfit_bin_sort(self.proj, self.cams_dev, self.V, self.n, self.T, self.sort_ws, self.keys, self.vals,
                         self.capacity, self.n_instances, self.ranges, self.status, stream, self.tile_order)

    def render_fwd(self, stream=None):
        G.gsfit_render_fwd(self.proj, self.cams_dev, self.V, self.n, self.T, self.vals, self.ranges, self.bg,
                           self.rgb, self.alpha, self.T_final, self.n_contrib, stream, self.tile_order, self.status,
                           self.opts)

    def loss(self, stream=None):
        G.gsfit_loss(self.cams_dev, self.V, self.rgb, self.alpha, self.target_rgb, self.target_alpha, self.bg,
                     self.lam, self.dL_drgb, self.dL_dalpha, self.loss_out, self.loss_ws, stream)

    def render_bwd(self, stream=None):
        G.gsfit_render_bwd(self.params, self.n, self.sh_degree, self.proj, self.cams_dev, self.V, self.T,
                           self.vals, self.ranges, self.bg, self.T_final, self.n_contrib, self.dL_drgb,
                           self.dL_dalpha, self.grad2d, self.grads, stream, self.tile_order, self.status,
                           self.features, self.feature_dtype, self.opts)

    def blend_bwd(self, stream=None):
        G.gsfit_blend_bwd(self.proj, self.cams_dev, self.V, self.n, self.T, self.vals, self.ranges, self.bg,
                          self.T_final, self.n_contrib, self.dL_drgb, self.dL_dalpha, self.grad2d, stream,
                          self.tile_order, self.status, self.opts)

    def project_bwd(self, stream=None):
        G.gsfit_project_bwd(self.params, self.n, self.sh_degree, self.proj, self.cams_dev, self.V, self.grad2d,
                            self.grads, stream, self.features, self.feature_dtype)

    def project_bwd_adam(self, stream=None):
        G.gsfit_project_bwd_adam(self.params, self.n, self.sh_degree, self.proj, self.cams_dev, self.V, self.grad2d,
                                 self.grads if self.keep_grads else None, self.m, self.v, self.lr, 0.9, 0.999,
                                 self.eps, self.step_count, stream, self.features, self.feature_dtype, self.status)

    def blended_pairs(self) -> int:
        """Blended (pixel, Gaussian) pairs of the last forward pass (syncs)."""
        cnt = torch.zeros(1, dtype=torch.int64, device=self.device)
        G.gsfit_render_count(self.proj, self.cams_dev, self.V, self.n, self.T, self.vals, self.ranges,
                             self.n_contrib, cnt, None, self.tile_order, self.opts)
        return int(cnt.item())

    def tune_batch(self, reps: int = 3) -> dict:
        """Measures the compositing batch depths on this state's current view
        batch (one forward and loss first, for realistic lists and
        cotangents), keeps the fastest forward and the fastest adjoint depth
        in self.opts and drops any captured graph. Returns {depth: (forward
        ms, adjoint ms)}; synchronises."""
        self.forward()
        self.loss()
        best, times = G.gsfit_render_autotune(self.proj, self.cams_dev, self.V, self.n, self.T, self.vals,
                                              self.ranges, self.tile_order, self.bg, self.rgb, self.alpha,
                                              self.T_final, self.n_contrib, self.dL_drgb, self.dL_dalpha,
                                              self.grad2d, self.tile, reps, None, self.status)
        self.opts = best
        self.opts.exp_half2 = int(self.exp_half2)
        self.graph = None
        return times

    def adam(self, stream=None):
        G.gsfit_adam_step(self.params, self.grads, self.m, self.v, self.n, self.n_planes, self.lr, 0.9, 0.999,
                          self.eps, self.step_count, stream, self.features, self.feature_dtype)

    def forward(self, stream=None):
        self.project(stream)
        self.bin_sort(stream)
        self.render_fwd(stream)

    def step(self, stream=None, marks: "StageMarks | None" = None):
        """One fit iteration (no host synchronisation). marks: timing events
        recorded before the first stage and after each of TIMED_STAGES (the
        adjoint as its two halves, the same kernels as render_bwd; with
        fuse_adam the second half and Adam as one stage)."""
        if marks is None:
            self.forward(stream)
            self.loss(stream)
            if self.fuse_adam:
                self.blend_bwd(stream)
                self.project_bwd_adam(stream)
            else:
                self.render_bwd(stream)
                self.adam(stream)
            return
        marks.record(0, stream)
        for k, name in enumerate(self.TIMED_STAGES):
            with torch.cuda.nvtx.range(name):
                getattr(self, name)(stream)
            marks.record(k + 1, stream)

    STAGES = ("project", "bin_sort", "render_fwd", "loss", "render_bwd", "adam")
    TIMED_STAGES_SEPARATE = ("project", "bin_sort", "render_fwd", "loss", "blend_bwd", "project_bwd", "adam")
    TIMED_STAGES_FUSED = ("project", "bin_sort", "render_fwd", "loss", "blend_bwd", "project_bwd_adam")
    TIMED_STAGES = TIMED_STAGES_SEPARATE  # the default state's; each state sets its own from fuse_adam

    # -- graphs ---------------------------------------------------------
    def capture(self, warmup: int = 1, stage_marks: bool = False):
        """Captures one iteration in a CUDA graph (replay with .replay()).
        stage_marks: the graph also records timing events between the
        stages (event-record nodes), read with stage_times() after a replay."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                self.step(s)
        torch.cuda.current_stream().wait_stream(s)
        self.marks = StageMarks(len(self.TIMED_STAGES) + 1) if stage_marks else None
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.step(marks=self.marks)
        self.graph = g
        return g

    def stage_times(self) -> dict:
        """Per-stage milliseconds of the last replay of a graph captured with
        stage_marks (synchronises)."""
        if self.marks is None:
            raise RuntimeError("capture(stage_marks=True) first")
        torch.cuda.synchronize()
        return {name: self.marks.elapsed(k, k + 1) for k, name in enumerate(self.TIMED_STAGES)}

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def reset_optimizer(self):
        """Discards the optimiser state (restart of the refinement, Section 4.2)."""
        self.m.zero_()
        self.v.zero_()
        self.step_count.zero_()

    # -- host views -----------------------------------------------------
    def gaussians(self) -> dict:
        return G.unpack_params(self.params.cpu().numpy(), self.sh_degree)

    def gaussians_first(self) -> dict:
        """The first Gaussian only (a placeholder for states that share these parameters)."""
        return G.unpack_params(self.params[:, :1].cpu().numpy(), self.sh_degree)

    def gradients(self) -> dict:
        return G.unpack_params(self.grads.cpu().numpy(), self.sh_degree)


class GsfitRender(torch.autograd.Function):
    """Differentiable render of a FitState's view batch.

    forward: project + bin/sort + composite; keeps the projected records, the
    sorted lists, T_final and n_contrib (no per-(pixel, Gaussian) state).
    backward: the hand-written adjoint (recomputes per-pixel transmittance
    from T_final and n_contrib) chained through the projection.
    """

    @staticmethod
    def forward(ctx, params, state: FitState):
        if params.data_ptr() != state.params.data_ptr():
            state.params.copy_(params.detach())
            state.refresh_features()
        state.forward()
        ctx.state = state
        ctx.save_for_backward(state.T_final, state.n_contrib)
        return state.rgb.clone(), state.alpha.clone()

    @staticmethod
    def backward(ctx, g_rgb, g_alpha):
        st = ctx.state
        st.dL_drgb.copy_(g_rgb if g_rgb is not None else torch.zeros_like(st.dL_drgb))
        st.dL_dalpha.copy_(g_alpha if g_alpha is not None else torch.zeros_like(st.dL_dalpha))
        st.render_bwd()
        return st.grads.clone(), None


def render(params, state: FitState):
    return GsfitRender.apply(params, state)


class HostFeed:
    """Feeds a FitState new per-step inputs (target images and backgrounds)
    from pinned host memory, as a frame source (the path tracer's views) does
    on every step, without stalling the GPU.

    prefetch(k) starts copying step k's inputs into one of two staging
    buffers on a copy stream; step() replays an iteration captured against
    that staging buffer (one CUDA graph per buffer, so the inputs are read
    where the copy put them, with no device-to-device copy) and starts the
    device-to-host copy of its loss; loss(handle) waits for that copy only.
    So the transfer of step k + 1 overlaps step k, and reading step k's loss
    while step k + 1 runs keeps the GPU busy. Staging buffer k % 2 is reused
    by prefetch(k + 2) only after step k has finished with it. The state's
    own target and background buffers are not used by these steps."""

    def __init__(self, state: FitState):
        self.st = state
        self.copy_stream = torch.cuda.Stream()
        self.stage = [(torch.empty_like(state.target_rgb), torch.empty_like(state.target_alpha),
                       torch.empty_like(state.bg)) for _ in range(2)]
        self.staged = [torch.cuda.Event() for _ in range(2)]
        self.consumed = [torch.cuda.Event() for _ in range(2)]
        self.loss_host = [torch.empty(1, dtype=torch.float32).pin_memory() for _ in range(2)]
        self.loss_done = [torch.cuda.Event() for _ in range(2)]
        self.issued = 0  # prefetches issued
        self.stepped = 0  # steps issued
        self.h2d_bytes = state.target_rgb.numel() * 4 + state.target_alpha.numel() * 4 + state.bg.numel() * 4
        self.graphs = [self._capture(b) for b in range(2)]

    def _capture(self, b: int):
        """One iteration captured with staging buffer b as its inputs."""
        st = self.st
        saved = (st.target_rgb, st.target_alpha, st.bg)
        st.target_rgb, st.target_alpha, st.bg = self.stage[b]
        try:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                st.step()
        finally:
            st.target_rgb, st.target_alpha, st.bg = saved
        return g

    def prefetch(self, host_rgb, host_alpha, host_bg) -> None:
        """Copies the next step's inputs (pinned host tensors) to the device."""
        b = self.issued % 2
        rgb, alpha, bg = self.stage[b]
        with torch.cuda.stream(self.copy_stream):
            if self.issued >= 2:
                self.copy_stream.wait_event(self.consumed[b])
            rgb.copy_(host_rgb, non_blocking=True)
            alpha.copy_(host_alpha, non_blocking=True)
            bg.copy_(host_bg, non_blocking=True)
            self.staged[b].record(self.copy_stream)
        self.issued += 1

    def step(self) -> int:
        """One fit iteration on the oldest staged inputs; returns a handle for loss()."""
        if self.stepped >= self.issued:
            raise RuntimeError("HostFeed.step without a prefetched input")
        b = self.stepped % 2
        st = self.st
        cur = torch.cuda.current_stream()
        cur.wait_event(self.staged[b])
        self.graphs[b].replay()
        self.consumed[b].record(cur)
        self.loss_host[b].copy_(st.loss_out, non_blocking=True)
        self.loss_done[b].record(cur)
        self.stepped += 1
        return b

    def loss(self, handle: int) -> float:
        """The loss of the step with this handle (waits for that step only);
        read it before issuing two more steps."""
        self.loss_done[handle].synchronize()
        return float(self.loss_host[handle].item())
