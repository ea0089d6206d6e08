"""Autotuner of the batched launch: the tile edge and the batch depths of the
compositing kernels (the number of Gaussians staged per shared-memory slot,
chosen for the forward and the adjoint kernel separately).

The batch depths only change the compositing kernels, so the library measures
them itself (gsfit_render_autotune, through FitState.tune_batch). The tile edge
changes the projection's rectangles, the pair count and the sort as well, so
it is compared on whole iterations: for each tile edge a state is built,
its batch depth tuned, one iteration captured as a CUDA graph and replayed.
The winner is cached per device and workload signature in a JSON file next to
this module (not part of the sources), so later runs skip the search.
"""
from __future__ import annotations

import hashlib
import json
from pathlib import Path

import numpy as np

CACHE = Path(__file__).resolve().parent / "_tuning.json"
TILES = (8, 16)


def signature(n: int, sh_degree: int, cams: dict, features: str = "f32") -> str:
    """Device name + workload shape (Gaussian count, SH degree, view sizes, feature storage)."""
    import torch
    sizes = np.stack([np.asarray(cams["width"], np.int64), np.asarray(cams["height"], np.int64)], 1)
    h = hashlib.sha1(sizes.tobytes()).hexdigest()[:12]
    return f"{torch.cuda.get_device_name()}|n={n}|sh={sh_degree}|views={len(sizes)}:{h}|{features}"


def _load_cache() -> dict:
    try:
        return json.loads(CACHE.read_text())
    except (OSError, ValueError):
        return {}


def _store(key: str, entry: dict) -> None:
    data = _load_cache()
    data[key] = entry
    try:
        CACHE.write_text(json.dumps(data, indent=1, sort_keys=True))
    except OSError:
        pass  # a read-only install just re-tunes next time


def time_iterations(st, steps: int = 20, warmup: int = 3) -> float:
    """Mean ms per captured iteration of a FitState (graph replay)."""
    import torch
    st.capture()
    for _ in range(warmup):
        st.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        st.replay()
    e1.record()
    torch.cuda.synchronize()
    if st.check_status() != 0:
        raise RuntimeError("device status set while tuning")
    return e0.elapsed_time(e1) / steps


def autotune(make_state, key: str, tiles=TILES, steps: int = 20, use_cache: bool = True) -> dict:
    """Picks (tile, batch, batch_bwd) for a workload. make_state(tile, batch,
    batch_bwd) returns a FitState of the workload (targets set) laid out for
    that tile edge. Returns {"tile", "batch", "batch_bwd", "ms_per_step",
    "candidates": {tile: {...}}, "cached"}."""
    import torch
    if use_cache:
        hit = _load_cache().get(key)
        if hit and "batch_bwd" in hit:
            return dict(hit, cached=True)
    cands = {}
    for tile in tiles:
        st = make_state(tile, 128, 64)
        depth_ms = st.tune_batch()
        ms = time_iterations(st, steps)
        cands[int(tile)] = {"batch": int(st.opts.batch), "batch_bwd": int(st.opts.batch_bwd), "ms_per_step": ms,
                            "depth_ms": {int(d): [float(f), float(b)] for d, (f, b) in depth_ms.items()}}
        del st
        torch.cuda.empty_cache()
    tile = min(cands, key=lambda t: cands[t]["ms_per_step"])
    entry = {"tile": int(tile), "batch": cands[tile]["batch"], "batch_bwd": cands[tile]["batch_bwd"],
             "ms_per_step": cands[tile]["ms_per_step"],
             "candidates": {str(t): c for t, c in cands.items()}}
    _store(key, entry)
    return dict(entry, cached=False)
