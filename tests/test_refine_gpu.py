"""Continuous refinement (Section 4.2): streamed foveal views enter the batch
through Eq. 1, their targets are rendered from the target set, the fit keeps
improving, and a restart keeps the Gaussians but discards the optimiser
state. Small scene (20k Gaussians, 256^2 periphery frames, 64..128 px crops)."""
import itertools

import numpy as np
import pytest

import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KW = dict(periphery_size=256, crop_min=64, crop_max=128)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2601_22026_gb300 as pkg
    pkg.build()


def _setup(features="f32"):
    from paper_2601_22026_gb300 import refine
    from paper_2601_22026_gb300.fit import FitState, boosted_lr
    cams = scenes.periphery_batch_cameras(0, n_crops=6, **KW)
    V = len(cams["width"])
    zeros = np.zeros((V, 3), np.float32)
    gs = scenes.random_gaussians(20000, 3, 61, log_scale_mean=-4.0)
    tg = scenes.random_gaussians(20000, 3, 62, log_scale_mean=-4.0)
    tgt = FitState(tg, cams, bg=zeros)
    tgt.forward()
    st = FitState(gs, cams, bg=zeros, lr=boosted_lr(), features=features)
    st.target_rgb.copy_(tgt.rgb)
    st.target_alpha.copy_(tgt.alpha)
    ev = refine.view_state(st, cams, bg=zeros)
    ev.target_rgb.copy_(tgt.rgb)
    ev.target_alpha.copy_(tgt.alpha)
    stream = (scenes.foveal_crops(0, 1, 5000 + k, **KW) for k in itertools.count())
    loop = refine.ContinuousRefinement(st, tgt, cams, stream, scenes.backgrounds(V, 63, n_steps=64),
                                       replace_every=10, n_replace=2)
    return st, tgt, ev, loop


@pytest.mark.parametrize("features", ["f32", "f16"])
def test_refinement_streams_views_and_improves(features):
    from paper_2601_22026_gb300 import refine
    st, tgt, ev, loop = _setup(features)
    p0 = refine.psnr(ev)
    n0 = len(loop.views)
    for _ in range(40):
        loop.step()
    torch.cuda.synchronize()
    assert st.check_status() == 0
    assert loop.replacements == 3  # at iterations 10, 20, 30
    assert 0 < loop.accepted <= loop.offered
    assert len(loop.views) == n0 + loop.accepted
    # the replaced views' targets are the target set's render of the current batch
    tgt.forward()
    assert torch.equal(st.target_rgb, tgt.rgb)
    p1 = refine.psnr(ev)
    assert p1 > p0 + 0.5, (p0, p1)


def test_restart_keeps_gaussians_and_discards_optimizer_state():
    st, _, _, loop = _setup()
    for _ in range(5):
        loop.step()
    torch.cuda.synchronize()
    params = st.params.clone()
    loop.restart()
    torch.cuda.synchronize()
    assert torch.equal(st.params, params)
    assert float(st.m.abs().max()) == 0.0 and float(st.v.abs().max()) == 0.0
    assert int(st.step_count.item()) == 0


def test_regeneration_schedule_simplifies_and_keeps_fitting():
    from paper_2601_22026_gb300 import refine
    from paper_2601_22026_gb300.fit import FitState
    cams = scenes.periphery_batch_cameras(1, n_crops=4, **KW)
    V = len(cams["width"])
    zeros = np.zeros((V, 3), np.float32)
    gs = scenes.random_gaussians(12000, 3, 71, log_scale_mean=-4.0)
    tgt = FitState(scenes.random_gaussians(12000, 3, 72, log_scale_mean=-4.0), cams, bg=zeros)
    tgt.forward()
    before = FitState(gs, cams, bg=zeros)
    before.target_rgb.copy_(tgt.rgb)
    p0 = refine.psnr(before)
    del before
    st, info = refine.regenerate(gs, cams, tgt.rgb, tgt.alpha, scenes.backgrounds(V, 73, n_steps=64), iters=60,
                                 simplify_at=20, keep=3000)
    assert info["n_before"] == 12000 and 3000 <= info["n_after"] <= 3100
    assert st.n == info["n_after"] and info["wall_s"] > 0
    st.bg.zero_()
    assert refine.psnr(st) > p0 + 0.5


@pytest.mark.parametrize("reset", [False, True])
def test_checkpoint_resume(tmp_path, reset):
    from paper_2601_22026_gb300.fit import FitState, boosted_lr
    cams = scenes.periphery_batch_cameras(2, n_crops=3, **KW)
    V = len(cams["width"])
    zeros = np.zeros((V, 3), np.float32)
    tgt = FitState(scenes.random_gaussians(5000, 3, 82, log_scale_mean=-4.0), cams, bg=zeros)
    tgt.forward()
    a = FitState(scenes.random_gaussians(5000, 3, 81, log_scale_mean=-4.0), cams, bg=zeros, lr=boosted_lr())
    a.target_rgb.copy_(tgt.rgb)
    a.target_alpha.copy_(tgt.alpha)
    for _ in range(3):
        a.step()
    path = tmp_path / "ckpt.npz"
    a.save(path)
    b = FitState.resume(path, cams, reset_optimizer=reset, bg=zeros, lr=boosted_lr())
    b.target_rgb.copy_(tgt.rgb)
    b.target_alpha.copy_(tgt.alpha)
    torch.cuda.synchronize()
    assert torch.equal(a.params, b.params)
    if reset:
        assert float(b.m.abs().max()) == 0.0 and int(b.step_count.item()) == 0
    else:
        assert torch.equal(a.m, b.m) and torch.equal(a.v, b.v) and int(b.step_count.item()) == 3
        for _ in range(2):
            a.step()
            b.step()
        torch.cuda.synchronize()
        # the same updates (up to the order of the adjoint's float atomics)
        torch.testing.assert_close(b.params, a.params, rtol=1e-4, atol=1e-6)


def test_host_feed_matches_synchronous_steps():
    """HostFeed (inputs streamed from pinned host memory, the next step's copy
    overlapping the current step, losses read one step behind) gives the same
    loss sequence as copying the inputs and stepping synchronously."""
    from paper_2601_22026_gb300.fit import FitState, HostFeed, boosted_lr
    cams = scenes.periphery_batch_cameras(3, n_crops=3, **KW)
    V = len(cams["width"])
    tgt = FitState(scenes.random_gaussians(5000, 3, 92, log_scale_mean=-4.0), cams, bg=np.zeros((V, 3), np.float32))
    tgt.forward()
    host_rgb = tgt.rgb.cpu().pin_memory()
    host_alpha = tgt.alpha.cpu().pin_memory()
    bgs = torch.from_numpy(scenes.backgrounds(V, 93, n_steps=6)).pin_memory()
    runs = []
    for streamed in (False, True):
        st = FitState(scenes.random_gaussians(5000, 3, 91, log_scale_mean=-4.0), cams, bg=bgs[0].numpy(),
                      lr=boosted_lr())
        st.capture()
        losses = []
        if streamed:
            feed = HostFeed(st)
            feed.prefetch(host_rgb, host_alpha, bgs[0])
            prev = None
            for k in range(6):
                if k + 1 < 6:
                    feed.prefetch(host_rgb, host_alpha, bgs[k + 1])
                h = feed.step()
                if prev is not None:
                    losses.append(feed.loss(prev))
                prev = h
            losses.append(feed.loss(prev))
        else:
            for k in range(6):
                st.target_rgb.copy_(host_rgb)
                st.target_alpha.copy_(host_alpha)
                st.bg.copy_(bgs[k])
                st.replay()
                losses.append(float(st.loss_out.item()))
        assert st.check_status() == 0
        runs.append(np.array(losses))
    assert runs[0][0] > runs[0][-1]  # the fit progresses
    np.testing.assert_allclose(runs[1], runs[0], rtol=1e-4)
