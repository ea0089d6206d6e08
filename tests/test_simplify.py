"""Simplification by importance (the abbreviated regeneration of Section 4.2):
the importance of a Gaussian is the sum of its blend weights alpha T over the
batch's pixels, and the simplification keeps the Gaussians at or above the
keep-th largest importance. The oracle is pinned on the CPU; the GPU's
importance pass and simplification are compared with it (-m gpu)."""
import numpy as np
import pytest

import oracle
import scenes


def _one_view(W=64, H=48, fx=60.0):
    return scenes.stack_cameras([scenes.make_camera((0.0, 0.0, 3.0), (0, 0, 0), W, H, fx=fx)])


def test_importance_sums_to_the_total_alpha():
    """Per pixel the blend weights telescope to 1 - T_N."""
    gs = scenes.random_gaussians(400, 1, 21, log_scale_mean=-2.5)
    cams = scenes.stack_cameras([scenes.make_camera((0.2, 2.8, 1.0), (0, 0, 0), 96, 72, fx=80.0),
                                 scenes.make_camera((-2.0, 0.5, 2.0), (0.1, 0, 0), 64, 64, fx=60.0)])
    r = oracle.render(gs, cams, scenes.backgrounds(2, 5))
    assert r["importance"].sum() == pytest.approx(r["alpha"].sum(), rel=1e-12)
    assert np.all(r["importance"] >= 0)


def test_lone_gaussian_importance_is_its_alpha_image():
    gs = scenes.random_gaussians(1, 0, 22, log_scale_mean=-2.0)
    gs["means"][:] = 0.0
    r = oracle.render(gs, _one_view(), np.zeros((1, 3)))
    assert r["importance"][0] == pytest.approx(r["alpha"].sum(), rel=1e-12)
    assert r["importance"][0] > 1.0


def test_two_overlapping_gaussians_compose_exactly():
    """Front: sum of its alpha; behind: sum of its alpha times (1 - front alpha),
    from the two single-Gaussian alpha images (no stop applies: T >= 0.01)."""
    gs = scenes.random_gaussians(2, 0, 23, log_scale_mean=-2.0)
    gs["means"][:] = [[0, 0, 0.5], [0.05, 0, -0.5]]  # the camera at z = 3 sees index 0 in front
    gs["log_scales"][:] = -2.0
    gs["quats"][:] = [1, 0, 0, 0]
    gs["opacity_logits"][:] = 6.0  # opacity ~ 0.998: clamped to 0.99 near the centre
    cam, bg = _one_view(), np.zeros((1, 3))
    imp = oracle.render(gs, cam, bg)["importance"]
    a_front = oracle.render({k: v[:1] for k, v in gs.items()}, cam, bg)["alpha"]
    a_back = oracle.render({k: v[1:] for k, v in gs.items()}, cam, bg)["alpha"]
    assert imp[0] == pytest.approx(a_front.sum(), rel=1e-12)
    assert imp[1] == pytest.approx((a_back * (1.0 - a_front)).sum(), rel=1e-12)
    assert imp[0] > imp[1] > 0


def test_simplify_rule():
    gs = {"a": np.arange(10)}
    imp = np.array([5, 1, 9, 3, 9, 0, 7, 2, 8, 4], np.float32)
    kept, idx = oracle.simplify(gs, imp, 4)
    np.testing.assert_array_equal(idx, [2, 4, 6, 8])  # 9, 9, 7, 8: the four largest, in index order
    _, idx = oracle.simplify(gs, imp, 2)
    np.testing.assert_array_equal(idx, [2, 4])
    _, idx = oracle.simplify(gs, np.array([3, 3, 3, 1], np.float32), 2)
    np.testing.assert_array_equal(idx, [0, 1, 2])  # ties at the threshold are all kept
    _, idx = oracle.simplify(gs, imp, 50)
    np.testing.assert_array_equal(idx, np.arange(10))
    _, idx = oracle.simplify(gs, np.array([np.nan, -1, 2, 0], np.float32), 1)
    np.testing.assert_array_equal(idx, [2])


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2601_22026_gb300 as pkg
    pkg.build()
    return torch


@pytest.mark.gpu
def test_gpu_importance_matches_oracle():
    torch = _gpu()
    from paper_2601_22026_gb300 import gsfit as G
    from paper_2601_22026_gb300.fit import FitState
    from test_parity_gpu import _case
    gs, cams, bg = _case("sh3_uneven_views")
    st = FitState(gs, cams, bg=bg)
    st.forward()
    imp = torch.zeros(st.n, device="cuda")
    G.gsfit_render_importance(st.proj, st.cams_dev, st.V, st.n, st.T, st.vals, st.ranges, st.bg, st.rgb, st.alpha,
                              st.T_final, st.n_contrib, imp, None, st.tile_order, st.status, st.opts)
    torch.cuda.synchronize()
    assert st.check_status() == 0
    got = imp.cpu().numpy().astype(np.float64)
    ref = oracle.render(gs, cams, bg)
    r = ref["importance"]
    assert got.sum() == pytest.approx(float(st.alpha.sum().item()), rel=1e-4)
    amb = (ref["proj"][:, :, oracle.F["near_boundary"]] > 0).any(axis=0)
    # a pixel's threshold decisions move whole weights: compare per Gaussian away from flagged pixels' owners
    assert np.abs(got - r).sum() <= 2e-3 * r.sum()
    ok = ~amb & (r > 1e-3 * r.max())
    rel = np.abs(got[ok] - r[ok]) / r[ok]
    assert np.quantile(rel, 0.99) <= 1e-3, np.quantile(rel, 0.99)


@pytest.mark.gpu
@pytest.mark.parametrize("n,keep", [(5000, 300), (300, 1000), (70_000, 12_345)])
def test_gpu_simplify_matches_oracle(n, keep):
    torch = _gpu()
    from paper_2601_22026_gb300 import gsfit as G
    g = scenes.rng(n + keep)
    imp = (g.exponential(1.0, n) * (g.uniform(size=n) > 0.1)).astype(np.float32)
    imp[: n // 50] = imp[n // 2]  # a block of ties
    npl = G.num_planes(1)
    params = g.normal(size=(npl, n, 4)).astype(np.float32)
    P = torch.from_numpy(params).cuda()
    out = torch.zeros_like(P)
    n_out = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(G.gsfit_simplify_workspace_size(n), dtype=torch.uint8, device="cuda")
    G.gsfit_simplify(P, n, npl, torch.from_numpy(imp).cuda(), keep, out, n_out, ws)
    torch.cuda.synchronize()
    m = int(n_out.item())
    _, idx = oracle.simplify({"i": np.arange(n)}, imp, keep)
    assert m == len(idx)
    np.testing.assert_array_equal(out.cpu().numpy()[:, :m], params[:, idx])
