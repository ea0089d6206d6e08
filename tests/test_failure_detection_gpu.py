"""Failure detection without a GPU fault: every device-side wait is bounded
and reports GSFIT_ERR_TIMEOUT through the status word instead of hanging (the
diagnostics make a wait run out on a barrier or flag that nothing completes,
and the context stays usable); non-finite parameters are culled instead of
poisoning the images; the pair-capacity overflow is reported (the parity tests
cover that one)."""
import numpy as np
import pytest

import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2601_22026_gb300 as pkg
    pkg.build()


def _small_step_works():
    from paper_2601_22026_gb300.fit import FitState
    from test_parity_gpu import _case
    gs, cams, bg = _case("sh1_ragged")
    st = FitState(gs, cams, bg=bg)
    st.step()
    torch.cuda.synchronize()
    assert st.check_status() == 0
    assert torch.isfinite(st.params).all()


def test_mbarrier_wait_runs_out_and_reports():
    from paper_2601_22026_gb300 import gsfit as G
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    G.gsfit_selftest_wait_timeout(2_000_000, status)  # ~1 ms at 2 GHz
    torch.cuda.synchronize()
    assert int(status.item()) == G.GSFIT_ERR_TIMEOUT
    _small_step_works()  # the context is still usable


def test_lookback_wait_runs_out_and_reports():
    from paper_2601_22026_gb300 import gsfit as G
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    word = torch.zeros(1, dtype=torch.int32, device="cuda")  # no flag will ever appear
    G.gsfit_selftest_lookback_timeout(word, 2000, status)
    torch.cuda.synchronize()
    assert int(status.item()) == G.GSFIT_ERR_TIMEOUT
    _small_step_works()


def test_timed_out_status_makes_later_compositing_skip_its_work():
    from paper_2601_22026_gb300 import gsfit as G
    from paper_2601_22026_gb300.fit import FitState
    from test_parity_gpu import _case
    gs, cams, bg = _case("sh1_ragged")
    st = FitState(gs, cams, bg=bg)
    st.project()
    st.bin_sort()
    st.rgb.fill_(-3.0)
    st.status.fill_(G.GSFIT_ERR_TIMEOUT)
    st.render_fwd()
    torch.cuda.synchronize()
    assert float(st.rgb.max().item()) == -3.0  # every tile skipped
    assert st.check_status() == G.GSFIT_ERR_TIMEOUT


@pytest.mark.parametrize("field", ["means", "log_scales", "quats", "opacity_logits", "sh"])
def test_non_finite_gaussians_are_culled(field):
    """A set with NaN Gaussians renders exactly like the same set without
    them (an invariance of the culling, GPU against GPU), and the step's
    gradients stay finite: the culled Gaussians' gradients are zero (they
    reach no pixel), so nothing non-finite is reported either."""
    from paper_2601_22026_gb300.fit import FitState
    from test_parity_gpu import _case
    gs, cams, bg = _case("sh3_uneven_views")
    bad = np.zeros(len(gs["means"]), bool)
    bad[::37] = True
    gs_bad = {k: v.copy() for k, v in gs.items()}
    gs_bad[field][bad] = np.nan
    with_nan = FitState(gs_bad, cams, bg=bg)
    with_nan.forward()
    without = FitState({k: v[~bad] for k, v in gs.items()}, cams, bg=bg)
    without.forward()
    torch.cuda.synchronize()
    assert with_nan.check_status() == 0
    assert torch.equal(with_nan.rgb, without.rgb)
    assert torch.equal(with_nan.alpha, without.alpha)
    with_nan.loss()
    with_nan.render_bwd()
    with_nan.adam()
    torch.cuda.synchronize()
    assert with_nan.check_status() == 0
    g = with_nan.gradients()
    assert all(np.isfinite(np.asarray(v)).all() for v in g.values())
    assert all((np.asarray(v)[bad] == 0).all() for v in g.values())


def test_non_finite_gradient_is_reported():
    """A non-finite upstream gradient (a NaN in dL/dimage at one pixel, as a
    corrupt target image would give) makes the parameter gradients of the
    Gaussians blended there non-finite: the adjoint reports it through the
    status word (GSFIT_ERR_NONFINITE) instead of handing it on silently; the
    same call on finite inputs reports nothing, and the context stays usable."""
    from paper_2601_22026_gb300 import gsfit as G
    from paper_2601_22026_gb300.fit import FitState
    from test_parity_gpu import _case
    gs, cams, bg = _case("sh1_ragged")
    st = FitState(gs, cams, bg=bg)
    st.forward()
    torch.cuda.synchronize()
    P = st.P
    nc = st.n_contrib.cpu().numpy()
    pix = int(np.flatnonzero(nc > 0)[0])  # a pixel where some Gaussian blends
    st.dL_drgb.copy_(torch.from_numpy(scenes.cotangents(3 * P, 901, 1e-3)))
    st.dL_dalpha.copy_(torch.from_numpy(scenes.cotangents(P, 902, 1e-3)))
    st.render_bwd()
    torch.cuda.synchronize()
    assert st.check_status() == 0
    assert torch.isfinite(st.grads).all()
    st.dL_drgb[pix] = float("nan")
    st.render_bwd()
    torch.cuda.synchronize()
    assert st.check_status() == G.GSFIT_ERR_NONFINITE
    assert not torch.isfinite(st.grads).all()
    # the projection adjoint fused with Adam reports it the same way
    st.status.zero_()
    st.keep_grads = True
    st.blend_bwd()
    st.project_bwd_adam()
    torch.cuda.synchronize()
    assert st.check_status() == G.GSFIT_ERR_NONFINITE
    assert not torch.isfinite(st.grads).all()
    _small_step_works()
