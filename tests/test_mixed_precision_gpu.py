"""The mixed-precision form of the fit step: the SH coefficients stored as
16-bit floats (IEEE half or bfloat16) and read by the projection and its
adjoint; means, opacity logits, rotations, scales, every computed quantity,
the gradients and the Adam state in float32.

Two questions, two kinds of test:
  * parity of the arithmetic: the GPU's 16-bit path against the FP64 oracle
    on inputs whose 16-bit copy is exact (the seeded features snapped to
    16-bit values on the host, the same set given to both sides), at the
    float32 tolerances;
  * the error of the form: the GPU's 16-bit path against the oracle on the
    unrounded features, per output (image, alpha, each gradient group),
    printed as a table; images within 2e-3 for half storage.
"""
import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F = oracle.F
KINDS = ["f16", "bf16"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2601_22026_gb300 as pkg
    pkg.build()


def _round_bf16(x):
    """float32 -> nearest bfloat16 (ties to even), widened back to float32."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32).reshape(np.shape(x))


def _to16(x, kind):
    """Nearest 16-bit value (ties to even) of x, as float64."""
    x = np.asarray(x, np.float64)
    if kind == "f16":
        return x.astype(np.float16).astype(np.float64)
    return _round_bf16(x.astype(np.float32)).astype(np.float64)


def _snapped(gs, kind):
    """A Gaussian set whose 16-bit copy is exact: the SH coefficients are
    16-bit values. Both sides of a parity test get this set."""
    out = dict(gs)
    out["sh"] = _to16(gs["sh"], kind).astype(np.float32)
    return out


def _state(gs, cams, bg, kind):
    from paper_2601_22026_gb300.fit import FitState
    return FitState(gs, cams, bg=bg, features=kind, keep_keys=True)


def _scene(name):
    from test_parity_gpu import _case
    if name == "differentiation_512":
        sc = scenes.differentiation_scene(0)
        return sc["gaussians"], sc["cameras"], sc["bg"]
    return _case(name)


@pytest.mark.parametrize("kind", KINDS)
def test_feature_copy_is_round_to_nearest_even(kind):
    from paper_2601_22026_gb300 import gsfit as G
    gs = scenes.random_gaussians(1237, 3, 51, log_scale_mean=-2.0)
    gs["sh"] = gs["sh"] * np.float32(37.0)  # spread the exponents
    cams = scenes.stack_cameras([scenes.make_camera((0, 0, 3), (0, 0, 0), 32, 32, fx=30.0)])
    st = _state(gs, cams, None, kind)
    torch.cuda.synchronize()
    got = st.features.cpu().view(torch.int16).numpy().view(np.uint16)
    planes = G.pack_params(gs)[3:].astype(np.float64)  # the SH planes

    def bits(x):
        if kind == "f16":
            return x.astype(np.float16).view(np.uint16).astype(np.int64)
        return (_round_bf16(x.astype(np.float32)).view(np.uint32) >> 16).astype(np.int64)

    # the float32 SH coefficients rounded to nearest even, bit for bit
    assert got.shape[0] == G.num_planes(3) - 3
    np.testing.assert_array_equal(got.astype(np.int64), bits(planes))


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("name", ["sh3_uneven_views", "differentiation_512"])
def test_forward_matches_oracle_on_the_16bit_features(kind, name):
    from test_parity_gpu import _pairs_excluding, _pixel_tile_mask, _radius_flips, _rgb_to_pixels
    gs, cams, bg = _scene(name)
    gr = _snapped(gs, kind)
    st = _state(gr, cams, bg, kind)
    st.forward()
    torch.cuda.synchronize()
    assert st.check_status() == 0
    ref = oracle.render(gr, cams, bg)
    flips = _radius_flips(st, ref["proj"])
    n_inst = int(st.n_instances.item())
    keys = st.keys[:n_inst].cpu().numpy().view(np.uint64)
    vals = st.vals[:n_inst].cpu().numpy().view(np.uint32)
    gk, gv, bad_g = _pairs_excluding(keys, vals, ref["proj"], cams, st.n, flips)
    rk, rv, bad_o = _pairs_excluding(ref["keys"], ref["vals"], ref["proj"], cams, st.n, flips)
    np.testing.assert_array_equal(gk, rk)
    np.testing.assert_array_equal(gv, rv)
    skip = ref["ambiguous"] | _pixel_tile_mask(cams, bad_g | bad_o)
    ok = ~skip
    assert ok.mean() > 0.98, ok.mean()
    rgb = _rgb_to_pixels(st.rgb.cpu().numpy().astype(np.float64), cams)
    assert np.abs(rgb - _rgb_to_pixels(ref["rgb"], cams))[ok].max() <= 1e-4
    assert np.abs(st.alpha.cpu().numpy() - ref["alpha"])[ok].max() <= 1e-4
    np.testing.assert_array_equal(st.n_contrib.cpu().numpy()[ok], ref["n_contrib"][ok])


@pytest.mark.parametrize("kind", KINDS)
def test_gradients_match_oracle_on_the_16bit_features(kind):
    from test_parity_gpu import _grad_check
    gs, cams, bg = _scene("sh3_uneven_views")
    gr = _snapped(gs, kind)
    P = scenes.num_pixels(cams)
    w_rgb = scenes.cotangents(3 * P, 701, 1e-3)
    w_a = scenes.cotangents(P, 702, 1e-3)
    st = _state(gr, cams, bg, kind)
    st.forward()
    st.dL_drgb.copy_(torch.from_numpy(w_rgb))
    st.dL_dalpha.copy_(torch.from_numpy(w_a))
    st.render_bwd()
    torch.cuda.synchronize()
    ref = oracle.render_bwd(gr, cams, bg, w_rgb.astype(np.float64), w_a.astype(np.float64))
    amb = ref["gauss_ambiguous"].any(axis=0) | (oracle.project(gr, cams)[:, :, F["near_boundary"]] > 0).any(axis=0)
    assert amb.mean() < 0.05
    _grad_check(st.gradients(), ref["grads"], amb)


@pytest.mark.parametrize("kind", KINDS)
def test_error_of_the_16bit_form_against_full_precision(kind):
    """Per-output error of the 16-bit form against the FP64 oracle on the
    unrounded float32 features (SH 3, 50k Gaussians, one 512^2 view), and the
    bounds of the mixed-precision target for the half form: images within
    2e-3, gradients within 1e-3 relative.

    Only colours are stored in 16 bits, and the compositing's skip, clamp and
    stop decisions depend on the splat geometry and opacity alone: the oracle
    takes the same decision at every pixel on both feature sets (checked).
    Pixels the oracle flags as near a threshold (where the float32 GPU and the
    FP64 oracle may legitimately decide differently, as in the float32 form)
    are left out of the image bounds and counted."""
    from test_parity_gpu import _rgb_to_pixels
    gs, cams, bg = _scene("differentiation_512")
    P = scenes.num_pixels(cams)
    w_rgb = scenes.cotangents(3 * P, 711, 1e-3)
    w_a = scenes.cotangents(P, 712, 1e-3)
    st = _state(gs, cams, bg, kind)
    st.forward()
    st.dL_drgb.copy_(torch.from_numpy(w_rgb))
    st.dL_dalpha.copy_(torch.from_numpy(w_a))
    rgb = _rgb_to_pixels(st.rgb.cpu().numpy().astype(np.float64), cams)
    alpha = st.alpha.cpu().numpy().astype(np.float64)
    st.render_bwd()
    torch.cuda.synchronize()
    ref = oracle.render(gs, cams, bg)
    ref16 = oracle.render(_snapped(gs, kind), cams, bg)
    refg = oracle.render_bwd(gs, cams, bg, w_rgb.astype(np.float64), w_a.astype(np.float64))
    # rounding colours moves no decision
    np.testing.assert_array_equal(ref["n_contrib"], ref16["n_contrib"])
    np.testing.assert_array_equal(ref["n_blended"], ref16["n_blended"])
    same = ~ref["ambiguous"] & ~ref16["ambiguous"]
    err = np.abs(rgb - _rgb_to_pixels(ref["rgb"], cams))
    aerr = np.abs(alpha - ref["alpha"])
    rows = {"image, max abs (unflagged pixels)": float(err[same].max()),
            "image, max abs (all pixels)": float(err.max()),
            "image, mean abs (all pixels)": float(err.mean()),
            "alpha, max abs (unflagged pixels)": float(aerr[same].max()),
            "alpha, max abs (all pixels)": float(aerr.max()),
            "pixels flagged near a threshold": float(1.0 - same.mean())}
    grads = st.gradients()
    for k in ["means", "log_scales", "quats", "opacity_logits", "sh"]:
        a = np.asarray(grads[k], np.float64).reshape(-1)
        b = np.asarray(refg["grads"][k], np.float64).reshape(-1)
        rows[f"grad {k}, rel. norm"] = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    print(f"\n16-bit form ({kind}) vs FP64 oracle on float32 features, 50k Gaussians SH3, 512x512:")
    for k, v in rows.items():
        print(f"  {k:36s} {v:.3e}")
    assert rows["pixels flagged near a threshold"] <= 0.02
    assert rows["image, max abs (all pixels)"] <= 2.0 / 255.0  # at most about one threshold jump
    if kind == "f16":
        assert rows["image, max abs (unflagged pixels)"] <= 2e-3
        assert rows["alpha, max abs (unflagged pixels)"] <= 2e-3
        for k in ["means", "log_scales", "quats", "opacity_logits", "sh"]:
            assert rows[f"grad {k}, rel. norm"] <= 1e-3, k
    else:
        # bfloat16 keeps 8 significant bits (half: 11): sanity bounds only
        assert rows["image, max abs (unflagged pixels)"] <= 4e-3
        for k in ["means", "log_scales", "quats", "opacity_logits", "sh"]:
            assert rows[f"grad {k}, rel. norm"] <= 5e-3, k


def test_error_of_the_half2_exponent_option():
    """The half2-exponent option of the half form: 16-bit features and
    exp(power) of every (pixel, Gaussian) pair in packed half precision (the
    forward pass takes two Gaussians per instruction). Error against the FP64
    oracle on the unrounded float32 features, per output. Besides the feature
    rounding, half precision rounds power (at most 2^-9 absolute for
    |power| <= 5.6, the range that passes the alpha test) and exp (2^-11
    relative): the weight moves by at most about 3e-3 relative, so pixels where
    a decision could move are found with the oracle's threshold flags widened
    to 5e-3 relative; the 2e-3 image bound applies to the others."""
    from paper_2601_22026_gb300.fit import FitState
    from test_parity_gpu import _rgb_to_pixels
    gs, cams, bg = _scene("differentiation_512")
    P = scenes.num_pixels(cams)
    w_rgb = scenes.cotangents(3 * P, 711, 1e-3)
    w_a = scenes.cotangents(P, 712, 1e-3)
    st = FitState(gs, cams, bg=bg, features="f16", exp_half2=True)
    assert st.opts.exp_half2 == 1
    st.forward()
    st.dL_drgb.copy_(torch.from_numpy(w_rgb))
    st.dL_dalpha.copy_(torch.from_numpy(w_a))
    rgb = _rgb_to_pixels(st.rgb.cpu().numpy().astype(np.float64), cams)
    alpha = st.alpha.cpu().numpy().astype(np.float64)
    st.render_bwd()
    torch.cuda.synchronize()
    assert st.check_status() == 0
    with oracle.threshold_margin(5e-3):
        ref = oracle.render(gs, cams, bg)
        ref16 = oracle.render(_snapped(gs, "f16"), cams, bg)
    refg = oracle.render_bwd(gs, cams, bg, w_rgb.astype(np.float64), w_a.astype(np.float64))
    same = ((ref["n_contrib"] == ref16["n_contrib"]) & (ref["n_blended"] == ref16["n_blended"]) &
            ~ref["ambiguous"] & ~ref16["ambiguous"])
    err = np.abs(rgb - _rgb_to_pixels(ref["rgb"], cams))
    aerr = np.abs(alpha - ref["alpha"])
    rows = {"image, max abs (same decisions)": float(err[same].max()),
            "image, max abs (all pixels)": float(err.max()),
            "image, mean abs (all pixels)": float(err.mean()),
            "alpha, max abs (same decisions)": float(aerr[same].max()),
            "pixels with a changed or near decision": float(1.0 - same.mean())}
    grads = st.gradients()
    for k in ["means", "log_scales", "quats", "opacity_logits", "sh"]:
        a = np.asarray(grads[k], np.float64).reshape(-1)
        b = np.asarray(refg["grads"][k], np.float64).reshape(-1)
        rows[f"grad {k}, rel. norm"] = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    print("\nhalf form with the half2 exponent vs FP64 oracle on float32 features, 50k Gaussians SH3, 512x512:")
    for k, v in rows.items():
        print(f"  {k:40s} {v:.3e}")
    assert rows["pixels with a changed or near decision"] <= 0.5
    assert rows["image, max abs (all pixels)"] <= 2.0 / 255.0
    assert rows["image, mean abs (all pixels)"] <= 3e-4
    assert rows["image, max abs (same decisions)"] <= 2e-3
    assert rows["alpha, max abs (same decisions)"] <= 2e-3
    for k in ["means", "log_scales", "quats", "opacity_logits", "sh"]:
        assert rows[f"grad {k}, rel. norm"] <= 3e-2, k


def test_half2_exponent_pairs_do_not_matter():
    """exp(power) of a pair is evaluated in one f16x2 instruction next to
    whichever Gaussian shares it: the forward pairs list entries two by two,
    the adjoint evaluates one at a time. With identical values either way the
    adjoint takes the forward's decisions: its T recovery ends at T = 1 in
    front of the first Gaussian, which the gradients of the opacity would
    otherwise betray. Checked here as: the half2 form's image and gradients
    against the float32-exponent form on the same half features, closer than
    the threshold jumps allow for a mismatch."""
    from paper_2601_22026_gb300.fit import FitState
    gs, cams, bg = _scene("differentiation_512")
    P = scenes.num_pixels(cams)
    w_rgb = torch.from_numpy(scenes.cotangents(3 * P, 721, 1e-3))
    w_a = torch.from_numpy(scenes.cotangents(P, 722, 1e-3))
    out = {}
    for e16 in (False, True):
        st = FitState(gs, cams, bg=bg, features="f16", exp_half2=e16)
        st.forward()
        st.dL_drgb.copy_(w_rgb)
        st.dL_dalpha.copy_(w_a)
        st.render_bwd()
        torch.cuda.synchronize()
        assert st.check_status() == 0
        out[e16] = (st.rgb.cpu().numpy().astype(np.float64), st.gradients())
    # half precision moves each weight by at most about 3e-3 relative: a
    # typical pixel moves by well under 1e-4; a pixel whose decision moves by
    # at most one threshold jump
    d = np.abs(out[True][0] - out[False][0])
    assert np.median(d) <= 1e-4 and d.mean() <= 1e-4 and d.max() <= 2.0 / 255.0
    for k in ["means", "opacity_logits", "sh"]:
        a = np.asarray(out[True][1][k], np.float64).reshape(-1)
        b = np.asarray(out[False][1][k], np.float64).reshape(-1)
        assert np.linalg.norm(a - b) <= 3e-2 * np.linalg.norm(b), k


@pytest.mark.parametrize("kind", KINDS)
def test_adam_writes_the_rounded_features(kind):
    from paper_2601_22026_gb300 import gsfit as G
    n, deg = 1003, 1
    npl = G.num_planes(deg)
    g = scenes.rng(43)
    p0 = g.normal(size=(npl, n, 4)).astype(np.float32)
    lr = G.lr_table(deg, 1e-3, 2e-3, 3e-3, 4e-3, 5e-3)
    P = torch.from_numpy(p0.copy()).cuda()
    m, v = torch.zeros_like(P), torch.zeros_like(P)
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    tdt = torch.float16 if kind == "f16" else torch.bfloat16
    feats = torch.zeros((npl - 3, n, 4), dtype=tdt, device="cuda")
    rp, rm, rv = p0.astype(np.float64).reshape(-1), np.zeros(p0.size), np.zeros(p0.size)
    lr_full = np.broadcast_to(lr[:, None, :], p0.shape).reshape(-1).astype(np.float64)
    for k in range(1, 3):
        gr = g.normal(size=p0.shape).astype(np.float32)
        G.gsfit_adam_step(P, torch.from_numpy(gr).cuda(), m, v, n, npl, lr, 0.9, 0.999, 1e-15, step,
                          features=feats, feature_dtype=G.FEATURES[kind])
        oracle.adam(rp, gr.astype(np.float64).reshape(-1), rm, rv, lr_full, 0.9, 0.999, 1e-15, k)
    torch.cuda.synchronize()
    got = feats.cpu().view(torch.int16).numpy().view(np.int16).astype(np.int64)
    ref = rp.reshape(p0.shape)[3:].copy()  # the SH planes
    if kind == "f16":
        want = ref.astype(np.float16).view(np.int16).astype(np.int64)
    else:
        want = (_round_bf16(ref.astype(np.float32)).view(np.uint32) >> 16).astype(np.uint16).view(np.int16)
        want = want.astype(np.int64)
    # the float32 update and the FP64 one may round to neighbouring 16-bit values
    assert np.abs(got - want).max() <= 1
    assert (got == want).mean() > 0.99
    # planes 0-2 have no 16-bit copy; the float32 master update matches as in the float32 test
    np.testing.assert_allclose(P.cpu().numpy().reshape(-1), rp, rtol=2e-6, atol=1e-7)
