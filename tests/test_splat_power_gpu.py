"""The compositing kernels' splat exponent (Section 4.2: the 3DGS power
-1/2 d^T Sigma'^-1 d at pixel offset d) is evaluated twice per blended pair:
by the forward pass with scalar operations on records as stored, and by the
adjoint with packed two-lane operations on records rearranged in shared
memory. The adjoint replays the forward's skip and stop decisions only if the
two round identically, so this checks bit equality on the device, and that
both are the exponent (against float64)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2601_22026_gb300 as pkg
    pkg.build()


def _conics(rng, n):
    """Inverse covariances of splats with standard deviations 0.3 to 300 px, any orientation."""
    sig = np.exp(rng.uniform(np.log(0.3), np.log(300.0), size=(n, 2)))
    th = rng.uniform(0.0, np.pi, n)
    c, s = np.cos(th), np.sin(th)
    ia, ib = 1.0 / sig[:, 0] ** 2, 1.0 / sig[:, 1] ** 2
    a = c * c * ia + s * s * ib
    b = c * s * (ia - ib)
    cc = s * s * ia + c * c * ib
    return np.stack([a, b, cc, rng.uniform(0.0, 1.0, n)], 1).astype(np.float32), sig


def _edge_rows():
    """Zero, signed-zero and one-ulp offsets, denormal products, large coordinates."""
    one_ulp = np.nextafter(np.float32(1000.0), np.float32(2000.0))
    rows = [
        ((0.5, 0.1, 0.3, 1.0), (10.0, 20.0, 10.0, 20.0)),          # d = 0
        ((0.5, -0.1, 0.3, 1.0), (0.0, 0.0, -0.0, 0.0)),            # d = (+0, 0) from -0
        ((2.0, 0.5, 1.0, 1.0), (1000.0, 7.0, one_ulp, 7.0)),       # d of one ulp
        ((1e-30, 1e-31, 2e-30, 1.0), (1.0, 1.0, 1.0 - 1e-7, 1.0 - 2e-7)),  # denormal products
        ((1e-20, 0.0, 1e-20, 1.0), (3.0, 3.0, 3.0 + 2e-9, 3.0)),   # denormal power
        ((4.0, 1.9, 1.0, 1.0), (4095.0, 4095.0, 4094.75, 4095.5)),  # large coordinates
        ((1e4, 0.0, 1e4, 1.0), (512.0, 512.0, 511.999, 512.001)),   # very narrow splat
    ]
    co = np.array([r[0] for r in rows], np.float32)
    pix = np.array([r[1] for r in rows], np.float32)
    return co, pix


def test_forward_and_adjoint_exponents_round_identically():
    from paper_2601_22026_gb300 import gsfit as G
    rng = np.random.default_rng(5)
    n = 1 << 20
    co, sig = _conics(rng, n)
    px = rng.integers(0, 4096, size=(n, 2)).astype(np.float32)
    uv = (px + rng.normal(0.0, 1.0, (n, 2)) * sig * 3.0).astype(np.float32)
    pix = np.concatenate([px, uv], 1)
    eco, epix = _edge_rows()
    co = np.concatenate([co, eco])
    pix = np.concatenate([pix, epix])
    m = len(co)
    dco = torch.from_numpy(co).cuda()
    dpix = torch.from_numpy(pix).cuda()
    out = torch.empty(m, 2, dtype=torch.float32, device="cuda")
    G.gsfit_selftest_splat_power(dco, dpix, m, out)
    torch.cuda.synchronize()
    res = out.cpu().numpy()
    bits = res.view(np.uint32)
    mismatch = np.nonzero(bits[:, 0] != bits[:, 1])[0]
    assert mismatch.size == 0, (mismatch[:5], res[mismatch[:5]])
    # and it is the exponent: float64 from the same float32 inputs, within the
    # rounding of its few float32 operations relative to the term magnitudes
    c64 = co.astype(np.float64)
    dx = pix[:, 0].astype(np.float64) - pix[:, 2]
    dy = pix[:, 1].astype(np.float64) - pix[:, 3]
    ref = -0.5 * (c64[:, 0] * dx * dx + c64[:, 2] * dy * dy) - c64[:, 1] * dx * dy
    scale = 0.5 * (np.abs(c64[:, 0]) * dx * dx + np.abs(c64[:, 2]) * dy * dy) + np.abs(c64[:, 1] * dx * dy)
    # the offsets themselves are float32 differences (one rounding each)
    scale = scale + (np.abs(c64[:, 0] * dx) + np.abs(c64[:, 1] * dy)) * np.abs(pix[:, 0]) * 2.0 ** -24 \
        + (np.abs(c64[:, 1] * dx) + np.abs(c64[:, 2] * dy)) * np.abs(pix[:, 1]) * 2.0 ** -24
    err = np.abs(res[:, 0] - ref)
    tiny = np.finfo(np.float32).tiny
    assert np.all(err <= 8 * 2.0 ** -24 * scale + 4 * tiny), np.max(err / (scale + tiny))
    # zero offset gives a zero exponent
    assert res[n, 0] == 0.0 and res[n + 1, 0] == 0.0


def test_splat_power_selftest_rejects_bad_arguments():
    from paper_2601_22026_gb300 import gsfit as G
    out = torch.empty(2, dtype=torch.float32, device="cuda")
    with pytest.raises(RuntimeError):
        G.gsfit_selftest_splat_power(None, None, 1, out)
    with pytest.raises(RuntimeError):
        G.gsfit_selftest_splat_power(out, out, -1, out)
    G.gsfit_selftest_splat_power(None, None, 0, None)  # empty: nothing to do
