"""gsfit_loss_noalloc, the loss entry point for callers that cannot allocate
device memory (a real-time frame loop where an allocation could stall the
device, or a plug-in whose host application owns every device allocation):
its accumulators live in a fixed array inside the library instead of a
caller-provided workspace. Called through the C ABI, it must give what
gsfit_loss gives on the same inputs, on two calls in a row (the second call
must not see the first call's sums, which stay in the shared array).

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _inputs(cams, seed):
    """Seeded render / target images in the packed layout (rgb planes, alpha)."""
    import oracle
    off = oracle.pixel_offsets(cams)
    g = scenes.rng(seed)
    img = scenes.smooth_images(cams, seed + 1, channels=4)
    tgt = scenes.smooth_images(cams, seed + 2, channels=4)
    rgb, alpha, trgb, talpha = [], [], [], []
    for v in range(len(cams["width"])):
        P = int(off[v + 1] - off[v])
        a = img[4 * off[v]:4 * off[v + 1]]
        b = tgt[4 * off[v]:4 * off[v + 1]]
        rgb.append(a[:3 * P] + g.normal(0, 0.05, 3 * P).astype(np.float32))
        alpha.append(a[3 * P:])
        trgb.append(b[:3 * P])
        talpha.append(b[3 * P:])
    return [np.concatenate(x) for x in (rgb, alpha, trgb, talpha)]


def test_loss_noalloc_matches_loss_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2601_22026_gb300 as pkg
    from paper_2601_22026_gb300 import gsfit as G
    pkg.build()
    lib = G.load()
    cams = scenes.stack_cameras([scenes.make_camera((0, 0, 3), (0, 0, 0), w, h, fx=50.0)
                                 for w, h in [(70, 45), (33, 64), (129, 97)]])
    V = len(cams["width"])
    table = G.camera_table(cams)
    cams_dev = G.cameras_to_device(table)
    P = table.total_pixels
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    for call, seed in enumerate((101, 202)):  # two calls in a row, different inputs
        rgb, alpha, trgb, talpha = map(dev, _inputs(cams, seed))
        bg = dev(scenes.backgrounds(V, seed + 3))
        # the allocating entry point, with its caller-provided workspace
        ws = torch.zeros(G.gsfit_loss_workspace_size(V) // 4, device="cuda")
        g_ref, a_ref, L_ref = torch.zeros(3 * P, device="cuda"), torch.zeros(P, device="cuda"), torch.zeros(1, device="cuda")
        rc = lib.gsfit_loss(p(cams_dev), V, p(rgb), p(alpha), p(trgb), p(talpha), p(bg), 0.2, p(g_ref), p(a_ref),
                            p(L_ref), p(ws), ws.numel() * 4, stream)
        assert rc == G.GSFIT_OK
        # the allocation-free entry point
        g_na, a_na, L_na = torch.zeros(3 * P, device="cuda"), torch.zeros(P, device="cuda"), torch.zeros(1, device="cuda")
        rc = lib.gsfit_loss_noalloc(p(cams_dev), V, p(rgb), p(alpha), p(trgb), p(talpha), p(bg), 0.2, p(g_na),
                                    p(a_na), p(L_na), stream)
        assert rc == G.GSFIT_OK
        torch.cuda.synchronize()
        assert float(L_na.item()) == pytest.approx(float(L_ref.item()), rel=1e-6), call
        np.testing.assert_allclose(g_na.cpu().numpy(), g_ref.cpu().numpy(), rtol=1e-6, atol=1e-12)
        np.testing.assert_allclose(a_na.cpu().numpy(), a_ref.cpu().numpy(), rtol=1e-6, atol=1e-12)
    # sizes beyond the fixed array are refused
    assert lib.gsfit_loss_noalloc(p(cams_dev), G.GSFIT_MAX_VIEWS + 1, p(rgb), p(alpha), p(trgb), p(talpha), p(bg),
                                  0.2, p(g_na), p(a_na), p(L_na), stream) == G.GSFIT_ERR_INVALID_ARG
