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
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import scenes
from noalloc_reset_child import loss_inputs as _inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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
        # the scalar sums are float atomics in completion order: equal up to reordering
        assert float(L_na.item()) == pytest.approx(float(L_ref.item()), rel=1e-5), call
        import oracle
        Lo = oracle.loss(*_inputs(cams, seed), scenes.backgrounds(V, seed + 3), cams)[0]
        assert float(L_na.item()) == pytest.approx(Lo, rel=2e-5), call
        np.testing.assert_allclose(g_na.cpu().numpy(), g_ref.cpu().numpy(), rtol=1e-6, atol=1e-12)
        np.testing.assert_allclose(a_na.cpu().numpy(), a_ref.cpu().numpy(), rtol=1e-6, atol=1e-12)
    # sizes beyond the fixed array are refused
    assert lib.gsfit_loss_noalloc(p(cams_dev), G.GSFIT_MAX_VIEWS + 1, p(rgb), p(alpha), p(trgb), p(talpha), p(bg),
                                  0.2, p(g_na), p(a_na), p(L_na), stream) == G.GSFIT_ERR_INVALID_ARG


def test_loss_noalloc_after_context_reset():
    """The library finds its fixed array's address again after the context
    is reset (in a child process, so this process's CUDA state is kept):
    both entry points agree before and after cudaDeviceReset."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2601_22026_gb300 as pkg
    pkg.build()
    child = os.path.join(os.path.dirname(os.path.abspath(__file__)), "noalloc_reset_child.py")
    r = subprocess.run([sys.executable, child], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    calls = json.loads(r.stdout.strip().splitlines()[-1])
    assert [c["phase"] for c in calls] == [0, 0, 1, 1]
    for c in calls:
        assert c["rc"] == [0, 0], c
        assert c["loss"][1] == pytest.approx(c["loss"][0], rel=1e-5), c
        assert c["grad_rgb_maxdiff"] <= 1e-6 * c["grad_rgb_max"], c
        assert c["grad_alpha_maxdiff"] <= 1e-9, c
