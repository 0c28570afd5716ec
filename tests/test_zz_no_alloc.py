"""The allocation-free weight gradient, d2ip_conv3d_wgrad_noalloc, against the
workspace version d2ip_conv3d_wgrad.

It serves callers that cannot allocate device memory when they need the gradient (a
fixed-footprint monitoring loop, or an application whose device memory belongs to another
allocator).  Its partial sums live in a static device array shared by all calls, so two
calls in a row must each give the workspace version's result, whatever the previous call
left behind.  This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-5


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_noalloc_wgrad_matches_workspace_version_on_two_calls(d2ip):
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row with different shapes (stride 2, then stride 1 with batch 3)
    for call, (din, ci, co, k, s, B) in enumerate([((9, 7, 11), 16, 32, 3, 2, 2),
                                                   ((8, 16, 16), 8, 8, 3, 1, 3)]):
        rng = np.random.default_rng(100 + call)
        dout = tuple((d + 2 * ((k - 1) // 2) - k) // s + 1 for d in din)
        x = torch.from_numpy(rng.standard_normal((B, *din, ci)).astype(np.float32)).cuda()
        dy = torch.from_numpy(rng.standard_normal((B, *dout, co)).astype(np.float32)).cuda()
        blk = co * k ** 3 * ci + co
        ws_bytes = d2ip.d2ip_conv3d_wgrad_workspace(B, *din, ci, co, k, s)
        ws = torch.empty(ws_bytes // 4 + 1, device="cuda")
        ref = torch.zeros((B, blk), device="cuda")
        d2ip.d2ip_conv3d_wgrad(x, dy, ref, B, *din, ci, co, k, s, blk, 0, ws, ws_bytes, stream)
        out = torch.full((B, blk), float("nan"), device="cuda")
        d2ip.d2ip_conv3d_wgrad_noalloc(x, dy, out, B, *din, ci, co, k, s, blk, 0, stream)
        torch.cuda.synchronize()
        assert _rel(out.cpu().numpy(), ref.cpu().numpy()) <= TOL, call


def test_noalloc_wgrad_rejects_sizes_beyond_its_scratch(d2ip):
    # 64^3 voxels, 128 -> 128 channels: about 113 MB of partial sums, above the 16 MiB array
    with pytest.raises(d2ip.D2IPError) as e:
        d2ip.d2ip_conv3d_wgrad_noalloc(1, 1, 1, 1, 64, 64, 64, 128, 128, 3, 1, 0, 0, None)
    assert e.value.status == -2
    assert "static scratch" in str(e.value)
