"""The sensitivity products on the tensor cores (d2ip_sensitivity_products_tc, the form the
BF16 precisions use in a context) against the oracle's data term (Eq. 4): r = J x - dv and
g = (2/m) J^T r, for groups of 13 problems (one block of 16 in the MMA's N) and 20 (two
blocks), with measurement counts whose last 128-row tile is ragged (208, 328) or full of two
rings (416), and voxel counts with a ragged last 64-voxel block.

Bars.  Split form (J, x and r as hi + lo, the lo*lo product dropped: operands good to about
2^-17 relative, FP32 accumulation): r and g within 1e-4 of the FP64 oracle (norm-wise).  Plain
BF16 (operands rounded to 8 bits, relative 2^-9 each): 2e-2.  The oracle's g is taken from
the GPU's own r, so it checks the adjoint product alone.  Repeated calls are bit-identical
(fixed-order partial sums)."""
import numpy as np
import pytest

from oracle import dip
from tests.problems import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = [(208, 3960, 13), (416, 2048, 20), (328, 22 * 18 * 10, 13), (416, 48 * 48 * 24, 13)]
BARS = {0: 2e-2, 1: 1e-4}


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("split", [0, 1])
@pytest.mark.parametrize("m,n,B", CASES)
def test_tensor_core_products_against_oracle(d2ip, m, n, B, split):
    rng = np.random.default_rng(m * 7 + n + B + split)
    J = (rng.standard_normal((m, n)) / np.sqrt(n)).astype(np.float32)
    x = rng.standard_normal((B, n)).astype(np.float32)
    dv = rng.standard_normal((B, m)).astype(np.float32)
    stream = torch.cuda.current_stream().cuda_stream
    wsb = d2ip.d2ip_sensitivity_tc_workspace(B, m, n, split)
    assert wsb > 0
    ws = torch.zeros(wsb, dtype=torch.uint8, device="cuda")
    Jd, xd, dvd = _dev(J), _dev(x), _dev(dv)
    outs = []
    for _ in range(2):
        r = torch.zeros((B, m), device="cuda")
        g = torch.zeros((B, n), device="cuda")
        d2ip.d2ip_sensitivity_products_tc(Jd, xd, dvd, r, g, 2.0 / m, B, m, n, split, ws, wsb,
                                          stream)
        torch.cuda.synchronize()
        outs.append((r.cpu().numpy(), g.cpu().numpy()))
    off = (-ws.data_ptr()) % 256
    assert int(ws[off:off + 4].view(torch.int32).item()) == 0
    r, g = outs[0]
    np.testing.assert_array_equal(outs[1][0], r)
    np.testing.assert_array_equal(outs[1][1], g)
    J64 = J.astype(np.float64)
    er = eg = 0.0
    for b in range(B):
        rr, _ = dip.data_term(J64, x[b].astype(np.float64), dv[b].astype(np.float64))
        gg = dip.data_term_grad(J64, r[b].astype(np.float64))
        er, eg = max(er, rel(r[b], rr)), max(eg, rel(g[b], gg))
    print(f"m {m} n {n} B {B} split {split}: r {er:.2e} g {eg:.2e}")
    assert er < BARS[split] and eg < BARS[split]


def test_rejects_unaligned_measurement_count(d2ip):
    assert d2ip.d2ip_sensitivity_tc_workspace(13, 210, 2048, 1) < 0
