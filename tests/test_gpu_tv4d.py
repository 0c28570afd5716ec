"""The 4D-TV regulariser (Sec. III-E) on the GPU against the FP64 oracle: the op alone
(value and gradient, with and without earlier frames), and inside a UPWS/TPP sequence."""
import numpy as np
import pytest

from oracle import dip, tv4d
from tests import problems
from tests.problems import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,nprev", [((5, 7, 9), 0), ((5, 7, 9), 3), ((8, 16, 16), 5)])
def test_tv4d_op_matches_oracle(d2ip, dims, nprev):
    rng = np.random.default_rng(sum(dims) + nprev)
    B = 2
    n = int(np.prod(dims))
    s = rng.standard_normal((B, n)).astype(np.float32)
    prev = rng.standard_normal((B, max(nprev, 1), n)).astype(np.float32)
    lam, ls, lt, eps = 0.002, 1.0, 0.1, 1e-6
    wsb = d2ip.d2ip_tv4d_workspace(B, *dims)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    g = torch.zeros((B, n), device="cuda")
    val = np.zeros(B)
    d2ip.d2ip_tv4d(torch.from_numpy(s).cuda(), torch.from_numpy(prev).cuda(), nprev, g, val, B,
                   *dims, lam, ls, lt, eps, ws, wsb, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for b in range(B):
        reg = tv4d.regulariser(dims, [prev[b, j].astype(np.float64) for j in range(nprev)], lam,
                               ls, lt, eps)
        rv, rg = reg(s[b].astype(np.float64))
        assert abs(val[b] - rv) <= 1e-5 * abs(rv)
        assert rel(g[b].cpu().numpy(), rg) < 1e-5


def test_sequence_with_4dtv_matches_oracle(d2ip):
    pb = problems.make((16, 16, 8), 1, 2, (8, 16), seed=4, T=3)
    lr, up, first, later = 1e-3, 20, 10, 8
    dims = pb.spec.dims(0)
    ref = dip.fit_sequence(pb.spec, pb.Jn64, pb.Zin.astype(np.float64), pb.V, pb.theta0, up,
                           first, later, lr,
                           reg_factory=lambda i, outs: tv4d.regulariser(dims, outs))
    c = d2ip.Context(pb.spec.grid, 2, (8, 16), 8, 0, 1)
    c.load_J(pb.J)
    c.set_input(pb.Zin, pb.theta0)
    c.set_optim(lr)
    c.set_regularizer(tv4d.LAMBDA_TV, tv4d.LAMBDA_S, tv4d.LAMBDA_T, tv4d.TV_EPS)
    Sig, res = c.fit_sequence(pb.V[None], up, first, later)
    for i in range(3):
        e_gpu = dip.err_ratio(Sig[0, i], pb.truth[i])
        e_ref = dip.err_ratio(ref.Sigma[i], pb.truth[i])
        assert abs(e_gpu - e_ref) <= 1e-3 * e_ref, i
    # the regulariser changes the fit: without it the outputs differ
    c2 = d2ip.Context(pb.spec.grid, 2, (8, 16), 8, 0, 1)
    c2.load_J(pb.J)
    c2.set_input(pb.Zin, pb.theta0)
    c2.set_optim(lr)
    Sig2, _ = c2.fit_sequence(pb.V[None], up, first, later)
    assert rel(Sig2[0, 2], Sig[0, 2]) > 1e-6
