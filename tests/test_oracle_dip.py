"""Pins for the oracle's network composition, data term, Adam and the UPWS/TPP schedule
(no GPU)."""
import json
import os

import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import dip
from oracle import network as net
from paper_2507_14046_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _theta(spec, seed):
    table = [(k, o, c, f) for _, _, k, f, o, c in net.param_layout(spec)]
    return synth.kaiming_theta(table, seed).astype(np.float64)


def _torch_net(spec, theta, Zin):
    """The same U-Net written with torch.nn.functional library ops (NCDHW), for a pin of the
    oracle's composition and (through autograd) of its backward pass."""
    P = {k: torch.from_numpy(v.copy()) for k, v in net.unpack(spec, theta).items()}
    for v in P.values():
        v.requires_grad_(True)

    def conv(x, name, s):
        W = P[name + ".W"].permute(0, 4, 1, 2, 3)  # (co, ci, kz, ky, kx)
        return F.conv3d(x, W, P[name + ".b"], stride=s, padding=(W.shape[2] - 1) // 2)

    def ln(x, name):
        y = F.layer_norm(x.permute(0, 2, 3, 4, 1), (x.shape[1],), P[name + ".g"],
                         P[name + ".beta"], eps=1e-5)
        return y.permute(0, 4, 1, 2, 3)

    act = lambda t: F.leaky_relu(t, 0.2)

    def res(x, name):
        h = act(ln(conv(x, name + ".a", 1), name + ".lna"))
        h = ln(conv(h, name + ".b", 1), name + ".lnb")
        p = conv(x, name + ".p", 1) if (name + ".p.W") in P else x
        return act(h + p)

    x = torch.from_numpy(np.asarray(Zin).reshape(*spec.dims(0), spec.c_in).copy())
    x = x.permute(3, 0, 1, 2)[None]
    e = [res(act(ln(conv(x, "stem", 1), "stem.ln")), "enc0")]
    for l in range(1, spec.levels):
        e.append(res(act(ln(conv(e[-1], f"down{l}", 2), f"down{l}.ln")), f"enc{l}"))
    cur = e[-1]
    for l in range(spec.levels - 2, -1, -1):
        u = F.interpolate(cur, size=spec.dims(l), mode="trilinear", align_corners=False)
        cur = res(torch.cat([u, e[l]], dim=1), f"dec{l}")
    return conv(cur, "tail", 1).reshape(-1), P


SPECS = [net.NetSpec((5, 4, 6), 2, (4, 6), 3), net.NetSpec((7, 6, 5), 3, (3, 4, 5), 2),
         net.NetSpec((16, 16, 8), 2, (8, 16), 8)]


@pytest.mark.parametrize("spec", SPECS)
def test_network_forward_backward_match_torch_reference(spec):
    rng = np.random.default_rng(11)
    n = int(np.prod(spec.grid))
    Zin = 0.1 * rng.standard_normal((n, spec.c_in))
    th = _theta(spec, 5)
    ds, kept = net.forward(spec, th, Zin, keep=True)
    ref, P = _torch_net(spec, th, Zin)
    np.testing.assert_allclose(ds, ref.detach().numpy(), rtol=1e-10, atol=1e-12)
    w = rng.standard_normal(n)
    g = net.backward(spec, kept, w)
    (ref * torch.from_numpy(w)).sum().backward()
    gref = net.pack(spec, {k: v.grad.numpy() for k, v in P.items()})
    np.testing.assert_allclose(g, gref, rtol=1e-9, atol=1e-9 * np.abs(gref).max())


def test_whole_iteration_gradient_finite_difference():
    """dL/dtheta of the full iteration against central differences along one random
    direction per parameter tensor (FP64, h = 1e-5 on a unit direction)."""
    spec = SPECS[0]
    rng = np.random.default_rng(12)
    n = int(np.prod(spec.grid))
    Zin = 0.1 * rng.standard_normal((n, spec.c_in))
    J = rng.standard_normal((30, n))
    dv = rng.standard_normal(30)
    th = _theta(spec, 3)
    ds, kept = net.forward(spec, th, Zin, keep=True)
    r, _ = dip.data_term(J, ds, dv)
    g = net.backward(spec, kept, dip.data_term_grad(J, r))
    L = lambda t: dip.data_term(J, net.forward(spec, t, Zin), dv)[1]
    h = 1e-5
    for name, shape, kind, fi, off, cnt in net.param_layout(spec):
        d = np.zeros_like(th)
        d[off:off + cnt] = rng.standard_normal(cnt)
        d /= np.linalg.norm(d)
        fd = (L(th + h * d) - L(th - h * d)) / (2 * h)
        assert abs(fd - g @ d) <= 1e-6 * max(abs(fd), 1e-3), name


def test_data_term_gradient_and_adjoint():
    rng = np.random.default_rng(13)
    J = rng.standard_normal((17, 40))
    dv = rng.standard_normal(17)
    x = rng.standard_normal(40)
    r, L = dip.data_term(J, x, dv)
    assert np.isclose(L, np.mean((J @ x - dv) ** 2), rtol=1e-14)
    g = dip.data_term_grad(J, r)
    d = rng.standard_normal(40)
    h = 1e-6
    fd = (dip.data_term(J, x + h * d, dv)[1] - dip.data_term(J, x - h * d, dv)[1]) / (2 * h)
    assert abs(fd - g @ d) < 1e-8 * abs(fd)
    # adjoint: <J x, r> = <x, J^T r> through the gradient routine
    assert abs((J @ x) @ r - x @ (dip.data_term_grad(J, r) * 17 / 2)) < 1e-11 * abs((J @ x) @ r)


def test_column_normalisation_and_single_ring_decay_cancels():
    J = synth.sensitivity_raw((8, 6, 5), 1, seed=3)
    Jn, c = dip.normalise_columns(J)
    np.testing.assert_allclose(np.sqrt((Jn ** 2).sum(0)), 1.0, rtol=1e-14)
    # one ring: the decay multiplies every row by the same per-column factor, which the
    # column normalisation removes exactly (up to the float32 rounding of the raw matrix)
    J0 = synth.sensitivity_raw((8, 6, 5), 1, seed=3, decay=False)
    Jn0, _ = dip.normalise_columns(J0)
    np.testing.assert_allclose(Jn, Jn0, rtol=0, atol=1e-6)
    # two rings: it does not cancel
    J2 = synth.sensitivity_raw((8, 6, 5), 2, seed=3)
    J20 = synth.sensitivity_raw((8, 6, 5), 2, seed=3, decay=False)
    assert np.abs(dip.normalise_columns(J2)[0] - dip.normalise_columns(J20)[0]).max() > 1e-2


def test_adam_matches_closed_form_and_torch():
    rng = np.random.default_rng(14)
    th0 = rng.standard_normal(50)
    g1, g2, g3 = (rng.standard_normal(50) for _ in range(3))
    lr = 1e-3
    st = dip.AdamState.fresh(50)
    th1 = dip.adam_step(th0, g1, st, lr)
    # first step from zero moments: the bias corrections cancel
    np.testing.assert_allclose(th1, th0 - lr * g1 / (np.abs(g1) + 1e-8), rtol=1e-15)
    th2 = dip.adam_step(th1, g2, st, lr)
    m2 = (0.09 * g1 + 0.1 * g2) / (1 - 0.9 ** 2)
    v2 = (0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2) / (1 - 0.999 ** 2)
    np.testing.assert_allclose(th2, th1 - lr * m2 / (np.sqrt(v2) + 1e-8), rtol=1e-13)
    th3 = dip.adam_step(th2, g3, st, lr)
    # library special case: torch.optim.Adam in float64
    p = torch.nn.Parameter(torch.from_numpy(th0.copy()))
    opt = torch.optim.Adam([p], lr=lr, betas=(0.9, 0.999), eps=1e-8)
    for g in (g1, g2, g3):
        p.grad = torch.from_numpy(g.copy())
        opt.step()
    np.testing.assert_allclose(th3, p.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_adam_on_least_squares_reaches_normal_equations():
    """Weak pin: with phi(theta) = theta the fit is Adam on least squares; on an
    overdetermined problem it approaches the normal-equation solution."""
    rng = np.random.default_rng(15)
    J = rng.standard_normal((40, 6))
    dv = rng.standard_normal(40)
    x_ls = np.linalg.solve(J.T @ J, J.T @ dv)
    x = np.zeros(6)
    st = dip.AdamState.fresh(6)
    losses = []
    for k in range(6000):
        r, L = dip.data_term(J, x, dv)
        losses.append(L)
        x = dip.adam_step(x, dip.data_term_grad(J, r), st, 1e-2 if k < 3000 else 1e-4)
    assert np.linalg.norm(x - x_ls) < 1e-3 * np.linalg.norm(x_ls)
    assert losses[-1] <= min(losses[:100])


def test_sequence_equals_manual_chaining():
    """UPWS then TPP is fit_frame chained by hand, bit for bit; T=1 with no UPWS is plain
    DIP."""
    spec = net.NetSpec((4, 3, 4), 2, (3, 4), 2)
    rng = np.random.default_rng(16)
    n = 48
    Zin = 0.1 * rng.standard_normal((n, 2))
    J = rng.standard_normal((10, n))
    V = rng.standard_normal((3, 10))
    th = _theta(spec, 2)
    seq = dip.fit_sequence(spec, J, Zin, V, th, 4, 3, 2, 1e-3)
    t = dip.fit_frame(spec, J, Zin, V[0], th, 4, 1e-3).theta
    np.testing.assert_array_equal(seq.theta_upws, t)
    outs = []
    for i in range(3):
        fr = dip.fit_frame(spec, J, Zin, V[i], t, 3 if i == 0 else 2, 1e-3)
        t = fr.theta
        outs.append(fr.dsigma)
    np.testing.assert_array_equal(seq.Sigma, np.array(outs))
    np.testing.assert_array_equal(seq.theta, t)
    one = dip.fit_sequence(spec, J, Zin, V[:1], th, 0, 5, 5, 1e-3)
    np.testing.assert_array_equal(one.Sigma[0], dip.fit_frame(spec, J, Zin, V[0], th, 5,
                                                              1e-3).dsigma)


def test_sequence_carrying_the_adam_state():
    """carry_state keeps one Adam state through UPWS and the frames: on a sequence whose frames
    are all the same measurement, UPWS and the frames together are one uninterrupted fit of
    the total step count (bit for bit), while the paper's fresh state per frame is not."""
    spec = net.NetSpec((4, 3, 4), 2, (3, 4), 2)
    rng = np.random.default_rng(17)
    n = 48
    Zin = 0.1 * rng.standard_normal((n, 2))
    J = rng.standard_normal((10, n))
    v = rng.standard_normal(10)
    V = np.stack([v, v, v])
    th = _theta(spec, 3)
    carry = dip.fit_sequence(spec, J, Zin, V, th, 4, 3, 2, 1e-3, carry_state=True)
    whole = dip.fit_frame(spec, J, Zin, v, th, 4 + 3 + 2 + 2, 1e-3)
    np.testing.assert_array_equal(carry.theta, whole.theta)
    np.testing.assert_array_equal(carry.Sigma[-1], whole.dsigma)
    reset = dip.fit_sequence(spec, J, Zin, V, th, 4, 3, 2, 1e-3)
    assert np.abs(reset.theta - whole.theta).max() > 1e-6


def test_err_ratio():
    assert dip.err_ratio([1.0, 2.0], [1.0, 2.0]) == 0.0
    assert np.isclose(dip.err_ratio([0.0, 0.0], [3.0, 4.0]), 1.0)
    assert np.isclose(dip.err_ratio([3.0, 0.0], [0.0, 4.0]), 5.0 / 4.0)


def test_paper_hyperparameters_fixture():
    """The paper's schedule and loss weights (Sec. IV-D) as stored in the golden fixture are
    the defaults the oracle's regulariser uses."""
    with open(os.path.join(GOLDEN, "paper_hyperparameters.json")) as f:
        gold = json.load(f)
    assert (gold["upws_iters"], gold["first_frame_iters"], gold["later_frame_iters"]) == (
        1800, 450, 250)
    from oracle import tv4d
    assert tv4d.LAMBDA_TV == gold["lambda_tv"]
    assert tv4d.LAMBDA_S == gold["lambda_s"]
    assert tv4d.LAMBDA_T == gold["lambda_t"]
