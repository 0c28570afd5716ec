"""Parity of the paper-form 3D-FastResUNet variant (Sec. III-D; depthwise separable
ResConv3D blocks, SE, ASPP, attention gates, sigmoid tail) on the CUDA path, through the C
ABI, against the FP64 oracle (oracle.fastres):

* the parameter table is bit-identical to the oracle's layout;
* teacher-forced iteration: from the oracle's theta_k (and Adam moments) one step gives
  Delta sigma, the loss, dL/dtheta per tensor and theta_{k+1} within 1e-5 norm-wise;
* batching: two problems in one context equal the same problems run alone (bit-identical);
* a short fit: the loss trace follows the oracle's for 10 steps.
"""
import numpy as np
import pytest

from oracle import dip
from oracle import fastres as ofr
from paper_2507_14046_gb300 import synth
from tests.problems import rel

pytestmark = pytest.mark.gpu
TOL = 1e-5

SHAPES = [((16, 16, 8), 1, 2, (8, 16)),
          ((11, 9, 7), 1, 2, (8, 16)),           # odd grid: ragged levels, 1-voxel bottleneck axis
          ((32, 32, 16), 2, 3, (16, 32, 64))]    # the sequence workload's grid and widths


def make(grid, rings, L, widths, seed=1, c_in=8):
    J = synth.sensitivity_raw(grid, rings, seed)
    truth = synth.ellipsoid_phantom(grid, synth.lung_pair(grid), 0.3)
    V = synth.measurements(J, truth[None], seed)
    n = J.shape[1]
    Z = synth.input_noise(n, c_in, seed)
    spec = ofr.FastSpec(tuple(grid), L, tuple(widths), c_in)
    theta0 = synth.kaiming_theta(ofr.table(spec), seed)
    Jn, _ = dip.normalise_columns(J)
    return spec, J, Jn, V, Z, theta0


def ctx(d2ip, spec, J, Z, theta, lr=1e-3, batch=1):
    c = d2ip.Context(spec.grid, spec.levels, spec.widths, spec.c_in, d2ip.D2IP_FP32, batch,
                     net="fastres")
    c.load_J(J)
    c.set_input(np.tile(Z[None], (batch, 1, 1)), np.tile(theta[None], (batch, 1)))
    c.set_optim(lr)
    return c


@pytest.mark.parametrize("grid,rings,L,widths", SHAPES)
def test_parameter_table_matches_oracle_layout(d2ip, grid, rings, L, widths):
    spec = ofr.FastSpec(tuple(grid), L, tuple(widths), 8)
    c = d2ip.Context(grid, L, widths, 8, d2ip.D2IP_FP32, 1, net="fastres")
    np.testing.assert_array_equal(c.table(), np.array(ofr.table(spec), dtype=np.int64))
    assert c.P == ofr.param_count(spec)


@pytest.mark.parametrize("grid,rings,L,widths", SHAPES)
@pytest.mark.parametrize("k_pre", [0, 2])
def test_teacher_forced_iteration(d2ip, grid, rings, L, widths, k_pre):
    spec, J, Jn, V, Z, theta0 = make(grid, rings, L, widths)
    lr = 1e-3
    Z64, dv = Z.astype(np.float64), V[0].astype(np.float64)
    th = theta0.astype(np.float64)
    st = dip.AdamState.fresh(th.size)
    for _ in range(k_pre):
        th = dip.dip_step(spec, Jn, Z64, dv, th, st, lr).theta
    th32, m32, v32 = (a.astype(np.float32) for a in (th, st.m, st.v))
    st = dip.AdamState(m32.astype(np.float64), v32.astype(np.float64), st.t)
    ref = dip.dip_step(spec, Jn, Z64, dv, th32.astype(np.float64), st, lr)

    c = ctx(d2ip, spec, J, Z, theta0, lr)
    c.set_state(th32[None], m32[None], v32[None], k_pre)
    ds = c.forward()[0]
    tr = c.run_steps(V[:1], 1, trace=True)
    g = c.grad()[0]
    th1, m1, v1, t1 = c.state()
    assert rel(ds, ref.dsigma) < TOL
    assert abs(tr[0, 0] - ref.loss) <= TOL * ref.loss
    bad = [name for name, shape, kind, fan, off, cnt in ofr.param_layout(spec)
           if rel(g[off:off + cnt], ref.grad[off:off + cnt]) >= TOL]
    assert not bad, [(n, rel(g[o:o + k], ref.grad[o:o + k])) for n, _, _, _, o, k in
                     ofr.param_layout(spec) if n in bad][:8]
    assert rel(th1[0], ref.theta) < TOL
    assert rel(m1[0], st.m) < TOL and rel(v1[0], st.v) < TOL
    assert t1 == k_pre + 1


def test_batch_equals_independent_problems(d2ip):
    spec, J, Jn, V, Z, theta0 = make((16, 16, 8), 1, 2, (8, 16))
    th2 = synth.kaiming_theta(ofr.table(spec), 5)
    Z2 = synth.input_noise(Z.shape[0], 8, 5)
    c = d2ip.Context(spec.grid, 2, (8, 16), 8, d2ip.D2IP_FP32, 2, net="fastres")
    c.load_J(J)
    c.set_input(np.stack([Z, Z2]), np.stack([theta0, th2]))
    c.set_optim(1e-3)
    tr = c.run_steps(np.stack([V[0], V[0][::-1].copy()]), 3, trace=True)
    ds = c.forward()
    for i, (zz, tt, vv) in enumerate([(Z, theta0, V[0]), (Z2, th2, V[0][::-1].copy())]):
        s = ctx(d2ip, spec, J, zz, tt)
        tri = s.run_steps(vv[None], 3, trace=True)
        np.testing.assert_array_equal(tri[:, 0], tr[:, i])
        np.testing.assert_array_equal(s.forward()[0], ds[i])


def test_short_fit_follows_oracle(d2ip):
    spec, J, Jn, V, Z, theta0 = make((16, 16, 8), 1, 2, (8, 16))
    lr = 1e-3
    fr = dip.fit_frame(spec, Jn, Z.astype(np.float64), V[0].astype(np.float64),
                       theta0.astype(np.float64), 10, lr)
    c = ctx(d2ip, spec, J, Z, theta0, lr)
    tr = c.run_steps(V[:1], 10, trace=True)[:, 0]
    np.testing.assert_allclose(tr, fr.losses, rtol=1e-4)
    assert rel(c.forward()[0], fr.dsigma) < 1e-4


def test_fp32_only_and_width_rule(d2ip):
    from paper_2507_14046_gb300.binding import D2IPError
    with pytest.raises(D2IPError):
        d2ip.Context((16, 16, 8), 2, (8, 16), 8, d2ip.D2IP_BF16, 1, net="fastres")
    with pytest.raises(D2IPError):
        d2ip.Context((16, 16, 8), 2, (12, 16), 8, d2ip.D2IP_FP32, 1, net="fastres")
