"""The split BF16 precision (D2IP_BF16X3) against the FP64 oracle.

Every convolution operand v is carried as hi = bf16(v) and lo = bf16(v - hi), and the
tensor cores sum hi*hi + lo*hi + hi*lo with FP32 accumulation, so an operand keeps about
16 significant bits (relative 2^-17) against plain BF16's 8 (2^-9).  Bars, from evaluating
the same split products in the oracle (FP64 accumulation) on these problems, times 10 for
the FP32 accumulation order of the GPU:
* one teacher-forced iteration: dsigma and the loss within 1e-4 (emulated 1.3e-5); dL/dtheta
  within 2e-3 overall and 4e-2 per tensor -- weight gradients are sums over all voxels
  whose terms cancel, which multiplies the operand error (emulated at 32 x 32 x 16: 2.2e-4
  overall, 4.2e-3 for the worst tensor); theta_1 within 2e-3 (emulated 2.1e-4: the first Adam
  step is about lr sign(g), and elements whose gradient lies below the noise move);
* end to end: ERR of a 100-step frame fit within 1e-3 relative of the oracle's, the target
  of the BF16 workload (plain BF16 ends 3.4e-3 away; it is printed beside); on sequences,
  per frame, the bar below.
"""
import json
import os

import numpy as np
import pytest

from oracle import dip, network as onet
from tests import problems
from tests.problems import rel

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "seq_oracle.json")


def _ctx(d2ip, pb, lr, precision, batch=1):
    s = pb.spec
    c = d2ip.Context(s.grid, s.levels, s.widths, s.c_in, precision, batch)
    c.load_J(pb.J)
    c.set_input(np.tile(pb.Zin[None], (batch, 1, 1)), np.tile(pb.theta0[None], (batch, 1)))
    c.set_optim(lr)
    return c


SHAPES = [((16, 16, 8), 1, 2, (16, 32)),
          ((22, 18, 10), 1, 2, (16, 32)),        # ragged tiles in x, y and z
          ((32, 32, 16), 2, 3, (16, 32, 64))]    # the 20-frame workload's network


@pytest.mark.parametrize("grid,rings,L,widths", SHAPES)
def test_bf16x3_teacher_forced_iteration(d2ip, grid, rings, L, widths):
    pb = problems.make(grid, rings, L, widths, seed=1)
    lr = 1e-3
    Z64, dv = pb.Zin.astype(np.float64), pb.V[0].astype(np.float64)
    st = dip.AdamState.fresh(pb.theta0.size)
    ref = dip.dip_step(pb.spec, pb.Jn64, Z64, dv, pb.theta0.astype(np.float64), st, lr)
    c = _ctx(d2ip, pb, lr, d2ip.D2IP_BF16X3)
    ds = c.forward()[0]
    tr = c.run_steps(pb.V[:1], 1, trace=True)
    g = c.grad()[0]
    th1 = c.state()[0][0]
    per = {name: rel(g[off:off + cnt], ref.grad[off:off + cnt])
           for name, _, _, _, off, cnt in onet.param_layout(pb.spec)}
    e = {"dsigma": rel(ds, ref.dsigma), "loss": abs(tr[0, 0] - ref.loss) / ref.loss,
         "grad": rel(g, ref.grad), "grad_tensor_max": max(per.values()),
         "theta1": rel(th1, ref.theta)}
    print("BF16x3 iteration", grid, {k: f"{v:.2e}" for k, v in e.items()})
    assert e["dsigma"] < 1e-4 and e["loss"] < 1e-4
    assert e["grad"] < 2e-3 and e["grad_tensor_max"] < 4e-2, per
    assert e["theta1"] < 2e-3


def test_bf16x3_after_three_steps_and_batch(d2ip):
    """From the oracle's state after 3 steps, with the problem repeated over a batch of 3:
    every batch member matches the oracle's next step at the bars above."""
    pb = problems.make((16, 16, 8), 1, 2, (16, 32), seed=4)
    lr, Z64, dv = 1e-3, pb.Zin.astype(np.float64), pb.V[0].astype(np.float64)
    th = pb.theta0.astype(np.float64)
    st = dip.AdamState.fresh(th.size)
    for _ in range(3):
        th = dip.dip_step(pb.spec, pb.Jn64, Z64, dv, th, st, lr).theta
    th32, m32, v32 = (a.astype(np.float32) for a in (th, st.m, st.v))
    st = dip.AdamState(m32.astype(np.float64), v32.astype(np.float64), st.t)
    ref = dip.dip_step(pb.spec, pb.Jn64, Z64, dv, th32.astype(np.float64), st, lr)
    c = _ctx(d2ip, pb, lr, d2ip.D2IP_BF16X3, batch=3)
    tile = lambda a: np.ascontiguousarray(np.tile(a[None], (3, 1)))
    c.set_state(tile(th32), tile(m32), tile(v32), 3)
    ds = c.forward()
    c.run_steps(tile(pb.V[0]), 1)
    g = c.grad()
    for b in range(3):
        assert rel(ds[b], ref.dsigma) < 1e-4
        assert rel(g[b], ref.grad) < 2e-3
    np.testing.assert_array_equal(ds[0], ds[2])


def test_bf16x3_frame_fit_err_within_1e3_of_oracle(d2ip):
    """100 Adam steps on the 16 x 16 x 8 frame (lr 1e-3): the split precision ends within
    1e-3 relative ERR of the FP64 oracle; plain BF16 is printed beside it."""
    pb = problems.make((16, 16, 8), 1, 2, (16, 32), seed=0)
    ref = dip.fit_frame(pb.spec, pb.Jn64, pb.Zin.astype(np.float64), pb.V[0].astype(np.float64),
                        pb.theta0, 100, 1e-3)
    e_ref = dip.err_ratio(ref.dsigma, pb.truth[0])
    out = {}
    for prec in (d2ip.D2IP_BF16, d2ip.D2IP_BF16X3):
        ds, _, _ = _ctx(d2ip, pb, 1e-3, prec).fit_frame(pb.V[:1], 100)
        out[prec] = (dip.err_ratio(ds[0], pb.truth[0]), rel(ds[0], ref.dsigma))
    print(f"ERR oracle {e_ref:.6f}; BF16 {out[1][0]:.6f} (rel {abs(out[1][0] - e_ref) / e_ref:.2e}, "
          f"dsigma {out[1][1]:.2e}); BF16x3 {out[2][0]:.6f} "
          f"(rel {abs(out[2][0] - e_ref) / e_ref:.2e}, dsigma {out[2][1]:.2e})")
    assert abs(out[2][0] - e_ref) <= 1e-3 * e_ref


@pytest.mark.parametrize("case", ["seq16", "seq32"])
def test_bf16x3_sequence_per_frame_err_against_oracle(d2ip, case):
    """Short UPWS/TPP sequences against the oracle fits stored by
    tests/golden/make_sequence_oracle.py: seq16 (16 x 16 x 8, widths 16/32) and seq32, the
    20-frame workload's grid and network (32 x 32 x 16, two rings, 16/32/64), lr 5e-4.

    Adam on this loss amplifies small per-step differences, and the amplification grows along
    a sequence: the FP32 path itself (per-iteration agreement 1e-6) drifts to 1e-3 relative ERR
    after about 60 iterations, so a fixed 1e-3 bar cannot hold on every frame for any
    precision.  The split precision's per-iteration gradient error is about ten times the FP32
    path's (1e-5 against 1e-6, teacher-forced tests), so its gaps are held to 10 x the FP32
    path's own: the mean over frames of |ERR - ERR_oracle| / ERR_oracle within max(1e-3, 10 x
    FP32's mean), and of the relative dsigma error at 512 fixed voxels within max(1e-2, 10 x
    FP32's).  Means, not single frames: one frame's gap is one sample of a chaotic process
    (the FP32 path's is 3e-4 on one frame and 4e-3 on the next).  The golden file's floor (the
    oracle's ERR moved by a 1e-7 scaling of theta0) and plain BF16 are printed beside it."""
    with open(GOLDEN) as f:
        gold = json.load(f)["cases"][case]
    c = gold["case"]
    pb = problems.make(tuple(c["grid"]), c["rings"], c["levels"], tuple(c["widths"]),
                       seed=c["seed"], T=c["T"])
    idx = (np.arange(c["samples"], dtype=np.int64) * pb.n) // c["samples"]
    report = {}
    for prec in (d2ip.D2IP_FP32, d2ip.D2IP_BF16, d2ip.D2IP_BF16X3):
        Sig, res = _ctx(d2ip, pb, c["lr"], prec).fit_sequence(pb.V[None], c["upws"], c["first"],
                                                               c["later"])
        rows = []
        for i, fr in enumerate(gold["frames"]):
            e = dip.err_ratio(Sig[0, i], pb.truth[i])
            smp = np.asarray(fr["samples"])
            rows.append((abs(e - fr["err"]) / fr["err"],
                         float(np.abs(Sig[0, i][idx] - smp).max()),
                         rel(Sig[0, i][idx], smp)))
        report[prec] = rows
        print(case, ["FP32", "BF16", "BF16x3"][prec],
              "per frame (ERR rel, dsigma max abs, dsigma rel):",
              [tuple(f"{v:.1e}" for v in r) for r in rows])
    print(case, "oracle floor per frame:", [f"{fr['floor']:.1e}" for fr in gold["frames"]])
    mean = {p: np.mean(np.asarray(r), axis=0) for p, r in report.items()}
    f_err, _, f_ds = mean[d2ip.D2IP_FP32]
    err_rel, _, ds_rel = mean[d2ip.D2IP_BF16X3]
    print(case, f"means: FP32 {f_err:.1e} / {f_ds:.1e}, BF16 {mean[1][0]:.1e} / {mean[1][2]:.1e}, "
          f"BF16x3 {err_rel:.1e} / {ds_rel:.1e}")
    assert err_rel <= max(1e-3, 10 * f_err), (err_rel, f_err)
    assert ds_rel <= max(1e-2, 10 * f_ds), (ds_rel, f_ds)
