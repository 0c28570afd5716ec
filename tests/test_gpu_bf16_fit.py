"""The plain BF16 tensor-core precision of the whole DIP iteration against the FP64 oracle.

Convolutions whose channel counts are multiples of 16 run on tcgen05 with BF16 operands and
FP32 accumulation (the stem's 8 input channels are zero-padded to 16; the 1-channel tail
stays FP32); J products read a BF16 copy of J; every other step is FP32.  BF16 rounds each
operand to 8 significant bits (relative 2^-9), so the per-iteration agreement is about 1e-2,
not the FP32 path's 1e-5.  Any operand precision below about 15 bits (BF16, and TF32 too)
carries the 100-step fit onto a different Adam trajectory, which ends 3e-3 to 4e-3 away from
the oracle's ERR: this precision is bounded at 2e-2 here.  The 1e-3 ERR target is met by the
split precision D2IP_BF16X3 (tests/test_gpu_bf16x3.py)."""
import numpy as np
import pytest

from oracle import dip, network as onet
from tests import problems
from tests.problems import rel

pytestmark = pytest.mark.gpu


def _ctx(d2ip, pb, lr, precision):
    s = pb.spec
    c = d2ip.Context(s.grid, s.levels, s.widths, s.c_in, precision, 1)
    c.load_J(pb.J)
    c.set_input(pb.Zin, pb.theta0)
    c.set_optim(lr)
    return c


def test_bf16_teacher_forced_iteration(d2ip):
    pb = problems.make((16, 16, 8), 1, 2, (16, 32), seed=1)
    Z64, dv = pb.Zin.astype(np.float64), pb.V[0].astype(np.float64)
    st = dip.AdamState.fresh(pb.theta0.size)
    ref = dip.dip_step(pb.spec, pb.Jn64, Z64, dv, pb.theta0.astype(np.float64), st, 1e-3)
    c = _ctx(d2ip, pb, 1e-3, d2ip.D2IP_BF16)
    ds = c.forward()[0]
    tr = c.run_steps(pb.V[:1], 1, trace=True)
    g = c.grad()[0]
    e_ds, e_loss, e_g = rel(ds, ref.dsigma), abs(tr[0, 0] - ref.loss) / ref.loss, rel(g, ref.grad)
    print(f"BF16 iteration: dsigma {e_ds:.2e} loss {e_loss:.2e} grad {e_g:.2e}")
    assert e_ds < 2e-2 and e_loss < 4e-2 and e_g < 5e-2
    per = {name: rel(g[off:off + cnt], ref.grad[off:off + cnt])
           for name, _, _, _, off, cnt in onet.param_layout(pb.spec)}
    assert max(per.values()) < 0.1, per


def test_bf16_frame_fit_err_close_to_oracle(d2ip):
    pb = problems.make((16, 16, 8), 1, 2, (16, 32), seed=0)
    ref = dip.fit_frame(pb.spec, pb.Jn64, pb.Zin.astype(np.float64), pb.V[0].astype(np.float64),
                        pb.theta0, 100, 1e-3)
    e_ref = dip.err_ratio(ref.dsigma, pb.truth[0])
    out = {}
    for prec in (d2ip.D2IP_FP32, d2ip.D2IP_BF16):
        c = _ctx(d2ip, pb, 1e-3, prec)
        ds, res, _ = c.fit_frame(pb.V[:1], 100)
        out[prec] = dip.err_ratio(ds[0], pb.truth[0])
    print(f"ERR oracle {e_ref:.5f} fp32 {out[0]:.5f} bf16 {out[1]:.5f}")
    assert abs(out[0] - e_ref) <= 1e-3 * e_ref
    assert abs(out[1] - e_ref) <= 2e-2 * e_ref
