"""The LayerNorm backward fused into the data-gradient epilogue (d2ip_set_ln_backward_fusion):
with it on, fewer kernels run per iteration, one teacher-forced iteration meets the oracle at
the bars of each tensor-core precision (every LayerNorm's dgamma and dbeta is its own tensor
of the per-tensor check), and it agrees with the unfused context to the FP32 summation order
(split precision) -- on a grid with ragged tiles and on the 20-frame workload's network,
whose encoder has stride-2 units after the stem."""
import numpy as np
import pytest

from oracle import dip, network as onet
from tests import problems
from tests.problems import rel

pytestmark = pytest.mark.gpu

# (dsigma, dL/dtheta overall, per tensor) bars of one teacher-forced iteration (the bars of
# tests/test_gpu_bf16x3.py and tests/test_gpu_batched_bf16.py)
BARS = {1: (2e-2, 5e-2, 0.25), 2: (1e-4, 2e-3, 4e-2)}


def _run(d2ip, pb, precision, fused, plan=None):
    s = pb.spec
    c = d2ip.Context(s.grid, s.levels, s.widths, s.c_in, precision, 1, tile_plan=plan)
    c.set_ln_backward_fusion(fused)
    c.load_J(pb.J)
    c.set_input(pb.Zin, pb.theta0)
    c.set_optim(1e-3)
    ds = c.forward()[0]
    c.run_steps(pb.V[:1], 1)
    nk = c.graph_kernels()[0]
    return c, ds, c.grad()[0], nk


@pytest.mark.parametrize("grid,rings,L,widths", [((22, 18, 10), 1, 2, (16, 32)),
                                                 ((32, 32, 16), 2, 3, (16, 32, 64))])
@pytest.mark.parametrize("precision", [1, 2])
def test_fused_layernorm_backward(d2ip, grid, rings, L, widths, precision):
    pb = problems.make(grid, rings, L, widths, seed=7)
    ref = dip.dip_step(pb.spec, pb.Jn64, pb.Zin.astype(np.float64), pb.V[0].astype(np.float64),
                       pb.theta0.astype(np.float64), dip.AdamState.fresh(pb.theta0.size), 1e-3)
    c0, ds0, g0, nk0 = _run(d2ip, pb, precision, False)
    plan, _ = c0.tile_plan()
    _, ds1, g1, nk1 = _run(d2ip, pb, precision, True, plan)
    per = [rel(g1[off:off + cnt], ref.grad[off:off + cnt])
           for _, _, _, _, off, cnt in onet.param_layout(pb.spec)]
    print(f"precision {precision} {grid}: kernels {nk0} -> {nk1}; fused vs oracle dsigma "
          f"{rel(ds1, ref.dsigma):.2e} grad {rel(g1, ref.grad):.2e} worst {max(per):.2e}; "
          f"fused vs unfused grad {rel(g1, g0):.2e}")
    assert nk1 < nk0  # LayerNorm backward launches folded into data gradients
    np.testing.assert_array_equal(ds1, ds0)  # the forward pass is unchanged
    b_ds, b_g, b_t = BARS[precision]
    assert rel(ds1, ref.dsigma) < b_ds and rel(g1, ref.grad) < b_g and max(per) < b_t
    if precision == 2:
        assert rel(g1, g0) < 1e-5
