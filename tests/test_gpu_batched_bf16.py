"""The tensor-core precisions (BF16 and split BF16x3) with many problems per context, the
form the batched workload runs: every problem of a B = 7 context on a grid whose level-0
convolutions span several persistent-kernel tiles (24 x 24 x 12) against a B = 1 context of
that problem and against the oracle's teacher-forced step; and d2ip_fit_batched over two
uneven groups against separate d2ip_fit_sequence calls.

The forward pass has no reduction across problems, so with the same tilings Delta sigma and
the loss are bit-identical whatever the batch; the weight gradients are split-K sums whose
chunking is sized to fill the GPU for the batch at hand, so they agree to FP32 rounding order
only."""
import numpy as np
import pytest

from oracle import dip, network as onet
from tests import problems
from tests.problems import rel

pytestmark = pytest.mark.gpu

GRID, LEVELS, WIDTHS, B = (24, 24, 12), 3, (16, 32, 64), 7


def _group(seeds):
    pbs = [problems.make(GRID, 2, LEVELS, WIDTHS, seed=s, random_phantom=True) for s in seeds]
    # one J per (grid, m) group, as in the batched workload; measurements of each problem
    # through that J
    base = pbs[0]
    V = np.stack([problems.synth.measurements(base.J, p.truth, s)[0]
                  for p, s in zip(pbs, seeds)])
    return base, pbs, V


def _ctx(d2ip, base, Zs, thetas, precision, batch, tile_plan=None):
    c = d2ip.Context(GRID, LEVELS, WIDTHS, 8, precision, batch, tile_plan=tile_plan)
    c.load_J(base.J)
    c.set_input(np.ascontiguousarray(Zs), np.ascontiguousarray(thetas))
    c.set_optim(5e-4)
    return c


@pytest.mark.parametrize("precision", [1, 2])
def test_batch_of_seven_equals_single_problem_contexts(d2ip, precision):
    seeds = list(range(20, 20 + B))
    base, pbs, V = _group(seeds)
    Zs = np.stack([p.Zin for p in pbs])
    th = np.stack([p.theta0 for p in pbs])
    cb = _ctx(d2ip, base, Zs, th, precision, B)
    ds_b = cb.forward()
    tr_b = cb.run_steps(V, 1, trace=True)
    g_b = cb.grad()
    th_b = cb.state()[0]
    # the single-problem contexts take the batch context's tilings (the autotuner chooses per
    # shape and batch size, and a different tiling sums in a different order)
    plan, _ = cb.tile_plan()
    for i in range(B):
        c1 = _ctx(d2ip, base, Zs[i:i + 1], th[i:i + 1], precision, 1, tile_plan=plan)
        ds1 = c1.forward()
        tr1 = c1.run_steps(V[i:i + 1], 1, trace=True)
        np.testing.assert_array_equal(ds_b[i], ds1[0])
        assert tr_b[0, i] == tr1[0, 0]
        assert rel(g_b[i], c1.grad()[0]) < 1e-5, i
        assert rel(th_b[i], c1.state()[0][0]) < 1e-5, i


# (dsigma, loss, dL/dtheta overall, per tensor) bars of one teacher-forced iteration.
# BF16: operands rounded to 8 bits; evaluating the BF16-rounded products in the oracle on
# the 16 x 16 x 8 problem already gives 7e-3, 4e-3, 2e-2 and 0.1 (the stem's weight
# gradient, a sum over all voxels with cancelling terms), so 2e-2, 4e-2, 5e-2 and 0.25.
# BF16x3: the bars of tests/test_gpu_bf16x3.py.
BARS = {1: (2e-2, 4e-2, 5e-2, 0.25), 2: (1e-4, 1e-4, 2e-3, 4e-2)}


@pytest.mark.parametrize("precision", [1, 2])
def test_batch_of_seven_matches_oracle_step(d2ip, precision):
    """Problems 0 and 5 of the B = 7 context against the oracle's teacher-forced step, at the
    bars of the single-problem iteration tests of each precision."""
    seeds = list(range(30, 30 + B))
    base, pbs, V = _group(seeds)
    Zs = np.stack([p.Zin for p in pbs])
    th = np.stack([p.theta0 for p in pbs])
    cb = _ctx(d2ip, base, Zs, th, precision, B)
    ds_b = cb.forward()
    tr_b = cb.run_steps(V, 1, trace=True)
    g_b = cb.grad()
    for i in (0, 5):
        ref = dip.dip_step(pbs[i].spec, base.Jn64, Zs[i].astype(np.float64),
                           V[i].astype(np.float64), th[i].astype(np.float64),
                           dip.AdamState.fresh(th.shape[1]), 5e-4)
        e_ds, e_g = rel(ds_b[i], ref.dsigma), rel(g_b[i], ref.grad)
        e_l = abs(tr_b[0, i] - ref.loss) / ref.loss
        per = [rel(g_b[i][off:off + cnt], ref.grad[off:off + cnt])
               for _, _, _, _, off, cnt in onet.param_layout(pbs[i].spec)]
        print(f"precision {precision} problem {i}: dsigma {e_ds:.2e} loss {e_l:.2e} "
              f"grad {e_g:.2e} worst tensor {max(per):.2e}")
        b_ds, b_l, b_g, b_t = BARS[precision]
        assert e_ds < b_ds and e_l < b_l and e_g < b_g
        assert max(per) < b_t


@pytest.mark.parametrize("precision", [1, 2])
def test_fit_batched_uneven_groups_equals_separate_sequences(d2ip, precision):
    """Two groups of different grids and batch sizes fitted together by d2ip_fit_batched give
    exactly what each gives alone through d2ip_fit_sequence."""
    T, up, first, later = 3, 10, 5, 4
    groups = []
    for grid, rings, seeds in (((24, 24, 12), 2, (41, 42, 43)), ((16, 16, 8), 1, (44, 45))):
        pbs = [problems.make(grid, rings, LEVELS, WIDTHS, seed=s, T=T, random_phantom=True)
               for s in seeds]
        groups.append((grid, pbs))

    def make_ctx(grid, pbs):
        c = d2ip.Context(grid, LEVELS, WIDTHS, 8, precision, len(pbs))
        c.load_J(pbs[0].J)
        c.set_input(np.stack([p.Zin for p in pbs]), np.stack([p.theta0 for p in pbs]))
        c.set_optim(5e-4)
        return c

    Vs = [np.ascontiguousarray(np.stack([p.V for p in pbs])) for _, pbs in groups]
    alone = []
    for (grid, pbs), V in zip(groups, Vs):
        alone.append(make_ctx(grid, pbs).fit_sequence(V, up, first, later))
    cs = [make_ctx(grid, pbs) for grid, pbs in groups]
    S = [np.zeros((len(pbs), T, pbs[0].n), np.float32) for _, pbs in groups]
    R = [np.zeros((len(pbs), T), np.float64) for _, pbs in groups]
    d2ip.d2ip_fit_batched([c.handle for c in cs], Vs, T, None, up, first, later, S, R)
    for k in range(2):
        np.testing.assert_array_equal(S[k], alone[k][0])
        np.testing.assert_array_equal(R[k], alone[k][1])
