"""Index maps without a GPU: the parameter tables the C ABI plans (d2ip_plan_param_table)
for the residual U-Net and the FastResUNet variant are bit-identical to the oracle's layouts
(offsets, counts, kinds, fan-ins), and bad shapes are refused."""
import numpy as np
import pytest

from oracle import fastres as ofr
from oracle import network as onet

SHAPES = [((16, 16, 8), 2, (8, 16)), ((11, 9, 7), 3, (8, 16, 32)), ((32, 32, 16), 3, (16, 32, 64)),
          ((6, 5, 1), 2, (8, 16)), ((64, 64, 32), 4, (16, 32, 64, 128)), ((7, 6, 5), 1, (8,))]


@pytest.mark.parametrize("grid,L,widths", SHAPES)
def test_resunet_table(d2ip, grid, L, widths):
    rows, P = d2ip.d2ip_plan_param_table("resunet", grid, L, widths, 8)
    spec = onet.NetSpec(grid, L, widths, 8)
    ref = np.array([(k, o, c, f) for _, _, k, f, o, c in onet.param_layout(spec)], dtype=np.int64)
    np.testing.assert_array_equal(rows, ref)
    assert P == onet.param_count(spec)


@pytest.mark.parametrize("grid,L,widths", SHAPES)
def test_fastres_table(d2ip, grid, L, widths):
    rows, P = d2ip.d2ip_plan_param_table("fastres", grid, L, widths, 8)
    spec = ofr.FastSpec(grid, L, widths, 8)
    np.testing.assert_array_equal(rows, np.array(ofr.table(spec), dtype=np.int64))
    assert P == ofr.param_count(spec)


def test_bad_plans_are_refused(d2ip):
    with pytest.raises(d2ip.D2IPError):
        d2ip.d2ip_plan_param_table("resunet", (16, 16, 8), 2, (8, 18), 8)     # not 4-aligned
    with pytest.raises(d2ip.D2IPError):
        d2ip.d2ip_plan_param_table("fastres", (16, 16, 8), 2, (12, 16), 8)    # not 8-aligned
    with pytest.raises(d2ip.D2IPError):
        d2ip.d2ip_plan_param_table("resunet", (0, 16, 8), 2, (8, 16), 8)


def test_seeded_sweep_of_shapes(d2ip):
    """40 seeded random (grid, depth, widths, c_in) draws per network: every plan equals the
    oracle's layout (sizes 1..40 per axis, 1-4 levels, widths multiples of 8 up to 128)."""
    rng = np.random.default_rng(2026)
    for _ in range(40):
        grid = tuple(int(v) for v in rng.integers(1, 41, size=3))
        L = int(rng.integers(1, 5))
        widths = tuple(int(8 * v) for v in rng.integers(1, 17, size=L))
        c_in = int(rng.choice([1, 4, 8, 16]))
        rows, P = d2ip.d2ip_plan_param_table("resunet", grid, L, widths, c_in)
        spec = onet.NetSpec(grid, L, widths, c_in)
        ref = [(k, o, c, f) for _, _, k, f, o, c in onet.param_layout(spec)]
        np.testing.assert_array_equal(rows, np.array(ref, dtype=np.int64))
        rows, P2 = d2ip.d2ip_plan_param_table("fastres", grid, L, widths, c_in)
        fspec = ofr.FastSpec(grid, L, widths, c_in)
        np.testing.assert_array_equal(rows, np.array(ofr.table(fspec), dtype=np.int64))
        assert (P, P2) == (onet.param_count(spec), ofr.param_count(fspec))
