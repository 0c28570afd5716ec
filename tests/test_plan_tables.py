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
