"""Host logic of the convergence ablation: running minimum, iterations to a target, plateau
detection and the summary over synthetic curves with known answers."""
import numpy as np
import pytest

from paper_2507_14046_gb300 import study


def test_running_min_and_targets():
    x = np.array([5.0, 3.0, 4.0, 2.0, 2.5, 1.0])
    np.testing.assert_array_equal(study.running_min(x), [5, 3, 3, 2, 2, 1])
    assert study.iters_to_reach(x, 3.0) == 2
    assert study.iters_to_reach(x, 2.0) == 4
    assert study.iters_to_reach(x, 0.5) is None
    # labelled samples (ERR every 10 iterations)
    assert study.iters_to_reach(x, 2.0, np.arange(10, 70, 10)) == 40
    # within 10 % of the minimum 1.0: only the last sample
    assert study.plateau_iter(x, 0.1) == 6
    # within 100 %: 2.0 reached at the fourth sample
    assert study.plateau_iter(x, 1.0) == 4


def test_oscillating_curve_credited_at_first_reach():
    k = np.arange(1, 1001)
    x = np.exp(-k / 100.0) * (1.0 + 0.5 * np.sin(k))
    t = 0.05
    got = study.iters_to_reach(x, t)
    assert x[got - 1] <= t and np.all(x[:got - 1] > t)


def test_summarise_orders_arms_by_decay_rate():
    n, every = 600, 10
    k = np.arange(1, n + 1)
    it = np.arange(every, n + 1, every)
    rates = {"dip": 400.0, "dip_reg": 300.0, "upws": 60.0, "d2ip": 30.0}
    res = {"loss": {a: 1e-3 + np.exp(-k / r) for a, r in rates.items()},
           "err": {a: 0.3 + np.exp(-it / r) for a, r in rates.items()},
           "err_iters": it}
    s = study.summarise(res, budget=250)
    assert s["targets"]["budget"] == 250
    a = s["arms"]
    assert a["d2ip"]["iters_to_loss_target"] <= 250
    assert a["d2ip"]["iters_to_err_target"] <= 250
    assert a["dip_reg"]["iters_to_loss_target"] is None
    assert a["upws"]["iters_to_err_target"] > a["d2ip"]["iters_to_err_target"]
    assert a["dip"]["iters_to_err_target"] is None or \
        a["dip"]["iters_to_err_target"] > a["upws"]["iters_to_err_target"]
    assert a["d2ip"]["loss_plateau_iter"] < a["upws"]["loss_plateau_iter"] < \
        a["dip"]["loss_plateau_iter"]
    assert a["dip"]["loss_at"][50] == res["loss"]["dip"][49]
    assert a["dip"]["err_at"][100] == res["err"]["dip"][9]


@pytest.mark.gpu
def test_acceleration_ordering_on_the_sequence(d2ip):
    """On frame 2 of the 20-frame 32x32x16 sequence (the paper's schedule: 1800 UPWS
    iterations, 450 on frame 1), the full method starts lowest, UPWS alone next and the
    Kaiming start last, in data loss and in ERR (the ordering of the paper's ablation)."""
    from paper_2507_14046_gb300 import synth
    res = study.run(synth.SEQ_32, iters=200, every=50)
    L, E = res["loss"], res["err"]
    for k in (50, 100, 200):
        assert L["d2ip"][k - 1] < L["upws"][k - 1] < L["dip"][k - 1], k
    assert E["d2ip"][-1] < E["upws"][-1] < E["dip"][-1]
    # the regulariser is small at lambda_tv = 0.002: its fit stays close to plain DIP
    assert abs(L["dip_reg"][-1] - L["dip"][-1]) < 0.05 * L["dip"][-1]


@pytest.mark.gpu
def test_ablation_arms_follow_the_oracle(d2ip):
    """Every arm of the ablation, as study.run drives it through the C ABI (FP32), against the
    oracle's fit of the same arm on a small sequence (8 x 8 x 4 grid, two levels 8/16, lr 1e-3):
    UPWS of 20 iterations on the random task, 10 on frame 1, then 20 traced iterations on
    frame 2 from each arm's start.  Loss traces within 1e-4 relative, per iteration."""
    from oracle import dip, network as onet, tv4d
    from paper_2507_14046_gb300 import synth
    w = synth.Workload("8x8x4 test sequence", (8, 8, 4), 1, 2, (8, 16), 8, 3, 0, 0, 0, 1e-3, 3)
    upws, first, iters, lr, reg = 20, 10, 20, 1e-3, (0.002, 1.0, 0.1, 1e-8)
    res = study.run(w, iters=iters, upws=upws, first=first, every=10, lr=lr, reg=reg)
    J, truth, V, Zin = synth.make_problem(w)
    task = synth.ellipsoid_phantom(w.grid, synth.random_ellipsoids(w.grid, w.seed + 1, 0))
    dV0 = synth.measurements(J, task[None, :], w.seed + 1)[0].astype(np.float64)
    spec = onet.NetSpec(w.grid, w.levels, w.widths, w.c_in)
    table = [(k, o, c, f) for _, _, k, f, o, c in onet.param_layout(spec)]
    theta0 = synth.kaiming_theta(table, w.seed).astype(np.float64)
    Jn, _ = dip.normalise_columns(J)
    Z64, V64 = Zin.astype(np.float64), V.astype(np.float64)
    th_u = dip.fit_frame(spec, Jn, Z64, dV0, theta0, upws, lr).theta
    th_f1 = dip.fit_frame(spec, Jn, Z64, V64[0], th_u, first, lr).theta
    tv = tv4d.regulariser(spec.dims(0), [], reg[0], reg[1], reg[2], reg[3])
    ref = {"dip": dip.fit_frame(spec, Jn, Z64, V64[1], theta0, iters, lr).losses,
           "dip_reg": dip.fit_frame(spec, Jn, Z64, V64[1], theta0, iters, lr, tv).losses,
           "upws": dip.fit_frame(spec, Jn, Z64, V64[1], th_u, iters, lr).losses,
           "d2ip": dip.fit_frame(spec, Jn, Z64, V64[1], th_f1, iters, lr).losses}
    for a in study.ARMS:
        got, want = np.asarray(res["loss"][a]), np.asarray(ref[a])
        assert got.shape == want.shape, a
        err = np.abs(got - want) / want
        print(a, f"max rel loss error {err.max():.2e}")
        assert err.max() < 1e-4, a
