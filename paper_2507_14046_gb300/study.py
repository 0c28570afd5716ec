"""Convergence ablation of the acceleration strategies (Sec. IV-A, the acceleration ablation
of the convergence analysis, and the runtime ablation of Sec. IV-A).

The target is the second frame of a synthetic breathing sequence.  Four starts of the same
DIP fit (lr 5e-4, Adam freshly reset) are run side by side:

* ``dip``      Kaiming weights, data term only (no acceleration, no handcrafted prior);
* ``dip_reg``  Kaiming weights, data term + 4D-TV (a lone frame has no earlier frame, so only
               the spatial term is active);
* ``upws``     the weights after ``upws`` iterations on a random reconstruction task (two
               random ellipsoids measured through the same J), Eq. upws_single;
* ``d2ip``     the ``upws`` weights fitted to frame 1 for ``first`` iterations and carried to
               frame 2 (TPP, Eq. tpp_output2).

Every arm records the per-iteration loss and the ERR of Delta sigma every ``every``
iterations.  Iterations-to-target uses the running minimum of a curve, so a curve that
oscillates (as the paper notes for noise-free data) is credited with the first time it
reaches the level.  Everything runs through the C ABI; the host only compares curves.
"""
from __future__ import annotations

import numpy as np

from . import synth

ARMS = ("dip", "dip_reg", "upws", "d2ip")
CHECKPOINTS = (50, 100, 200, 250, 300, 450, 1000, 1500, 2000, 3000)


def running_min(x: np.ndarray) -> np.ndarray:
    return np.minimum.accumulate(np.asarray(x, dtype=np.float64))


def iters_to_reach(curve: np.ndarray, target: float, iters: np.ndarray | None = None):
    """First iteration count at which the running minimum of ``curve`` is <= ``target``
    (``iters[i]`` labels sample i, default i + 1), or None."""
    rm = running_min(curve)
    hit = np.nonzero(rm <= target)[0]
    if hit.size == 0:
        return None
    i = int(hit[0])
    return int(iters[i]) if iters is not None else i + 1


def plateau_iter(curve: np.ndarray, rel: float = 0.1, iters: np.ndarray | None = None):
    """First iteration at which the running minimum is within a factor (1 + rel) of the
    curve's overall minimum."""
    rm = running_min(curve)
    return iters_to_reach(curve, (1.0 + rel) * rm[-1], iters)


def run(w, iters: int = 3000, upws: int = 1800, first: int = 450, every: int = 10,
        lr: float = 5e-4, precision: str = "fp32", device: int = 0, stream=None,
        reg=(0.002, 1.0, 0.1, 1e-8)) -> dict:
    """Runs the four arms on workload ``w`` (grid, rings, network, seed); returns the loss
    traces ([iters] per arm), the ERR samples and the iteration labels of those samples."""
    from . import binding as B

    J, truth, V, Zin = synth.make_problem(w)
    if V.shape[0] < 2:
        raise ValueError("the study needs a sequence of at least two frames")
    # the random reconstruction task of UPWS: two random ellipsoids through the same J
    task = synth.ellipsoid_phantom(w.grid, synth.random_ellipsoids(w.grid, w.seed + 1, 0))
    dV0 = synth.measurements(J, task[None, :], w.seed + 1)[0]
    prec = {"fp32": B.D2IP_FP32, "bf16": B.D2IP_BF16, "bf16x3": B.D2IP_BF16X3}[precision]

    def ctx(batch):
        c = B.Context(w.grid, w.levels, w.widths, w.c_in, prec, batch, device=device,
                      stream=stream)
        c.load_J(J)
        c.set_optim(lr)
        return c

    c1 = ctx(1)
    theta0 = synth.kaiming_theta([tuple(r) for r in c1.table()], w.seed)
    c1.set_input(Zin, theta0)
    c1.run_steps(dV0[None], upws)                       # UPWS on the random task
    th_u = c1.state()[0][0].copy()
    B.d2ip_reset_optimizer(c1.handle)
    c1.run_steps(V[0][None], first)                     # frame 1 from the UPWS weights
    th_f1 = c1.state()[0][0].copy()
    c1.close()

    starts = {"dip": theta0, "dip_reg": theta0, "upws": th_u, "d2ip": th_f1}
    plain = ("dip", "upws", "d2ip")
    ca = ctx(len(plain))
    ca.set_input(np.tile(Zin[None], (len(plain), 1, 1)), np.stack([starts[a] for a in plain]))
    cr = ctx(1)
    cr.set_input(Zin, theta0)
    cr.set_regularizer(*reg)

    target = truth[1].astype(np.float32)
    loss = {a: [] for a in ARMS}
    err = {a: [] for a in ARMS}
    labels = []
    done = 0
    while done < iters:
        k = min(every, iters - done)
        tr = ca.run_steps(np.tile(V[1][None], (len(plain), 1)), k, trace=True)
        trr = cr.run_steps(V[1][None], k, trace=True)
        done += k
        labels.append(done)
        e = ca.err_ratio(ca.forward(), np.tile(target[None], (len(plain), 1)))
        er = cr.err_ratio(cr.forward(), target[None])
        for j, a in enumerate(plain):
            loss[a].append(tr[:, j])
            err[a].append(e[j])
        loss["dip_reg"].append(trr[:, 0])
        err["dip_reg"].append(er[0])
    ca.close()
    cr.close()
    return {"loss": {a: np.concatenate(loss[a]) for a in ARMS},
            "err": {a: np.asarray(err[a]) for a in ARMS},
            "err_iters": np.asarray(labels, dtype=np.int64),
            "schedule": {"iters": iters, "upws": upws, "first": first, "every": every,
                         "lr": lr, "precision": precision, "reg": list(reg)}}


def summarise(res: dict, budget: int = 250) -> dict:
    """Per arm: loss and ERR at the checkpoints, the best ERR and where it falls, the
    iterations to the arm's own loss plateau (within 10 %) and to two common targets: the
    full D²IP arm's data loss and ERR after ``budget`` iterations (the per-frame budget)."""
    L, E, it = res["loss"], res["err"], res["err_iters"]
    n = len(L["d2ip"])
    b = min(budget, n)
    loss_t = float(running_min(L["d2ip"][:b])[-1])
    kb = int(np.searchsorted(it, b))
    err_t = float(running_min(E["d2ip"][:kb + 1])[-1])
    out = {"targets": {"budget": b, "loss": loss_t, "err": err_t}, "arms": {}}
    for a in ARMS:
        s = {"loss_at": {}, "err_at": {}}
        for c in CHECKPOINTS:
            if c <= n:
                s["loss_at"][c] = float(L[a][c - 1])
            j = np.nonzero(it == c)[0]
            if j.size:
                s["err_at"][c] = float(E[a][j[0]])
        j = int(np.argmin(E[a]))
        s["best_err"] = float(E[a][j])
        s["best_err_iter"] = int(it[j])
        s["loss_plateau_iter"] = plateau_iter(L[a], 0.1)
        s["iters_to_loss_target"] = iters_to_reach(L[a], loss_t) if a != "dip_reg" else None
        s["iters_to_err_target"] = iters_to_reach(E[a], err_t, it)
        out["arms"][a] = s
    return out
