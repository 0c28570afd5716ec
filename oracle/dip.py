"""Oracle: the D²IP per-frame fit, UPWS and TPP, in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Readings of the paper used here:
* Eq. 1: the sensitivity matrix J is column-normalised before use (each column scaled to
  unit l2 norm); no projection step (the paper does not give its recipe).
* Eq. 4 with the l2 norm (Sec. III-A) as a mean square: L = (1/M) ||J dsigma - dv||^2, so
  dL/d dsigma = (2/M) J^T (J dsigma - dv).
* Adam (Sec. III-A) with beta1 0.9, beta2 0.999, eps 1e-8 and bias correction; no weight
  decay.  The output of a frame is phi at the last iterate (Eq. 6).
* UPWS (Eqs. 5-7): N_0 steps on one frame from the initial weights; the result starts
  frame 1.  TPP (Eqs. 8-9): each frame starts from the previous frame's final weights.
  Only the weights are carried; the Adam moments and step count restart at each frame.
* ERR = ||dsigma_hat - dsigma_true|| / ||dsigma_true|| (Sec. V-A names it, no formula).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import network

BETA1, BETA2, ADAM_EPS = 0.9, 0.999, 1e-8


def _net(spec):
    """The network module of a spec: the paper-form variant for a FastSpec, else the
    residual U-Net."""
    from . import fastres
    return fastres if isinstance(spec, fastres.FastSpec) else network


def normalise_columns(J) -> tuple[np.ndarray, np.ndarray]:
    """Column-normalised J (Eq. 1) and the column norms c_j = ||J[:, j]||_2."""
    J = np.asarray(J, dtype=np.float64)
    c = np.sqrt((J * J).sum(axis=0))
    return J / c[None, :], c


def data_term(J, dsigma, dv):
    """r = J dsigma - dv and L = (1/M) r.r (l2 data fidelity of Eq. 4, as a mean)."""
    r = J @ dsigma - dv
    return r, float(r @ r) / J.shape[0]


def data_term_grad(J, r):
    """dL/d dsigma = (2/M) J^T r."""
    return (2.0 / J.shape[0]) * (J.T @ r)


@dataclass
class AdamState:
    m: np.ndarray
    v: np.ndarray
    t: int = 0

    @staticmethod
    def fresh(n: int) -> "AdamState":
        return AdamState(np.zeros(n), np.zeros(n), 0)


def adam_step(theta, g, st: AdamState, lr, b1=BETA1, b2=BETA2, eps=ADAM_EPS):
    """One Adam update (Kingma & Ba, Algorithm 1): returns the new theta; updates ``st``."""
    st.t += 1
    st.m = b1 * st.m + (1.0 - b1) * g
    st.v = b2 * st.v + (1.0 - b2) * g * g
    mhat = st.m / (1.0 - b1 ** st.t)
    vhat = st.v / (1.0 - b2 ** st.t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps)


@dataclass
class StepResult:
    dsigma: np.ndarray      # phi(theta_k | Z) (before the update)
    loss: float             # L at theta_k
    grad: np.ndarray        # dL/dtheta at theta_k
    theta: np.ndarray       # theta_{k+1}


def dip_step(spec, J, Zin, dv, theta, st: AdamState, lr, reg=None) -> StepResult:
    """One DIP iteration: forward phi, data term (+ optional regulariser callback
    ``reg(dsigma) -> (value, gradient)``), backward through J^T and phi, Adam."""
    net = _net(spec)
    ds, kept = net.forward(spec, theta, Zin, keep=True)
    r, loss = data_term(J, ds, dv)
    gds = data_term_grad(J, r)
    if reg is not None:
        rv, rg = reg(ds)
        loss += rv
        gds = gds + rg
    g = net.backward(spec, kept, gds)
    return StepResult(ds, loss, g, adam_step(np.asarray(theta, np.float64), g, st, lr))


@dataclass
class FrameResult:
    theta: np.ndarray
    dsigma: np.ndarray                  # phi(theta^(N) | Z) (Eq. 6)
    residual: float                     # (1/M)||J dsigma - dv||^2 at that output
    losses: list = field(default_factory=list)


def fit_frame(spec, J, Zin, dv, theta0, n_steps, lr, reg=None, state=None) -> FrameResult:
    """N Adam steps on one frame (Eq. 4), output phi at the last iterate (Eq. 6).
    A fresh Adam state is used unless ``state`` is given."""
    theta = np.asarray(theta0, dtype=np.float64).copy()
    st = state if state is not None else AdamState.fresh(theta.size)
    losses = []
    for _ in range(n_steps):
        res = dip_step(spec, J, Zin, dv, theta, st, lr, reg)
        losses.append(res.loss)
        theta = res.theta
    ds = _net(spec).forward(spec, theta, Zin)
    _, resid = data_term(J, ds, dv)
    return FrameResult(theta, ds, resid, losses)


@dataclass
class SequenceResult:
    Sigma: np.ndarray                   # (T, n)
    residuals: np.ndarray               # (T,)
    theta: np.ndarray                   # weights after the last frame
    theta_upws: np.ndarray              # weights after UPWS


def fit_sequence(spec, J, Zin, V, theta0, upws_steps, first_steps, later_steps, lr,
                 dv0=None, reg_factory=None, carry_state=False) -> SequenceResult:
    """UPWS (Eqs. 5-7) then TPP over the frames (Eqs. 8-9).

    UPWS runs ``upws_steps`` on ``dv0`` (default: frame 0) from ``theta0``; frame 0 then
    runs ``first_steps`` from the UPWS result and every later frame ``later_steps`` from
    the previous frame's weights.  ``reg_factory(i, previous_outputs)`` may return a
    regulariser callback for frame i.  The paper carries only the weights (a fresh Adam
    state per frame, the default); ``carry_state`` instead keeps one Adam state (moments and
    step count) through UPWS and all frames.
    """
    V = np.atleast_2d(np.asarray(V, dtype=np.float64))
    theta = np.asarray(theta0, dtype=np.float64).copy()
    st = AdamState.fresh(theta.size) if carry_state else None
    if upws_steps > 0:
        d0 = V[0] if dv0 is None else np.asarray(dv0, dtype=np.float64)
        reg = reg_factory(-1, []) if reg_factory else None
        theta = fit_frame(spec, J, Zin, d0, theta, upws_steps, lr, reg, state=st).theta
    theta_upws = theta.copy()
    outs, res = [], []
    for i in range(V.shape[0]):
        reg = reg_factory(i, list(outs)) if reg_factory else None
        fr = fit_frame(spec, J, Zin, V[i], theta, first_steps if i == 0 else later_steps,
                       lr, reg, state=st)
        theta = fr.theta
        outs.append(fr.dsigma)
        res.append(fr.residual)
    return SequenceResult(np.array(outs), np.array(res), theta, theta_upws)


def err_ratio(dsigma_hat, dsigma_true) -> float:
    """ERR = ||dsigma_hat - dsigma_true||_2 / ||dsigma_true||_2."""
    a = np.asarray(dsigma_hat, np.float64)
    b = np.asarray(dsigma_true, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
