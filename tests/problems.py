"""Seeded problems shared by the GPU parity tests: generator arrays, widened to float64
for the oracle."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from oracle import network as onet
from paper_2507_14046_gb300 import synth


@dataclass
class Problem:
    spec: onet.NetSpec
    J: np.ndarray          # raw float32 (m, n)
    Jn64: np.ndarray       # oracle's column-normalised J (float64)
    truth: np.ndarray      # (T, n) float64
    V: np.ndarray          # (T, m) float32
    Zin: np.ndarray        # (n, c_in) float32
    theta0: np.ndarray     # (P,) float32

    @property
    def n(self):
        return self.J.shape[1]

    @property
    def m(self):
        return self.J.shape[0]


def oracle_table(spec):
    return [(k, o, c, f) for _, _, k, f, o, c in onet.param_layout(spec)]


def make(grid, rings, levels, widths, c_in=8, seed=0, T=1, random_phantom=False, m=None):
    """m: keep the first m rows of J (a measurement count other than 208 per ring, e.g. the
    328 of the paper's 32-electrode, two-layer protocol, reproduced as a shape only)."""
    from oracle import dip
    J = synth.sensitivity_raw(grid, rings, seed)
    if m is not None:
        J = np.ascontiguousarray(J[:m])
    if random_phantom:
        base = synth.ellipsoid_phantom(grid, synth.random_ellipsoids(grid, seed, 0))
    else:
        base = synth.ellipsoid_phantom(grid, synth.lung_pair(grid))
    amp = synth.breathing_amplitude(T) if T > 1 else np.ones(1)
    truth = amp[:, None] * base[None, :]
    V = synth.measurements(J, truth, seed)
    n = J.shape[1]
    Zin = synth.input_noise(n, c_in, seed)
    spec = onet.NetSpec(tuple(grid), levels, tuple(widths), c_in)
    theta0 = synth.kaiming_theta(oracle_table(spec), seed)
    Jn64, _ = dip.normalise_columns(J)
    return Problem(spec, J, Jn64, truth, V, Zin, theta0)


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
