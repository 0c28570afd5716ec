"""Writes seq_oracle.json: FP64 oracle fits of short time sequences for the per-frame
comparison of the GPU precisions, with the oracle's own sensitivity ("floor") per frame.

Cases (UPWS then TPP, Secs. III-B and III-C; lr 5e-4, the paper's simulation value):
* seq16: 16 x 16 x 8 voxels, one ring (M 208), two levels of widths 16/32; 30 warm-start
  iterations on frame 0, then 15 on frame 0 and 10 on each of frames 1-3.
* seq32: the 20-frame workload's grid and network (32 x 32 x 16, two rings, M 416, three
  levels 16/32/64); no warm start, 40 iterations on frame 0 and 10 on each of frames 1-3.
Stored per frame: ERR, the data residual |J dsigma - dv|^2 / M, |dsigma|_2, max |dsigma|,
dsigma at 512 evenly spaced voxels, and the floor: |ERR' - ERR| / ERR where ERR' comes from
the same fit started from theta0 * (1 + 1e-7 sin(index)).  Adam on this loss is sensitive to
its starting point, so a difference between two precisions below the floor says nothing.
Only the input generator (synth, through tests/problems) and the oracle run here.

Usage: python tests/golden/make_sequence_oracle.py   (a few minutes on a CPU)
"""
from __future__ import annotations

import json
import os
import sys
from concurrent.futures import ProcessPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CASES = {
    "seq16": dict(grid=(16, 16, 8), rings=1, levels=2, widths=(16, 32), seed=2, T=4,
                  upws=30, first=15, later=10, lr=5e-4, samples=512),
    "seq32": dict(grid=(32, 32, 16), rings=2, levels=3, widths=(16, 32, 64), seed=0, T=4,
                  upws=0, first=40, later=10, lr=5e-4, samples=512),
}
OUT = os.path.join(HERE, "seq_oracle.json")


def sample_index(n: int, k: int) -> np.ndarray:
    return (np.arange(k, dtype=np.int64) * n) // k


def _fit(args):
    from oracle import dip
    from tests import problems
    name, perturb = args
    c = CASES[name]
    pb = problems.make(c["grid"], c["rings"], c["levels"], c["widths"], seed=c["seed"],
                       T=c["T"])
    th0 = pb.theta0.astype(np.float64)
    if perturb:
        th0 = th0 * (1.0 + 1e-7 * np.sin(np.arange(th0.size)))
    res = dip.fit_sequence(pb.spec, pb.Jn64, pb.Zin.astype(np.float64), pb.V, th0, c["upws"],
                           c["first"], c["later"], c["lr"])
    errs = [dip.err_ratio(res.Sigma[i], pb.truth[i]) for i in range(c["T"])]
    return name, perturb, res.Sigma, res.residuals, errs, pb.n


def main() -> None:
    jobs = [(name, p) for name in CASES for p in (False, True)]
    with ProcessPoolExecutor(max_workers=len(jobs)) as ex:
        runs = {(r[0], r[1]): r for r in ex.map(_fit, jobs)}
    out = {"_source": "oracle.dip.fit_sequence (FP64), written by make_sequence_oracle.py",
           "cases": {}}
    for name, c in CASES.items():
        _, _, Sig, resid, errs, n = runs[(name, False)]
        errs_p = runs[(name, True)][4]
        idx = sample_index(n, c["samples"])
        frames = []
        for i in range(c["T"]):
            ds = Sig[i]
            frames.append({"err": errs[i], "floor": abs(errs_p[i] - errs[i]) / errs[i],
                           "residual": float(resid[i]), "norm": float(np.linalg.norm(ds)),
                           "max_abs": float(np.abs(ds).max()),
                           "samples": [float(v) for v in ds[idx]]})
        out["cases"][name] = {
            "case": {k: list(v) if isinstance(v, tuple) else v for k, v in c.items()},
            "frames": frames}
        print(name, "ERR", [round(f["err"], 6) for f in frames],
              "floor", [f"{f['floor']:.1e}" for f in frames])
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
