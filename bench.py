"""Benchmark of the D²IP fitting path on GB300 (one JSON line on rank 0).

A step is one pass of the whole hot path over one synthetic workload: load and
column-normalise J, set Z and the Kaiming weights, then fit the whole sequence (UPWS on
frame 0, then every frame with TPP) through the C ABI, each DIP iteration being forward,
data term, adjoint, backward and Adam.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload batch64|seq32|...]
                    [--precision bf16x3|bf16|fp32]
    python bench.py --impl reference ...     (the FP64 oracle on the host cores)
    python bench.py --study 3000 [--workload seq32] [--study-out curves.npz]
                                             (convergence ablation of UPWS / TPP)

The default workload is the 64 batched sequences in the split BF16 precision (BF16x3): the
metric compares it with the plain FP32 form at equal ERR, and the line carries the evidence
(plain_fp32: per-frame ERR differences against the FP32 fits of a sample of the sequences,
and the FP32 fits' own floor under 1e-7 changes of their starting weights, four of them).

Multi-GPU: replicas only.  Every rank fits its own copy of the workload (weak scaling);
there is no collective on the data path, only a barrier and a max over ranks of the time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2507_14046_gb300 import replicas, synth  # noqa: E402

METRIC = "DIP iters/s and tsEIT frames/s at equal ERR; BF16 batched vs plain FP32"
UNIT = "DIP iters/s"
WORKLOADS = {"seq32": synth.SEQ_32, "single16": synth.SINGLE_16, "seq64": synth.SEQ_64,
             "batch64": synth.SEQ_32}
FP32_LANES_PER_SM = 128
SMS = 152
PRECISIONS = ("fp32", "bf16", "bf16x3")


def _prec_code(B, name: str) -> int:
    return {"fp32": B.D2IP_FP32, "bf16": B.D2IP_BF16, "bf16x3": B.D2IP_BF16X3}[name]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def iters_per_step(w) -> int:
    return w.upws_steps + w.first_steps + (w.frames - 1) * w.later_steps


# ------------------------------------------------------------------------------------------
# oracle (CPU baseline and the reference arm)
# ------------------------------------------------------------------------------------------

def _oracle_rate(w, grid, rings, iters: int, net: str = "resunet") -> float:
    """Seconds per FP64 oracle DIP iteration of network ``w`` on one seeded problem."""
    from oracle import dip, fastres as ofr, network as onet
    J = synth.sensitivity_raw(grid, rings, w.seed)
    truth = synth.ellipsoid_phantom(grid, synth.lung_pair(grid))[None]
    V = synth.measurements(J, truth, w.seed)
    n = grid[0] * grid[1] * grid[2]
    Zin = synth.input_noise(n, w.c_in, w.seed)
    if net == "fastres":
        spec = ofr.FastSpec(tuple(grid), w.levels, w.widths, w.c_in)
        table = ofr.table(spec)
    else:
        spec = onet.NetSpec(tuple(grid), w.levels, w.widths, w.c_in)
        table = [(k, o, c, f) for _, _, k, f, o, c in onet.param_layout(spec)]
    th = synth.kaiming_theta(table, w.seed).astype(np.float64)
    Jn, _ = dip.normalise_columns(J)
    Z64, dv = Zin.astype(np.float64), V[0].astype(np.float64)
    st = dip.AdamState.fresh(th.size)
    dip.dip_step(spec, Jn, Z64, dv, th, st, w.lr)  # warm the allocator
    t0 = time.perf_counter()
    for _ in range(iters):
        th = dip.dip_step(spec, Jn, Z64, dv, th, st, w.lr).theta
    return (time.perf_counter() - t0) / iters


def oracle_leg(workload: str, iters: int, net: str = "resunet") -> dict:
    """Time FP64 oracle DIP iterations on the workload (first frame, from the Kaiming
    weights); returns iterations/s.  For the batched workload every grid of the mix is timed
    and weighted by its number of sequences."""
    if workload == "batch64":
        shapes = synth.batch_problem_shapes(64, 1)
        w = synth.SEQ_32
        per_grid = {g: (max(1, iters * 4 // 3) if g[0] == 16 else
                        (max(1, iters // 3) if g[0] == 32 else max(1, iters // 6)))
                    for g in synth.BATCH_GRIDS}
        sec, total = 0.0, 0
        for g in synth.BATCH_GRIDS:
            cnt = sum(1 for gg, _ in shapes if gg == g)
            spi = _oracle_rate(w, g, 2, per_grid[g])
            sec += spi * per_grid[g]
            total += per_grid[g]
            per_grid[g] = (per_grid[g], spi, cnt)
        wsec = sum(spi * cnt for _, spi, cnt in per_grid.values()) / 64.0
        return {"iters": total, "seconds": sec, "iters_per_s": 1.0 / wsec,
                "detail": {f"{g[0]}x{g[1]}x{g[2]}": {"iters": k, "s_per_iter": spi,
                                                      "sequences": cnt}
                           for g, (k, spi, cnt) in per_grid.items()}}
    w = WORKLOADS[workload]
    spi = _oracle_rate(w, w.grid, w.rings, iters, net)
    return {"iters": iters, "seconds": spi * iters, "iters_per_s": 1.0 / spi}


def run_oracle_subprocess(workload: str, iters: int, net: str = "resunet",
                          threads: int | None = None) -> dict:
    cores = threads or os.cpu_count() or 1
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(cores)
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-leg", workload,
                          "--oracle-iters", str(iters), "--net", net], capture_output=True,
                         text=True,
                         env=env, check=True)
    res = json.loads(out.stdout.strip().splitlines()[-1])
    res["cores"] = cores
    return res


def oracle_iters_for(workload: str) -> int:
    # about 10-30 s of host work per sample on a Grace host
    return {"single16": 200, "seq32": 12, "seq64": 2, "batch64": 30}[workload]


# ------------------------------------------------------------------------------------------
# clocks
# ------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int, path: str):
        self.path = path
        self.proc = None
        try:
            self.f = open(path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------

def _err(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _clocks_path(args, rank):
    """Where the nvidia-smi samples of the timed region go (--clocks-dir, else the temp dir)."""
    d = args.clocks_dir or os.environ.get("TMPDIR", "/tmp")
    os.makedirs(d, exist_ok=True)
    return os.path.join(d, f"d2ip_clocks_r{rank}.csv")


def run_gpu(args, rank, world, local_rank):
    import torch

    from paper_2507_14046_gb300 import binding as B

    w = WORKLOADS[args.workload]
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    J, truth, V, Zin = synth.make_problem(w)
    stream = torch.cuda.Stream(device=dev)
    prec = _prec_code(B, args.precision)
    ctx = B.Context(w.grid, w.levels, w.widths, w.c_in, prec, 1, device=local_rank,
                    stream=stream.cuda_stream, net=args.net)
    table = ctx.table()
    theta0 = synth.kaiming_theta([tuple(r) for r in table], w.seed)
    m, n, T = J.shape[0], J.shape[1], w.frames
    Jd = torch.from_numpy(J).to(dev)
    Zd = torch.from_numpy(Zin).to(dev)
    thd = torch.from_numpy(theta0).to(dev)
    Vd = torch.from_numpy(np.ascontiguousarray(V)).to(dev)
    Sig = torch.zeros((1, T, n), device=dev)
    res = torch.zeros((1, T), dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    ctx.set_optim(w.lr)
    hd = ctx.handle

    def step(Jp, Zp, thp, Vp, Sp, Rp):
        B.d2ip_load_J(hd, Jp, m, n, 1)
        B.d2ip_set_input(hd, Zp, thp)
        B.d2ip_fit_sequence(hd, Vp, T, None, w.upws_steps, w.first_steps, w.later_steps, Sp, Rp)

    for _ in range(args.warmup):
        step(Jd, Zd, thd, Vd, Sig, res)
        with torch.cuda.stream(stream):
            flush.zero_()
    torch.cuda.synchronize()
    replicas.barrier()
    clocks = ClockSampler(local_rank, _clocks_path(args, rank))
    total_ms = 0.0
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(Jd, Zd, thd, Vd, Sig, res)
        e1.record(stream)
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = replicas.max_over_ranks(total_ms, dev)
    replicas.barrier()
    its = iters_per_step(w)
    value = replicas.job_rate(args.steps * its, total_ms / 1e3, world)
    frames_s = replicas.job_rate(args.steps * T, total_ms / 1e3, world)

    # equal-ERR record of the last step's reconstruction
    S = Sig.cpu().numpy()[0]
    errs = [_err(S[t], truth[t]) for t in range(T) if np.abs(truth[t]).max() > 0]

    # roofline of the dominant kernel class, from CUDA events around every launch
    ctx.set_input(Zd, thd)
    prof = ctx.profile(Vd[0], 10)
    roof = _roofline(prof, args, clk, 10)
    nk_step, nk_eval = ctx.graph_kernels()
    gpu_launches = int(args.steps * (its * nk_step + T * nk_eval))

    # end to end through the C ABI with pinned host buffers
    Jh = torch.from_numpy(J).pin_memory()
    Zh = torch.from_numpy(Zin).pin_memory()
    thh = torch.from_numpy(theta0).pin_memory()
    Vh = torch.from_numpy(np.ascontiguousarray(V)).pin_memory()
    Sh = torch.zeros((1, T, n)).pin_memory()
    Rh = torch.zeros((1, T), dtype=torch.float64).pin_memory()
    step(Jh, Zh, thh, Vh, Sh, Rh)
    e2e_s = 0.0
    e2e_steps = min(args.steps, 2)
    for _ in range(e2e_steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(Jh, Zh, thh, Vh, Sh, Rh)
        e2e_s += time.perf_counter() - t0
    e2e_s = replicas.max_over_ranks(e2e_s, dev)
    h2d = J.nbytes + Zin.nbytes + theta0.nbytes + V.nbytes
    d2h = Sh.numel() * 4 + Rh.numel() * 8
    ctx.close()
    return {
        "value": value, "ms_per_step": total_ms / args.steps, "frames_per_s": frames_s,
        "e2e": {"value": replicas.job_rate(e2e_steps * its, e2e_s, world), "unit": UNIT,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "frames_per_s": replicas.job_rate(e2e_steps * T, e2e_s, world),
                "steps": e2e_steps},
        "roofline": roof, "clocks": clk, "gpu_launches": gpu_launches,
        "err": {"mean": float(np.mean(errs)), "min": float(np.min(errs)),
                "max": float(np.max(errs)), "frames": len(errs)},
        "profile_ms_per_iter": {k: round(v[0] / 10.0, 4) for k, v in prof.items()},
    }


def run_batched(args, rank, world, local_rank):
    """BF16 batched form: all 64 sequences, one context per (grid, rings) group, fitted
    concurrently with d2ip_fit_batched.  Beside it, the plain FP32 single-problem form on a
    sample of the same sequences (one per group), for frames/s at equal ERR."""
    import torch

    from paper_2507_14046_gb300 import binding as B

    w = synth.SEQ_32  # network and schedule of the 20-frame workload
    T = w.frames
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    groups = synth.batch_workload(64, T, seed=1, c_in=w.c_in)
    prec = _prec_code(B, args.precision)
    ctxs, streams, dv = [], [], []
    table = None
    for g in groups:
        st = torch.cuda.Stream(device=dev)
        c = B.Context(g.grid, w.levels, w.widths, w.c_in, prec, len(g.problems),
                      device=local_rank, stream=st.cuda_stream)
        c.set_optim(w.lr)
        table = c.table() if table is None else table
        P = c.P
        th = np.stack([synth.kaiming_theta([tuple(r) for r in table], 1, stream_offset=p * P)
                       for p in g.problems])
        n, m = g.J.shape[1], g.J.shape[0]
        dv.append({"J": torch.from_numpy(g.J).to(dev), "Z": torch.from_numpy(g.Z).to(dev),
                   "th": torch.from_numpy(th).to(dev),
                   "V": torch.from_numpy(np.ascontiguousarray(g.V)).to(dev),
                   "S": torch.zeros((len(g.problems), T, n), device=dev),
                   "R": torch.zeros((len(g.problems), T), dtype=torch.float64, device=dev),
                   "th_np": th, "m": m, "n": n})
        ctxs.append(c)
        streams.append(st)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    its = iters_per_step(w)
    nseq = sum(len(g.problems) for g in groups)

    def step(bufs):
        for c, b in zip(ctxs, bufs):
            B.d2ip_load_J(c.handle, b["J"], b["m"], b["n"], 1)
            B.d2ip_set_input(c.handle, b["Z"], b["th"])
        B.d2ip_fit_batched([c.handle for c in ctxs], [b["V"] for b in bufs], T, None,
                           w.upws_steps, w.first_steps, w.later_steps, [b["S"] for b in bufs],
                           [b["R"] for b in bufs])

    for _ in range(args.warmup):
        step(dv)
        flush.zero_()
    torch.cuda.synchronize()
    replicas.barrier()
    clocks = ClockSampler(local_rank, _clocks_path(args, rank))
    total_ms = 0.0
    for _ in range(args.steps):
        starts = [torch.cuda.Event(enable_timing=True) for _ in streams]
        ends = [torch.cuda.Event(enable_timing=True) for _ in streams]
        for e, st in zip(starts, streams):
            e.record(st)
        step(dv)
        for e, st in zip(ends, streams):
            e.record(st)
        torch.cuda.synchronize()
        total_ms += max(starts[0].elapsed_time(e) for e in ends)
        flush.zero_()
        torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = replicas.max_over_ranks(total_ms, dev)
    value = replicas.job_rate(args.steps * nseq * its, total_ms / 1e3, world)
    frames_s = replicas.job_rate(args.steps * nseq * T, total_ms / 1e3, world)

    # ERR of every sequence of the last step (frames with a zero truth excluded)
    err_b = {}
    for g, b in zip(groups, dv):
        S = b["S"].cpu().numpy()
        for i, p in enumerate(g.problems):
            err_b[p] = [_err(S[i, t], g.truth[i, t]) for t in range(T)
                        if np.abs(g.truth[i, t]).max() > 0]
    # plain FP32 single-problem form on one sequence per group, at equal schedule; and the
    # same sequences in FP32 four times more, from theta0 * (1 + 1e-7 f(index)) with f = sin,
    # -cos, cos, -sin (rounded to FP32): how far the FP32 fit itself moves under a
    # rounding-level change of its start, the floor below which an ERR difference between two
    # precisions means nothing
    plain_s, plain_frames, err_p, err_f = 0.0, 0, {}, {}
    for g, b in zip(groups, dv):
        i, p = 0, g.problems[0]
        st = torch.cuda.Stream(device=dev)
        c1 = B.Context(g.grid, w.levels, w.widths, w.c_in, B.D2IP_FP32, 1, device=local_rank,
                       stream=st.cuda_stream)
        c1.set_optim(w.lr)
        S1 = torch.zeros((1, T, b["n"]), device=dev)
        R1 = torch.zeros((1, T), dtype=torch.float64, device=dev)
        ks = np.arange(b["th_np"].shape[1])
        th_pert = [torch.from_numpy((b["th_np"][i] * (1.0 + 1e-7 * f(ks))).astype(np.float32)
                                    [None]).to(dev)
                   for f in (np.sin, lambda k: -np.cos(k), np.cos, lambda k: -np.sin(k))]

        def one(th):
            B.d2ip_load_J(c1.handle, b["J"], b["m"], b["n"], 1)
            B.d2ip_set_input(c1.handle, b["Z"][i:i + 1], th)
            B.d2ip_fit_sequence(c1.handle, b["V"][i:i + 1], T, None, w.upws_steps,
                                w.first_steps, w.later_steps, S1, R1)

        def frame_errs():
            S = S1.cpu().numpy()[0]
            return [_err(S[t], g.truth[i, t]) for t in range(T)
                    if np.abs(g.truth[i, t]).max() > 0]
        one(b["th"][i:i + 1])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        one(b["th"][i:i + 1])
        e1.record(st)
        torch.cuda.synchronize()
        plain_s += e0.elapsed_time(e1) / 1e3
        plain_frames += T
        err_p[p] = frame_errs()
        err_f[p] = []
        for th in th_pert:
            one(th)
            torch.cuda.synchronize()
            err_f[p].append(frame_errs())
        c1.close()
    sample = sorted(err_p)
    eb = float(np.mean([np.mean(err_b[p]) for p in sample]))
    ep = float(np.mean([np.mean(err_p[p]) for p in sample]))
    # per-frame relative ERR differences against the plain FP32 form, over the sample
    d_bp = np.concatenate([np.abs(np.subtract(err_b[p], err_p[p])) / err_p[p] for p in sample])
    d_fp = [np.concatenate([np.abs(np.subtract(err_f[p][k], err_p[p])) / err_p[p]
                            for p in sample]) for k in range(len(err_f[sample[0]]))]
    floor = float(np.mean(np.concatenate(d_fp)))
    # a mean over six sequences of correlated frames: allow 1.5x for its sampling noise (the
    # four floor samples' means are reported side by side as a measure of it)
    equal_err = bool(np.mean(d_bp) <= max(1e-3, 1.5 * floor))

    # roofline of the dominant kernel class on the largest group
    gi = max(range(len(groups)), key=lambda k: groups[k].J.shape[1] * len(groups[k].problems))
    ctxs[gi].set_input(dv[gi]["Z"], dv[gi]["th"])
    prof = ctxs[gi].profile(dv[gi]["V"][:, 0].contiguous(), 5)
    roof = _roofline(prof, args, clk, 5)
    # kernels launched per step: the captured graphs' kernel nodes (a training iteration, an
    # evaluation) times how often each group replays them, plus two small kernels per frame
    gpu_launches = 0
    for c in ctxs:
        nk_step, nk_eval = c.graph_kernels()
        gpu_launches += its * nk_step + T * (nk_eval + 2) + 2
    gpu_launches *= args.steps

    # end to end through the C ABI from pinned host buffers
    hb = []
    for b in dv:
        hb.append({"J": b["J"].cpu().pin_memory(), "Z": b["Z"].cpu().pin_memory(),
                   "th": b["th"].cpu().pin_memory(), "V": b["V"].cpu().pin_memory(),
                   "S": b["S"].cpu().pin_memory(), "R": b["R"].cpu().pin_memory(),
                   "m": b["m"], "n": b["n"]})
    step(hb)
    e2e_s = 0.0
    e2e_steps = min(args.steps, 2)
    for _ in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(hb)
        e2e_s += time.perf_counter() - t0
    e2e_s = replicas.max_over_ranks(e2e_s, dev)
    h2d = sum(b["J"].numel() * 4 + b["Z"].numel() * 4 + b["th"].numel() * 4 + b["V"].numel() * 4
              for b in hb)
    d2h = sum(b["S"].numel() * 4 + b["R"].numel() * 8 for b in hb)
    for c in ctxs:
        c.close()
    return {
        "value": value, "ms_per_step": total_ms / args.steps, "frames_per_s": frames_s,
        "e2e": {"value": replicas.job_rate(e2e_steps * nseq * its, e2e_s, world), "unit": UNIT,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "frames_per_s": replicas.job_rate(e2e_steps * nseq * T, e2e_s, world),
                "steps": e2e_steps},
        "roofline": roof, "clocks": clk, "gpu_launches": gpu_launches,
        "err": {"mean": float(np.mean([np.mean(v) for v in err_b.values()])),
                "sequences": len(err_b)},
        "plain_fp32": {"frames_per_s": plain_frames / plain_s,
                       "iters_per_s": len(sample) * its / plain_s,
                       "sample": f"{len(sample)} sequences (one per grid/m group), one at a "
                                 "time, FP32 single-problem contexts",
                       "err_mean_sample": ep, "err_mean_batched_same_sequences": eb,
                       "err_rel_diff": abs(eb - ep) / ep,
                       "frame_err_rel_diff": {"mean": float(np.mean(d_bp)),
                                              "max": float(np.max(d_bp)),
                                              "frames": int(d_bp.size)},
                       "fp32_floor": {"mean": floor,
                                      "sample_means": [float(np.mean(d)) for d in d_fp],
                                      "max": float(max(np.max(d) for d in d_fp)),
                                      "how": "the same FP32 fits from theta0 * (1 + 1e-7 "
                                             "f(index)), f = sin, -cos, cos, -sin; per-frame "
                                             "relative ERR change"},
                       "equal_err": equal_err,
                       "equal_err_rule": "mean per-frame |ERR - ERR_fp32| / ERR_fp32 of the "
                                         "batched form <= max(1e-3, 1.5 x mean FP32 floor)",
                       "speedup_frames_per_s": frames_s / (plain_frames / plain_s),
                       "speedup_label": "at equal ERR" if equal_err else "NOT at equal ERR"},
        "groups": [{"grid": list(g.grid), "m": g.J.shape[0], "problems": len(g.problems)}
                   for g in groups],
        "profile_ms_per_iter": {k: round(v[0] / 5.0, 4) for k, v in prof.items()},
    }


def _source_digest(files=None):
    """sha1 over the named CUDA sources (default: every .cu/.cuh of the library)."""
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2507_14046_gb300", "csrc")
    names = sorted(files) if files else sorted(f for f in os.listdir(csrc)
                                               if f.endswith((".cu", ".cuh")))
    for f in names:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()


# per (workload, network, precision): the ncu traffic summary and the sources that hold the
# roofline class's kernels and their launch sequence (a change there voids the figure)
TRAFFIC_FILES = {
    ("batch64", "resunet", "bf16x3"): (
        "roofline_traffic_batch64_bf16x3.txt",
        ("common.cuh", "conv_bf16.cu", "conv_bf16.cuh", "conv_f32.cu", "pointwise.cu",
         "runtime.cu", "tc_prims.cuh")),
    ("seq32", "fastres", "fp32"): (
        "roofline_traffic_seq32_fastres_fp32.txt",
        ("common.cuh", "conv_f32.cu", "fastres.cu", "fastres.cuh", "fastres_ops.cu")),
}


def _traffic(cls, args):
    """DRAM bytes per launch of the class from the committed ncu summary, when it was taken on
    the kernels as they are now (same CUDA sources) and on this workload; else None."""
    entry = TRAFFIC_FILES.get((args.workload, args.net, args.precision))
    if entry is None:
        return None
    name, sources = entry
    path = os.path.join(ROOT, "profiles", name)
    try:
        with open(path) as fh:
            t = json.load(fh)
    except (OSError, ValueError):
        return None
    if t.get("source_sha1") != _source_digest(sources):
        return None
    v = t.get("bytes_per_launch", {}).get(cls)
    return float(v) if v is not None else None


def _roofline(prof, args, clk, iters):
    peaks, kind = _peaks()
    dom = max(prof, key=lambda k: prof[k][0])
    ms, work, cnt = prof[dom]
    avg_ms = ms / cnt
    per_launch = work / cnt
    if dom.startswith("conv") and args.precision.startswith("bf16"):
        peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        roof = {"bound": "tensor", "achieved": per_launch / (avg_ms * 1e-3) / 1e12,
                "peak": peak, "unit": "TFLOP/s", "traffic": _traffic(dom, args),
                "peak_source": f"{kind} bf16_tflops_sustained (kernel timed inside a long step); "
                               "the class also holds its BF16 staging, the partial-sum "
                               "reductions and the 1x1x1 single-channel last layer (FP32)"}
    elif dom.startswith("conv"):
        mhz = (clk or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
        peak = SMS * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": per_launch / (avg_ms * 1e-3) / 1e12, "peak": peak,
                "unit": "TFLOP/s", "traffic": _traffic(dom, args),
                "peak_source": f"FP32 FFMA: {SMS} SMs x {FP32_LANES_PER_SM} lanes x 2 x "
                               f"{mhz:.0f} MHz (median sampled SM clock)"}
    else:
        peak = peaks["hbm_gbs"]
        roof = {"bound": "hbm", "achieved": per_launch / (avg_ms * 1e-3) / 1e9, "peak": peak,
                "unit": "GB/s", "traffic": _traffic(dom, args), "peak_source": f"{kind} hbm_gbs"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    if args.precision == "bf16x3" and dom.startswith("conv"):
        # the split products issue three BF16 MMAs per multiply-add of the convolution
        roof["issued_mma_flops_factor"] = 3
        roof["issued_frac"] = 3 * roof["frac"]
    roof["kernel"] = dom
    roof["avg_launch_us"] = avg_ms * 1e3
    roof["work_per_launch"] = per_launch
    roof["share_of_traced_time"] = ms / sum(v[0] for v in prof.values())
    return roof


def run_probe(args):
    """The largest group of the batched workload alone (48x48x24, 13 problems, BF16): W
    training iterations, then K traced iterations; prints the per-class profile.  This is
    the case the bench's roofline is taken on, small enough for ncu captures."""
    import torch

    from paper_2507_14046_gb300 import binding as B

    w = synth.SEQ_32
    if args.net == "fastres":  # the variant on the 20-frame sequence's first frame, FP32
        J, truth, V, Zin = synth.make_problem(w)
        c = B.Context(w.grid, w.levels, w.widths, w.c_in, B.D2IP_FP32, 1, net="fastres")
        th = synth.kaiming_theta([tuple(r) for r in c.table()], w.seed)
        c.load_J(J)
        c.set_input(Zin, th)
        c.set_optim(w.lr)
        c.run_steps(V[:1], args.warmup)
        torch.cuda.synchronize()
        prof = c.profile(V[0], args.probe)
        nk_step, nk_eval = c.graph_kernels()
        print(json.dumps({"probe": f"FastResUNet variant, grid {list(w.grid)}, FP32",
                          "iters": args.probe, "step_graph_kernels": nk_step,
                          "profile_ms_per_iter": {k: round(v[0] / args.probe, 4)
                                                  for k, v in prof.items()},
                          "launches_per_iter": {k: v[2] / args.probe for k, v in prof.items()}}))
        c.close()
        return
    groups = synth.batch_workload(64, w.frames, seed=1, c_in=w.c_in)
    g = max(groups, key=lambda q: q.J.shape[1] * len(q.problems))
    nprob = min(args.probe_problems or len(g.problems), len(g.problems))
    plan = None
    if args.tile_plan_in:  # tilings saved by an earlier run (no timing sweep in this one)
        with open(args.tile_plan_in) as f:
            plan = json.load(f)["rows"]
    c = B.Context(g.grid, w.levels, w.widths, w.c_in, _prec_code(B, args.precision or "bf16"),
                  nprob, tile_plan=plan)
    table = c.table()
    th = np.stack([synth.kaiming_theta([tuple(r) for r in table], 1, stream_offset=p * c.P)
                   for p in g.problems[:nprob]])
    c.load_J(g.J)
    c.set_input(np.ascontiguousarray(g.Z[:nprob]), th)
    c.set_optim(w.lr)
    v0 = np.ascontiguousarray(g.V[:nprob, 0])
    c.run_steps(v0, args.warmup)
    torch.cuda.synchronize()
    prof = c.profile(v0, args.probe)
    nk_step, nk_eval = c.graph_kernels()
    if args.tile_plan_out:
        rows, us = c.tile_plan()
        with open(args.tile_plan_out, "w") as f:
            json.dump({"rows": rows.tolist(), "us": us.tolist()}, f)
    print(json.dumps({"probe": f"grid {list(g.grid)}, m {g.J.shape[0]}, {nprob} problems, "
                               f"{(args.precision or 'bf16').upper()}",
                      "iters": args.probe, "step_graph_kernels": nk_step,
                      "profile_ms_per_iter": {k: round(v[0] / args.probe, 4)
                                              for k, v in prof.items()},
                      "launches_per_iter": {k: v[2] / args.probe for k, v in prof.items()}}))
    c.close()


def run_study(args):
    """Convergence ablation (plain DIP, + 4D-TV, UPWS, full D²IP) on the second frame of a
    sequence workload; prints one JSON summary line, and the curves to --study-out (.npz)."""
    import torch

    from paper_2507_14046_gb300 import study

    w = WORKLOADS["seq32" if args.workload == "batch64" else args.workload]
    torch.cuda.set_device(0)
    t0 = time.time()
    res = study.run(w, iters=args.study, precision=args.precision or "fp32")
    secs = time.time() - t0
    summ = study.summarise(res)
    if args.study_out:
        np.savez_compressed(args.study_out, err_iters=res["err_iters"],
                            **{f"loss_{a}": res["loss"][a] for a in study.ARMS},
                            **{f"err_{a}": res["err"][a] for a in study.ARMS})
    print(json.dumps({"study": "acceleration ablation, frame 2", "workload": w.name,
                      "schedule": res["schedule"], "seconds": round(secs, 1), **summ}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch64", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=None, choices=list(PRECISIONS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-leg", default=None)
    ap.add_argument("--oracle-iters", type=int, default=5)
    ap.add_argument("--probe", type=int, default=0,
                    help="trace this many iterations of the largest batched group and exit")
    ap.add_argument("--probe-problems", type=int, default=0)
    ap.add_argument("--tile-plan-out", default="",
                    help="probe: write the tilings in use (JSON) to this file")
    ap.add_argument("--tile-plan-in", default="",
                    help="probe: apply the tilings of this file instead of timing them "
                         "(repeatable runs, e.g. under a profiler)")
    ap.add_argument("--study", type=int, default=0,
                    help="run the convergence ablation for this many iterations and exit")
    ap.add_argument("--study-out", default=None)
    ap.add_argument("--clocks-dir", default=None,
                    help="directory for the raw nvidia-smi samples of the timed region")
    ap.add_argument("--net", default="resunet", choices=["resunet", "fastres"],
                    help="network: the residual U-Net, or the paper-form FastResUNet variant "
                         "(FP32, single-sequence workloads)")
    args = ap.parse_args()
    if args.study:
        run_study(args)
        return
    if args.probe:
        run_probe(args)
        return

    if args.oracle_leg:
        print(json.dumps(oracle_leg(args.oracle_leg, args.oracle_iters, args.net)))
        return
    if args.net == "fastres":
        if args.workload == "batch64":
            args.workload = "seq32"
        if args.precision not in (None, "fp32"):
            ap.error("the FastResUNet variant runs in FP32")
    if args.precision is None:
        # the batched workload's headline precision is the one at equal ERR with the plain
        # FP32 form (plain BF16 differs from it by twice the FP32 floor)
        args.precision = "bf16x3" if args.workload == "batch64" else "fp32"

    rank, world, local_rank = replicas.world()
    w = WORKLOADS[args.workload]
    its = iters_per_step(w)
    config = {"workload": w.name + ", " + args.precision.upper(),
              "grid": list(w.grid), "m": w.m, "levels": w.levels, "widths": list(w.widths),
              "frames": w.frames, "schedule": [w.upws_steps, w.first_steps, w.later_steps],
              "lr": w.lr, "iters_per_step": its, "precision": args.precision,
              "l2": "512 MB buffer written between timed steps (working set < L2)",
              "parallelism": f"replicas x{args.gpus}"}
    if args.net == "fastres":
        config["workload"] = (w.name.replace("L3(16,32,64)", "FastResUNet(16,32,64)")
                              + ", FP32 (paper-form network variant)")
        config["net"] = "fastres"

    if args.workload == "batch64":
        config["workload"] = ("64 independent 20-frame sequences (grids 16x16x8 / 32x32x16 / "
                              f"48x48x24, m 208 / 416), L3(16,32,64), {args.precision.upper()} "
                              "batched")
        config["grid"] = "mixed"
        config["m"] = "mixed"
        config["iters_per_step"] = 64 * its

    if args.impl == "reference":
        if rank != 0:
            return
        if args.workload == "batch64":  # the same groups as the batched arm reports
            cnt = {}
            for g, r in synth.batch_problem_shapes(64, 1):
                cnt[(g, r)] = cnt.get((g, r), 0) + 1
            config["groups"] = [{"grid": list(g), "m": 208 * r, "problems": cnt[(g, r)]}
                                for g in synth.BATCH_GRIDS for r in synth.BATCH_RINGS
                                if (g, r) in cnt]
        per = oracle_iters_for(args.workload)
        per = max(1, per // 4)
        for _ in range(args.warmup):
            oracle_leg(args.workload, 1, args.net)
        tot_it, tot_s = 0, 0.0
        for _ in range(args.steps):
            r = oracle_leg(args.workload, per, args.net)
            tot_it += r["iters"]
            tot_s += r["seconds"]
        v = tot_it / tot_s
        cores = os.cpu_count() or 1
        sample = (f"{per} FP64 oracle DIP iterations per step (first frame of the workload, "
                  f"from the Kaiming weights) on {cores} host cores")
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample}}))
        return

    replicas.init()
    if args.workload == "batch64":
        out = run_batched(args, rank, world, local_rank)
        config["groups"] = out.pop("groups")
    else:
        out = run_gpu(args, rank, world, local_rank)
    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        r = run_oracle_subprocess(args.workload, oracle_iters_for(args.workload), args.net)
        cpu = {"value": r["iters_per_s"], "unit": UNIT, "cores": r["cores"], "kind": "oracle",
               "sample": f"{r['iters']} FP64 oracle DIP iterations (first frame of the same "
                         f"workload{', every grid of the mix, weighted by its sequences' if args.workload == 'batch64' else ''}"
                         f") in {r['seconds']:.1f} s, NumPy/BLAS on {r['cores']} host threads"}
        r1 = run_oracle_subprocess(args.workload, max(1, oracle_iters_for(args.workload) // 4),
                                   args.net, threads=1)
        cpu["single_core"] = {"value": r1["iters_per_s"], "unit": UNIT, "cores": 1,
                              "sample": f"{r1['iters']} iterations in {r1['seconds']:.1f} s, "
                                        "one host thread"}
    line = {"metric": METRIC, "value": out["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": out["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"bf16": "bf16", "bf16x3": "bf16x3 (hi/lo BF16 pairs, FP32 "
                      "accumulation)", "fp32": "f32"}[args.precision],
            "data": "synthetic", "config": config, "frames_per_s": out["frames_per_s"],
            "e2e": out["e2e"], "roofline": out["roofline"], "cpu_baseline": cpu,
            "clocks": out["clocks"], "gpu_launches": out["gpu_launches"], "err": out["err"],
            "profile_ms_per_iter": out["profile_ms_per_iter"]}
    if "plain_fp32" in out:
        line["plain_fp32"] = out["plain_fp32"]
    print(json.dumps(line))


if __name__ == "__main__":
    main()
