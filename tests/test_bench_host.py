"""Host logic of bench.py: the roofline arithmetic, the traffic lookup keyed to the sources of
a kernel class, and the step sizes of the workloads (no GPU)."""
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


class Args:
    def __init__(self, workload="batch64", net="resunet", precision="bf16"):
        self.workload, self.net, self.precision = workload, net, precision


def test_iterations_per_step(bench):
    from paper_2507_14046_gb300 import synth
    assert bench.iters_per_step(synth.SEQ_32) == 300 + 50 + 19 * 50
    assert bench.iters_per_step(synth.SINGLE_16) == 200
    assert bench.iters_per_step(synth.SEQ_64) == 400 + 40 + 99 * 40


def test_roofline_picks_the_dominant_class_and_divides_work_by_time(bench):
    # class: (ms total, work total, launches)
    prof = {"conv_fwd": (1.0, 2e12, 10), "conv_wgrad": (4.0, 4e12, 8), "ln_fwd": (0.5, 1e9, 5)}
    r = bench._roofline(prof, Args(), {"sm_mhz": 2070.0}, 1)
    assert r["kernel"] == "conv_wgrad" and r["bound"] == "tensor"
    per = 4e12 / 8
    dur = 4.0 / 8 * 1e-3
    assert r["achieved"] == pytest.approx(per / dur / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["share_of_traced_time"] == pytest.approx(4.0 / 5.5)
    fp32 = bench._roofline(prof, Args(precision="fp32"), {"sm_mhz": 2000.0}, 1)
    assert fp32["bound"] == "alu"
    assert fp32["peak"] == pytest.approx(152 * 128 * 2 * 2000e6 / 1e12)
    mem = bench._roofline({"ln_bwd": (1.0, 5e9, 2)}, Args(), None, 1)
    assert mem["bound"] == "hbm" and mem["unit"] == "GB/s"
    assert mem["achieved"] == pytest.approx(2.5e9 / 0.5e-3 / 1e9)


def test_traffic_only_for_a_matching_capture(bench, monkeypatch):
    import json
    key = ("seq32", "fastres", "fp32")
    name, sources = bench.TRAFFIC_FILES[key]
    with open(os.path.join(ROOT, "profiles", name)) as fh:
        stored = json.load(fh)
    cls = next(iter(stored["bytes_per_launch"]))
    # no capture for this workload at all
    assert bench._traffic(cls, Args("seq32", "resunet", "fp32")) is None
    # the sources match the capture: its figure; a class without a figure: None
    monkeypatch.setattr(bench, "_source_digest", lambda files=None: stored["source_sha1"])
    assert bench._traffic(cls, Args(*key)) == pytest.approx(stored["bytes_per_launch"][cls])
    assert bench._traffic("ln_fwd", Args(*key)) is None
    # a kernel source changed since the capture: no figure
    monkeypatch.setattr(bench, "_source_digest", lambda files=None: "0" * 40)
    assert bench._traffic(cls, Args(*key)) is None


def test_source_digest_depends_on_the_named_files(bench):
    a = bench._source_digest(["conv_f32.cu"])
    assert a == bench._source_digest(["conv_f32.cu"])
    assert a != bench._source_digest(["conv_f32.cu", "common.cuh"])
