"""The benchmark's host-side arithmetic (CPU only): the algorithmic FLOP count behind
`roofline.achieved`, the derived FP64 peak behind `roofline.peak`, and the clock sampler's
reading of nvidia-smi lines (median SM clock, the throttle reasons that reject a run)."""
import importlib.util
import json
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_algorithmic_flops_per_attempt_and_step(bench):
    with open(bench.OPCOUNT_FILE) as fh:
        oc = json.load(fh)
    w = bench.FLOP_WEIGHTS
    per = {k: sum(w[o] * v[o] for o in w) for k, v in oc["counts"].items()}
    N = oc["N"]
    flops, info = bench.algorithmic_flops(np.array([0]), np.array([0]))
    assert flops == 0
    # one attempt: W (N^2 + N), the LU, 5 solves, 2 rate evaluations and ~30 N vector work; one
    # accepted step adds a Jacobian with its rate evaluation
    assert info["per_attempt"] == N * N + N + per["lu"] + 5 * per["solve"] + 2 * per["rates"] + 30 * N
    assert info["per_accepted"] == per["jacobian"]
    # the figures quoted with the headline (53 species)
    assert (info["per_attempt"], info["per_accepted"]) == (229703, 148432)
    steps, rej = np.array([100, 250, 3]), np.array([2, 0, 1])
    flops, _ = bench.algorithmic_flops(steps, rej)
    assert flops == info["per_attempt"] * (steps.sum() + rej.sum()) + info["per_accepted"] * steps.sum()


def test_derived_fp64_peak(bench):
    # 2 FP64 FMA lanes per clock per SM x 152 SMs x 2.07 GHz x 2 flop = 1.259 TFLOP/s
    peak = bench.FP64_LANES_PER_SM_CLK * bench.N_SMS * bench.SM_MAX_CLOCK_GHZ * 2.0 / 1e3
    assert abs(peak - 1.25856) < 1e-12


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_sampler_reads_nvidia_smi_lines(bench):
    s = bench.ClockSampler(0)
    s.proc = _Done()
    s.lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2062, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 950.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    out = s.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    s2 = bench.ClockSampler(0)
    s2.proc = _Done()
    s2.lines = ["0, 1500, 2070, 1400.0, 0x8, Not Active, Active, Not Active, Not Active"]
    assert s2.stop()["reasons"] == ["hw_thermal_slowdown"]
    s3 = bench.ClockSampler(0)
    assert s3.stop()["reasons"] == ["nvidia-smi unavailable"]
