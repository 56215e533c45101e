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


def test_unit_weight_flops_below_weighted(bench):
    steps, rej = np.array([2000, 2100]), np.array([10, 12])
    fw, pw = bench.algorithmic_flops(steps, rej)
    fu, pu = bench.algorithmic_flops(steps, rej, bench.UNIT_WEIGHTS)
    with open(bench.OPCOUNT_FILE) as fh:
        oc = json.load(fh)["counts"]
    # the weighted count adds (34 - 1) per exp and (62 - 1) per log in every part
    d_att = 33 * (2 * oc["rates"]["exp"]) + 61 * (2 * oc["rates"]["log"])
    d_acc = 33 * oc["jacobian"]["exp"] + 61 * oc["jacobian"]["log"]
    assert pw["per_attempt"] - pu["per_attempt"] == d_att
    assert pw["per_accepted"] - pu["per_accepted"] == d_acc
    assert fu < fw


def test_budget_guard(bench):
    b = bench.Budget(100.0, t0=0.0)
    assert b.may_continue(0, 5, 0.0, 1000.0, now=99.0)  # the first timed step always runs
    assert b.may_continue(1, 5, 10.0, 20.0, now=60.0)  # 60 + 10 + 20 <= 100
    assert not b.may_continue(1, 5, 10.0, 31.0, now=60.0)
    assert not b.may_continue(5, 5, 0.0, 0.0, now=0.0)  # all requested steps done


def test_budget_projection(bench):
    """The driver's run: 20 steps of 83.3 s after ~25 s of start-up and CPU legs fit in 1740 s
    with the 20 s reserve; at 85.2 s per step only 19 do."""
    b = bench.Budget(1740.0, t0=0.0)
    pj = b.projection(1, 20, 83.3, 20.0, now=25.0 + 83.3)
    assert pj["steps_that_fit"] == 20 and pj["projected_end_s"] <= 1740.0
    assert b.projection(1, 20, 85.2, 20.0, now=25.0 + 85.2)["steps_that_fit"] == 19
    # the projection agrees with the loop's own test step by step
    done, now = 1, 25.0 + 85.2
    while b.may_continue(done, 20, 85.2, 20.0, now=now):
        done += 1
        now += 85.2
    assert done == 19
    assert bench.parse_args([]).budget_s == 1740.0


def test_sample_sizes(bench):
    n_all, n_one = bench.sample_sizes(36.0, 16, 15.0, 65536)
    assert n_all % 16 == 0 and 16 <= n_all <= 65536 and abs(n_all / 36.0 - 15.0) < 1.0
    assert 2 <= n_one <= 64
    assert bench.sample_sizes(0.01, 16, 15.0, 65536) == (16, 2)
    assert bench.sample_sizes(1e9, 16, 15.0, 1000)[0] <= 1000


def _fake_w():
    class M:
        K, R = 53, 325
    n = 64
    return {"name": "fake", "mech": M(), "T": np.full(n, 1000.0), "Y": np.full((53, n), 1.0 / 53), "dt": 1e-5,
            "p_Pa": 40 * 101325.0, "rtol": 1e-6, "atol": 1e-10}


def test_forward_line_assembly(bench):
    """The line of the forward workloads from fake measurements (no GPU): every key the contract
    asks for, the budget note when the loop stopped early, JSON-serialisable."""
    args = bench.parse_args(["--steps", "20", "--warmup", "5"])
    w = _fake_w()
    n = w["T"].shape[0]
    steps_np, rej_np = np.full(n, 2000, np.int32), np.full(n, 10, np.int32)
    peak = {"tflops": 1.25856, "measured_tflops": 1.05, "source": "derived"}
    common = dict(w=w, world=1, args=args, kern_ms=2000.0, e2e={"value": 1.0}, clk={"sm_mhz": 2070.0},
                  st_np=np.zeros(n, np.int32), steps_np=steps_np, rej_np=rej_np, peak=peak,
                  opts_info={"refine_sweeps": None, "warps_per_cell": 2, "cells_per_cta": 4}, dtype="f64",
                  rosen=True, traffic_ok=True, lowp_stats={}, warm_cells=608)
    line = bench.forward_line(steps_done=20, budget_stopped=False, **common)
    json.dumps(line)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "e2e", "gpu_launches", "roofline", "clocks"):
        assert key in line
    assert line["steps"] == 20 and "steps_requested" not in line
    assert abs(line["value"] - n * 20 / 2.0) < 1e-9
    rf = line["roofline"]
    assert rf["bound"] == "alu" and rf["frac"] < rf["frac_weighted"]
    assert abs(rf["frac"] - rf["achieved"] / peak["tflops"]) < 1e-15
    short = bench.forward_line(steps_done=7, budget_stopped=True, **common)
    assert short["steps"] == 7 and short["steps_requested"] == 20 and "budget" in short["budget_stop"]
    assert short["gpu_launches"] == 7


def test_adjoint_line_assembly(bench):
    args = bench.parse_args(["--workload", "adjoint", "--steps", "2", "--warmup", "3"])
    w = _fake_w()
    n = 64
    line = bench.adjoint_line(w=w, world=1, args=args, n=n, K=53, R=325, N=53, cap=100, fwd=1000.0, bwd=4000.0,
                              tot=5100.0, clk={}, ns=np.full(n, 50, np.int32), st=np.zeros(n, np.int32),
                              peak_bytes=123, warm=16, h2d=10, d2h=20)
    json.dumps(line)
    assert line["backward_over_forward"] == 4.0 and line["checkpoint"]["bytes_used"] == 50 * n * 54 * 8
    assert line["gpu_launches"] == 8
