"""Host-side pieces of the benchmark that decide what its JSON line reports,
checked without a GPU: the roofline entry and its measured-traffic key, the
accuracy gate's use of the stored whole oracle solve of the 3D benchmark
instance, and the calibration record of the oracle's timing model.

The stored oracle solve (tests/golden/c2_ipn_oracle.npz, written by a
committed script that calls only the oracle) is also pinned to something
other than itself: its u must reach the manufactured solution to the
discretisation's accuracy (relative L2 about 3.4e-6 on the evaluation grid,
Sec. 6.2's level for this setting), and it must hold the iteration counts
the file claims."""
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
import rfm_workloads as W  # noqa: E402


def test_roofline_entry_and_traffic_key():
    r = bench.roofline(["oz_gemm"], 1000.0, 10, 1e15, ("c2", 2))
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(1000.0)  # 1e15 flop in 1 s
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["launches"] == 10 and r["avg_launch_ms"] == pytest.approx(100.0)
    assert r["traffic"] == bench.MEASURED_TRAFFIC.get(("c2", 2, "oz_gemm"))
    # another workload or precision has no measured traffic
    assert bench.roofline(["oz_gemm"], 1000.0, 10, 1e15, ("c2", 1))["traffic"] is None
    assert bench.roofline(["oz_gemm"], 1000.0, 10, 1e15, ("c4", 2))["traffic"] is None
    # the FP64 families report against the derived FP64 ALU peak
    f = bench.roofline(["qr_update"], 1000.0, 4, 1e12, ("c2", 0))
    assert f["bound"] == "alu" and f["peak"] == pytest.approx(bench.FP64_ALU_PEAK_TFLOPS)


def test_gate_uses_the_stored_oracle_solve():
    wl = bench.workload("c2")
    ref = bench.stored_oracle_solve(None, wl)
    assert ref is not None, "tests/golden/c2_ipn_oracle.npz is committed"
    it, ls, src = bench.oracle_counts(wl)
    assert (it, ls, src) == (int(ref["outer_iters"]), int(np.sum(ref["lsqr_iters"])), "the stored oracle solve")
    assert (int(ref["outer_iters"]), int(ref["n_jac"])) == (4, 4) and int(np.sum(ref["lsqr_iters"])) == 137
    assert len(ref["lsqr_iters"]) == int(ref["outer_iters"])
    # AMIPN runs have no stored solve and fall back to the GPU's counts
    assert bench.stored_oracle_solve(None, bench.workload("c2", solver="amipn")) is None
    assert bench.oracle_counts(bench.workload("c2", solver="amipn"),
                               {"outer_iters": 5, "lsqr_iters_total": 99}) == (5, 99, "the GPU solve")


def test_calibration_record():
    cal = bench.calibration(bench.workload("c2"))
    assert cal is not None
    ref = np.load(os.path.join(bench.GOLDEN, "c2_ipn_oracle.npz"))
    assert cal["measured_wall_s"] == pytest.approx(float(ref["wall_s"]))
    assert (cal["outer_iters"], cal["lsqr_iters"]) == (4, 137)
    assert cal["projected_s"] > 0 and 0.05 < cal["measured_wall_s"] / cal["projected_s"] < 20
    assert cal["machine"] == str(ref["machine"]) and cal["cores"] == int(ref["cores"])
    assert bench.calibration(bench.workload("c1")) is None


def test_stored_c2_solution_reaches_the_manufactured_solution():
    from oracle.problem import Problem
    desc = W.config_c2()
    ref = np.load(os.path.join(bench.GOLDEN, "c2_ipn_oracle.npz"))
    X = W.eval_grid(desc)
    ue = Problem(desc).exact(X)
    u = np.asarray(ref["u"]).reshape(ue.shape)
    rel = np.linalg.norm(u - ue) / np.linalg.norm(ue)
    assert 1e-7 < rel < 1e-5, rel
    assert np.isfinite(float(ref["final_resid"])) and float(ref["final_resid"]) > 0
    assert json.loads(json.dumps(float(ref["wall_s"]))) > 0
