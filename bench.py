"""Benchmark: Newton solves/s of the RFM IPN solver on GB300 (one JSON line).

Workloads (seeded synthetic PDE instances; the paper uses no datasets):
  c2  3D -Lap u + u^3 = f, u* = prod sin(pi x), 4x4x4 subdomains, M=512
      (n = 32,768), 12^3 interior points and 6x6 per face (m = 124,416),
      Gaussian sketch with 65,536 rows, IPN.
  c1  2D analogue: 2x2 subdomains, M=100, 20x20 points, count sketch gamma=3.

A step is one complete IPN solve from u_0 = 0 (assembly, sketch, QR, LSQR,
line search, stopping test) of one instance already described on the device.
`value` = solves/s over the timed steps (CUDA events on the solver stream,
L2 flushed with a 512 MiB write between steps, outside the events).
`e2e` = the same through the public API from host memory: problem creation,
H2D of the initial guess from pinned memory, the solve, D2H of the solution.
Multi-GPU (torchrun): independent replicas, one instance per rank, no
collective on the data path; value = all ranks' solves / max rank time.

--impl reference times the CPU oracle (oracle/) on the same workload on the
host cores, rank 0 only.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import rfm_workloads as W  # noqa: E402

METRIC = "Newton solves/s at rel-L2<=1e-6 vs FP64 oracle (IPN)"
FP64_ALU_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12  # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz


PRECISION_NAMES = {0: "fp64", 1: "fp64 + tensor-core sketch", 2: "fp64 + tensor-core sketch and QR update"}


def workload(name, precision=None, solver=None):
    if name == "c1":
        p = 0 if precision is None else precision
        wl = dict(desc=W.config_c1(), opts=W.solve_opts(precision=p), solver=solver or "ipn",
                  label="c1: 2D -Lap u+u^3, 2x2 subdomains, M=100, n=400, m=1920, count sketch s=1200")
    elif name == "c2":
        p = 2 if precision is None else precision
        wl = dict(desc=W.config_c2(), opts=W.opts_c2(precision=p), solver=solver or "ipn",
                  label="c2: 3D -Lap u+u^3, 4x4x4 subdomains, M=512, n=32768, m=124416, Gaussian sketch s=65536")
    else:
        raise SystemExit(f"unknown workload {name}")
    wl["precision"] = wl["opts"]["precision"]
    return wl


# ------------------------------------------------------------------ clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                if out.returncode == 0 and out.stdout.strip():
                    self.samples.append([x.strip() for x in out.stdout.strip().split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ------------------------------------------------------------------ our arm
def problem_sizes(gp):
    return dict(m=gp.m, n=gp.n, W=gp.W, m_iface=gp.m_iface, nnz=gp.m * gp.W + gp.m_iface * gp.W)


def family_model(fam, sz, s, launches, nj):
    """(bound, total algorithmic units, unit) for the family over the measured
    launches.  Units per launch follow the hot-path cost model:
      qr_vta+qr_update  FP64 flops 2 n^2 (s - n/3) per factorisation
      sketch_gemm       FP64 flops 2 s nnz(J) per Jacobian
      trsv              bytes 8 n(n+1)/2 + 16 n per solve (R read once)
      jmv / jtmv        bytes 8 (nnz + m + n) per product
      assemble          bytes 8 (nnz + 2m) written per assembly"""
    n, m, nnz = sz["n"], sz["m"], sz["nnz"]
    if fam in ("qr_update", "qr_vta"):
        return "alu", nj * 2.0 * n * n * (s - n / 3.0) / 2.0, "flop"
    if fam == "sketch_gemm":
        return "alu", nj * 2.0 * s * nnz, "flop"
    if fam == "trsv":
        return "hbm", launches * (8.0 * n * (n + 1) / 2 + 16.0 * n), "byte"
    if fam in ("jmv", "jtmv"):
        return "hbm", launches * 8.0 * (nnz + m + n), "byte"
    if fam == "assemble":
        return "hbm", launches * 8.0 * (nnz + 2 * m), "byte"
    return "hbm", None, "byte"


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2510_04170_gb300 import build as _build
    from paper_2510_04170_gb300 import rfm

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    _build.build()
    lib = rfm.load()
    lib.rfm_profile_enable.argtypes = [rfm.ctypes.c_int]
    lib.rfm_launch_count.restype = rfm.ctypes.c_int64
    lib.rfm_profile_read.argtypes = [rfm.ctypes.c_int, rfm.ctypes.POINTER(rfm.ctypes.c_double),
                                     rfm.ctypes.POINTER(rfm.ctypes.c_int64)]
    lib.rfm_profile_name.restype = rfm.ctypes.c_char_p
    wl = workload(args.workload, args.precision, args.solver)
    desc, opts = wl["desc"], wl["opts"]
    stream = torch.cuda.Stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        gp = rfm.Problem(desc, stream=stream)
    solve = getattr(gp, f"rfm_{wl['solver']}_solve")
    sz = problem_sizes(gp)

    def one(prof_mask=0):
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            c, info = solve(opts)
            b.record(stream)
        b.synchronize()
        return a.elapsed_time(b), c, info

    nfam = lib.rfm_profile_count()
    names = [lib.rfm_profile_name(i).decode() for i in range(nfam)]
    # warm-up; the last warm-up step is profiled per family to pick the dominant kernel
    info = None
    for wi in range(args.warmup):
        if wi == args.warmup - 1:
            lib.rfm_profile_enable((1 << nfam) - 1)
        _, c, info = one()
    fam_ms = {}
    fam_cnt = {}
    for i in range(nfam):
        ms, cnt = rfm.ctypes.c_double(), rfm.ctypes.c_int64()
        lib.rfm_profile_read(i, rfm.ctypes.byref(ms), rfm.ctypes.byref(cnt))
        fam_ms[names[i]] = ms.value
        fam_cnt[names[i]] = cnt.value
    lib.rfm_profile_enable(0)
    dom = max(fam_ms, key=lambda k: fam_ms[k]) if any(fam_ms.values()) else "qr_update"
    # the QR trailing update is timed as one family pair
    dom_fams = ["qr_vta", "qr_update"] if dom in ("qr_vta", "qr_update") else [dom]
    mask = sum(1 << names.index(f) for f in dom_fams)

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    lib.rfm_profile_enable(mask)
    l0 = lib.rfm_launch_count()
    times = []
    with ClockSampler(local_rank) as clk:
        for _ in range(args.steps):
            ms, c, info = one()
            times.append(ms)
    launches = lib.rfm_launch_count() - l0
    torch.cuda.synchronize()
    dom_ms, dom_cnt = 0.0, 0
    for f in dom_fams:
        ms, cnt = rfm.ctypes.c_double(), rfm.ctypes.c_int64()
        lib.rfm_profile_read(names.index(f), rfm.ctypes.byref(ms), rfm.ctypes.byref(cnt))
        dom_ms += ms.value
        dom_cnt += cnt.value
    lib.rfm_profile_enable(0)
    total_s = sum(times) / 1e3
    t = torch.tensor([total_s], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
    max_s = float(t.item())

    # accuracy of the last solve
    X = W.eval_grid(desc)
    u = gp.rfm_eval(c, torch.as_tensor(X, device="cuda")).cpu().numpy()
    from oracle.problem import Problem as OProblem  # exact solution formula only
    ue = OProblem(desc).exact(X)
    rel_exact = float(np.linalg.norm(u - ue) / np.linalg.norm(ue))

    # end to end through the public API from host memory
    e2e_times = []
    c0_host = torch.zeros(gp.n, dtype=torch.float64).pin_memory()
    out_host = torch.empty(gp.n, dtype=torch.float64).pin_memory()
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            g2 = rfm.Problem(desc, stream=stream)
            c0 = torch.empty(g2.n, dtype=torch.float64, device="cuda")
            c0.copy_(c0_host, non_blocking=True)
            c2, inf2 = getattr(g2, f"rfm_{wl['solver']}_solve")(opts, c0)
            out_host.copy_(c2, non_blocking=True)
        stream.synchronize()
        g2.close()
        e2e_times.append(time.perf_counter() - t0)
    e2e_value = world / statistics.median(e2e_times) if e2e_times else None

    steps_per_rank = args.steps
    value = world * steps_per_rank / max_s
    nj = info["n_jac"]
    s_rows = opts.get("sketch_rows") or int(math.ceil(opts.get("gamma", 3.0) * gp.n))
    bound, units, unit = family_model(dom if len(dom_fams) == 1 else "qr_update", sz, s_rows, dom_cnt,
                                      nj * args.steps)
    if len(dom_fams) == 2:
        units = 2.0 * units
    roof = None
    if units is not None and dom_ms > 0:
        achieved = units / (dom_ms / 1e3)
        if bound == "hbm":
            peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] if os.path.exists(
                os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
            roof = {"bound": "hbm", "achieved": achieved / 1e9, "peak": peak, "unit": "GB/s",
                    "frac": achieved / 1e9 / peak, "traffic": None, "kernel": "+".join(dom_fams),
                    "launches": dom_cnt, "avg_launch_ms": dom_ms / max(1, dom_cnt),
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}
        else:
            roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": FP64_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / 1e12 / FP64_ALU_PEAK_TFLOPS, "traffic": None, "kernel": "+".join(dom_fams),
                    "launches": dom_cnt, "avg_launch_ms": dom_ms / max(1, dom_cnt),
                    "peak_source": "FP64 FMA: 152 SMs x 4 flop/clk x 2.07 GHz (derived; cuBLAS dgemm measured 1.10)"}
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * max_s / steps_per_rank, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["label"], "solver": wl["solver"], "parallelism": "replicas" if world > 1 else "1gpu",
                   "precision": PRECISION_NAMES[wl["precision"]],
                   "l2": "flushed (512 MiB write) between timed steps"},
        "accuracy": {"rel_l2_vs_exact": rel_exact, "outer_iters": info["outer_iters"], "n_jac": info["n_jac"],
                     "lsqr_iters_total": info["lsqr_iters_total"]},
        "phase_ms": {k: info[k] for k in ("t_assemble", "t_sketch", "t_qr", "t_lsqr", "t_linesearch", "t_total")},
        "kernel_ms_warmup_step": {k: round(v, 3) for k, v in fam_ms.items() if v > 0},
        "roofline": roof,
        "gpu_launches": int(launches),
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": 8 * gp.n, "d2h_bytes_per_step": 8 * gp.n,
                "includes": "problem creation + H2D c0 + solve + D2H c"},
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, budget_s=args.cpu_budget)
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


# ------------------------------------------------------------------ oracle
def _threads():
    try:
        from threadpoolctl import threadpool_info
        return max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        return os.cpu_count()


def cpu_baseline(wl, budget_s=15.0):
    """The oracle as it stands, timed on the host cores on a bounded sample."""
    from oracle import newton
    from oracle.problem import Problem as OProblem
    desc, opts = wl["desc"], wl["opts"]
    op = OProblem(desc)
    t0 = time.perf_counter()
    count = 0
    while True:
        getattr(newton, wl["solver"])(op, opts)
        count += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return {"value": count / el, "unit": "solves/s", "cores": _threads(), "kind": "oracle",
            "sample": f"{count} complete oracle {wl['solver'].upper()} solves of the same instance"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    wl = workload(args.workload, args.precision, args.solver)
    from oracle import newton
    from oracle.problem import Problem as OProblem
    op = OProblem(wl["desc"])
    fn = getattr(newton, wl["solver"])
    for _ in range(args.warmup):
        fn(op, wl["opts"])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        fn(op, wl["opts"])
    el = time.perf_counter() - t0
    v = args.steps / el
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["label"], "solver": wl["solver"]},
        "cpu_baseline": {"value": v, "unit": "solves/s", "cores": _threads(), "kind": "oracle",
                         "sample": f"{args.steps} complete oracle solves"},
        "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c1")
    ap.add_argument("--precision", type=int, default=None)
    ap.add_argument("--solver", default=None, choices=[None, "ipn", "amipn"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
