"""Benchmark: Newton solves/s of the RFM IPN solver on GB300 (one JSON line).

Workloads (seeded synthetic PDE instances; the paper uses no datasets):
  c2  3D -Lap u + u^3 = f, u* = prod sin(pi x), 4x4x4 subdomains, M=512
      (n = 32,768), 12^3 interior points and 6x6 per face (m = 124,416),
      Gaussian sketch with 65,536 rows, IPN.
  c1  2D analogue: 2x2 subdomains, M=100, 20x20 points, count sketch gamma=3.
  c3  3D steady Gray-Scott (two fields), n = 32,768, AMIPN with inner cap 5.
  c4  64 uneven instances (n = 1,024 .. 16,384) solved as one batch per step,
      QR configuration autotuned per instance size.
  c5  128 held-out instances of a parameterised family solved as one batch per
      step from the learned warm start's prediction (trained beforehand on 512
      solver outputs); the same instances from c_0 = 0 are timed for comparison.

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

T_START = time.time()

METRIC = "Newton solves/s at rel-L2<=1e-6 vs FP64 oracle (IPN)"
FP64_ALU_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12  # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz


PRECISION_NAMES = {0: "fp64", 1: "fp64 + tensor-core sketch", 2: "fp64 + tensor-core sketch and QR update",
                   -1: "autotuned per instance (fp64 or tensor-core QR update)"}


def workload(name, precision=None, solver=None):
    if name == "c1":
        p = 0 if precision is None else precision
        wl = dict(desc=W.config_c1(), opts=W.solve_opts(precision=p), solver=solver or "ipn",
                  label="c1: 2D -Lap u+u^3, 2x2 subdomains, M=100, n=400, m=1920, count sketch s=1200")
    elif name == "c2":
        p = 2 if precision is None else precision
        wl = dict(desc=W.config_c2(), opts=W.opts_c2(precision=p), solver=solver or "ipn", large=True,
                  oracle_npz="c2_ipn_oracle.npz" if (solver or "ipn") == "ipn" else None, forms=True,
                  oracle_timing="c2_oracle_timing.json",
                  label="c2: 3D -Lap u+u^3, 4x4x4 subdomains, M=512, n=32768, m=124416, Gaussian sketch s=65536")
    elif name == "c3":
        p = 2 if precision is None else precision
        wl = dict(desc=W.config_c3(), opts=W.solve_opts(precision=p, m_max=5), solver=solver or "amipn", large=True,
                  label="c3: 3D steady Gray-Scott, 2 fields, 4x4x4 subdomains, M=256 per field, n=32768, m=248832, "
                        "count sketch s=98304, AMIPN with inner cap 5")
    elif name == "c4":
        p = -1 if precision is None else precision
        wl = dict(descs=W.config_c4_instances(64, seed=1), opts=W.solve_opts(precision=p), solver=solver or "ipn",
                  kind="batch", streams=8,
                  label="c4: 64 instances of 3D -div(a grad u)+kappa u^3, g=2..4 subdomains/axis, M=128/256 "
                        "(n=1,024..16,384), kappa~U[0.1,10], count sketch gamma=3, batched")
    elif name == "c5":
        p = 2 if precision is None else precision
        wl = dict(opts=W.solve_opts(precision=p), solver=solver or "ipn", kind="warmstart", streams=8,
                  n_train=512, n_test=128,
                  label="c5: 128 held-out 3D -div(a grad u)+kappa u^3 = A prod sin(q pi x), 2x2x2 subdomains, "
                        "M=512 (n=4,096), kappa~U[0.1,10], A~U[0.5,2], q~U{1..4}; learned warm start trained "
                        "on 512 solver outputs, batched")
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


# kernel family -> roofline bound; algorithmic work per launch is recorded by the
# library at each launch site (rfm_profile_work)
BOUND = {"oz_gemm": "tensor", "qr_vta": "alu", "qr_update": "alu", "sketch_gemm": "alu",
         "trsv": "hbm", "jmv": "hbm", "jtmv": "hbm", "assemble": "hbm"}


def leaf_families(precision):
    """Families whose timed scope contains no other family's launches."""
    skip = set()
    if precision >= 1:
        skip.add("sketch_gemm")
    if precision >= 2:
        skip |= {"qr_vta", "qr_update"}
    return skip


def job_throughput(seconds_this_rank, units_this_rank, dist=None, device="cpu"):
    """Whole-job rate over replicas: every rank processed units_this_rank in
    its own seconds_this_rank; the job lasts as long as its slowest rank (max
    over ranks).  Returns (units of all ranks / that time, that time)."""
    import torch
    t = torch.tensor([float(seconds_this_rank)], dtype=torch.float64, device=device)
    world = 1
    if dist is not None and dist.is_initialized():
        world = dist.get_world_size()
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
    max_s = float(t.item())
    return world * units_this_rank / max_s, max_s


def setup_lib(rfm):
    lib = rfm.load()
    lib.rfm_profile_enable.argtypes = [rfm.ctypes.c_int]
    lib.rfm_launch_count.restype = rfm.ctypes.c_int64
    lib.rfm_profile_read.argtypes = [rfm.ctypes.c_int, rfm.ctypes.POINTER(rfm.ctypes.c_double),
                                     rfm.ctypes.POINTER(rfm.ctypes.c_int64)]
    lib.rfm_profile_name.restype = rfm.ctypes.c_char_p
    lib.rfm_profile_work.argtypes = [rfm.ctypes.c_int, rfm.ctypes.POINTER(rfm.ctypes.c_double)]
    return lib


def family_names(lib):
    return [lib.rfm_profile_name(i).decode() for i in range(lib.rfm_profile_count())]


def read_families(lib, rfm, names):
    out = {}
    for i, nm in enumerate(names):
        ms, cnt = rfm.ctypes.c_double(), rfm.ctypes.c_int64()
        lib.rfm_profile_read(i, rfm.ctypes.byref(ms), rfm.ctypes.byref(cnt))
        out[nm] = ms.value
    return out


def pick_dominant(fam_ms, names, precision):
    """Family with the most device time among the leaf families with a roofline
    bound; the FP64 QR trailing update is one pair of families."""
    skip = leaf_families(precision)
    cand = {k: v for k, v in fam_ms.items() if k not in skip and k in BOUND}
    dom = max(cand, key=lambda k: cand[k]) if any(cand.values()) else ("oz_gemm" if precision != 0 else "qr_update")
    dom_fams = ["qr_vta", "qr_update"] if dom in ("qr_vta", "qr_update") else [dom]
    return dom_fams, sum(1 << names.index(f) for f in dom_fams)


def read_dominant(lib, rfm, names, dom_fams):
    dom_ms, dom_cnt, dom_work = 0.0, 0, 0.0
    for f in dom_fams:
        ms, cnt, wk = rfm.ctypes.c_double(), rfm.ctypes.c_int64(), rfm.ctypes.c_double()
        lib.rfm_profile_read(names.index(f), rfm.ctypes.byref(ms), rfm.ctypes.byref(cnt))
        lib.rfm_profile_work(names.index(f), rfm.ctypes.byref(wk))
        dom_ms += ms.value
        dom_cnt += cnt.value
        dom_work += wk.value
    return dom_ms, dom_cnt, dom_work


# DRAM traffic per launch of a dominant kernel family, from one ncu capture of
# the same workload (dram__bytes_read.sum + dram__bytes_write.sum), keyed by
# (workload, precision, family).  c2 / 2 / oz_gemm: the first 600 k_oz_gemm
# launches of one c2 solve (the sketch and the larger early blocks of the
# first factorisation) moved 1,869 GB/s of their device time. That rate times
# the solve's mean launch duration (5.17 ms) gives the mean launch's bytes.
# Taken with the grouped-MMA, 16-epilogue-warp, split-K kernel and the T^T W
# product; it must be measured again whenever those launches change.
MEASURED_TRAFFIC = {("c2", 2, "oz_gemm"): 9.66e9}


def roofline(dom_fams, dom_ms, dom_cnt, dom_work, key=None):
    """Roofline entry of the dominant kernel family from its CUDA-event time,
    launch count and the algorithmic work the library recorded per launch."""
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    roof = None
    bound = BOUND.get(dom_fams[0])
    if bound and dom_ms > 0 and dom_work > 0:
        rate = dom_work / (dom_ms / 1e3)
        common = {"traffic": MEASURED_TRAFFIC.get(tuple(key or ()) + ("+".join(dom_fams),)), "kernel": "+".join(dom_fams),
                  "launches": dom_cnt,
                  "avg_launch_ms": dom_ms / max(1, dom_cnt), "work_per_launch": dom_work / max(1, dom_cnt)}
        if bound == "hbm":
            peak = peaks.get("hbm_gbs", 6800.0)
            roof = dict(bound="hbm", achieved=rate / 1e9, peak=peak, unit="GB/s", frac=rate / 1e9 / peak,
                        peak_source="MEASURED_PEAKS.json hbm_gbs (measured)", **common)
        elif bound == "tensor":
            peak = peaks.get("bf16_tflops_sustained", 1700.0)
            roof = dict(bound="tensor", achieved=rate / 1e12, peak=peak, unit="TFLOP/s", frac=rate / 1e12 / peak,
                        peak_source="MEASURED_PEAKS.json bf16_tflops_sustained (measured; kernel timed inside a long "
                                    "step); work = bf16 digit-pair products",
                        fp64_equivalent_tflops=rate / 1e12 / 36.0, **common)
        else:
            roof = dict(bound="alu", achieved=rate / 1e12, peak=FP64_ALU_PEAK_TFLOPS, unit="TFLOP/s",
                        frac=rate / 1e12 / FP64_ALU_PEAK_TFLOPS,
                        peak_source="FP64 FMA: 152 SMs x 4 flop/clk x 2.07 GHz (derived; cuBLAS dgemm measured 1.10)",
                        **common)
    return roof


def run_batch(args, rank, world, local_rank, wl, lib, rfm, dist):
    """Batched workloads: c4 (64 uneven instances per step) and c5 (128
    held-out instances per step, each started from the learned warm start's
    prediction, prediction included).  Each step is timed between CUDA events
    recorded after a device-wide synchronisation (the batch spreads over
    several streams); L2 is flushed between steps."""
    import torch
    from paper_2510_04170_gb300 import warmstart
    opts = wl["opts"]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    extra = {}
    if wl["kind"] == "batch":
        descs = wl["descs"]
        batch = rfm.Batch(descs, streams=wl["streams"])

        def work():
            return batch.solve(opts, solver=wl["solver"])
    else:
        ptrain = warmstart.sample_params(wl["n_train"], 1)
        ptest = warmstart.sample_params(wl["n_test"], 10001)
        t0 = time.perf_counter()
        bt = rfm.Batch([warmstart.family_desc(p) for p in ptrain], streams=wl["streams"])
        ctrain, _, _ = bt.solve(opts, solver=wl["solver"])
        bt.close()
        torch.cuda.synchronize()
        t_data = time.perf_counter() - t0
        t0 = time.perf_counter()
        ws = warmstart.train_warm_start(ptrain, torch.stack(ctrain), warmstart.family_desc(ptrain[0]))
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        del ctrain
        descs = [warmstart.family_desc(p) for p in ptest]
        batch = rfm.Batch(descs, streams=wl["streams"])
        params = torch.as_tensor(ptest, device="cuda")
        extra = {"warm_start": {"rank": ws.rank, "train_loss": ws.losses[-1], "t_training_data_s": t_data,
                                "t_train_s": t_train, "n_train": wl["n_train"]}}

        def work():
            c0 = ws.predict(params)
            return batch.solve(opts, solver=wl["solver"], c0=[c0[i] for i in range(len(descs))])

    def one():
        flush.zero_()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        out = work()
        torch.cuda.synchronize()
        b.record()
        b.synchronize()
        return a.elapsed_time(b), out

    names = family_names(lib)
    out = None
    for wi in range(args.warmup):
        if wi == args.warmup - 1:
            lib.rfm_profile_enable((1 << len(names)) - 1)
        _, out = one()
    fam_ms = read_families(lib, rfm, names)
    lib.rfm_profile_enable(0)
    dom_fams, mask = pick_dominant(fam_ms, names, 2 if wl["precision"] != 0 else 0)
    if dist:
        dist.barrier()
    lib.rfm_profile_enable(mask)
    l0 = lib.rfm_launch_count()
    times = []
    with ClockSampler(local_rank) as clk:
        for _ in range(args.steps):
            ms, out = one()
            times.append(ms)
    launches = lib.rfm_launch_count() - l0
    dom_ms, dom_cnt, dom_work = read_dominant(lib, rfm, names, dom_fams)
    lib.rfm_profile_enable(0)
    cs, infos, tuned = out
    count = len(descs)
    value, max_s = job_throughput(sum(times) / 1e3, count * args.steps, dist, "cuda")
    acc = {"outer_iters_mean": float(np.mean([i["outer_iters"] for i in infos])),
           "n_jac_mean": float(np.mean([i["n_jac"] for i in infos])),
           "lsqr_iters_mean": float(np.mean([i["lsqr_iters_total"] for i in infos]))}
    if wl["kind"] == "batch":
        from oracle.problem import Problem as OProblem  # exact solution formula only
        errs = []
        for d, gp, c in zip(descs, batch.problems, cs):
            X = W.eval_grid(d, per_axis=4)
            u = gp.rfm_eval(c, torch.as_tensor(X, device="cuda")).cpu().numpy()
            ue = OProblem(d).exact(X)
            errs.append(float(np.linalg.norm(u - ue) / np.linalg.norm(ue)))
        acc["rel_l2_vs_exact_max"] = max(errs)
        acc["tuned_precision_counts"] = {str(k): tuned.count(k) for k in sorted(set(tuned))}
    else:
        # the same held-out instances from c_0 = 0, for the comparison
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cz, iz, _ = batch.solve(opts, solver=wl["solver"])
        torch.cuda.synchronize()
        tz = time.perf_counter() - t0
        rel = []
        for d, gp, c, z in zip(descs, batch.problems, cs, cz):
            X = torch.as_tensor(W.eval_grid(d, per_axis=4), device="cuda")
            uw, uz = gp.rfm_eval(c, X).cpu().numpy(), gp.rfm_eval(z, X).cpu().numpy()
            rel.append(float(np.linalg.norm(uw - uz) / np.linalg.norm(uz)))
        acc.update({"rel_l2_warm_vs_zero_start_max": max(rel),
                    "zero_start": {"solves_per_s": count / tz,
                                   "n_jac_mean": float(np.mean([i["n_jac"] for i in iz])),
                                   "outer_iters_mean": float(np.mean([i["outer_iters"] for i in iz]))}})
    # end to end: problems from host descriptors, pinned H2D of c_0, solve, D2H
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b2 = rfm.Batch(descs, streams=wl["streams"])
    host0 = [torch.zeros(p.n, dtype=torch.float64).pin_memory() for p in b2.problems]
    c0d = [h.to("cuda", non_blocking=True) for h in host0]
    c2, _, _ = b2.solve(opts, solver=wl["solver"], c0=c0d)
    outs = [c.to("cpu") for c in c2]
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    nbytes = 8 * sum(p.n for p in b2.problems)
    del outs
    b2.close()
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * max_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["label"], "solver": wl["solver"], "instances_per_step": count,
                   "streams": wl["streams"], "parallelism": "replicas" if world > 1 else "1gpu",
                   "precision": PRECISION_NAMES[wl["precision"]],
                   "l2": "flushed (512 MiB write) between timed steps"},
        "accuracy": acc,
        "kernel_ms_warmup_step": {k: round(v, 3) for k, v in fam_ms.items() if v > 0},
        "roofline": roofline(dom_fams, dom_ms, dom_cnt, dom_work, (args.workload, wl["precision"])),
        "gpu_launches": int(launches),
        "e2e": {"value": world * count / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes, "includes": "batch creation + H2D c0 + solves + D2H c"},
        "clocks": clk.summary(),
    }
    line.update(extra)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = batch_cpu_baseline(wl, descs, infos)
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


def batch_cpu_baseline(wl, descs, infos):
    """Oracle projection per distinct instance shape (same operation-count
    scaling as the single-instance workloads), summed over the batch."""
    classes = {}
    for d, inf in zip(descs, infos):
        classes.setdefault((d["nsub"], d["M"]), []).append((d, inf))
    total, parts = 0.0, []
    for key, items in classes.items():
        d, _ = items[0]
        it = max(1, int(round(np.mean([i["outer_iters"] for _, i in items]))))
        ls = int(round(np.mean([i["lsqr_iters_total"] for _, i in items])))
        per, _, _ = oracle_projection(dict(desc=d, opts=W.solve_opts(), solver="ipn"), it, ls, qr_cols=1024)
        total += per * len(items)
        parts.append(f"{len(items)} x g={key[0][0]} M={key[1]}: {per:.1f} s")
    return {"value": len(descs) / total, "unit": "solves/s", "cores": _threads(), "kind": "oracle",
            "sample": "oracle steps timed on samples at each instance shape and scaled by operation counts "
                      "(as for c2), with the GPU solves' iteration counts; " + "; ".join(parts)}


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
    lib = setup_lib(rfm)
    wl = workload(args.workload, args.precision, args.solver)
    if wl.get("kind") and args.instances:
        if wl["kind"] == "batch":
            wl["descs"] = wl["descs"][:args.instances]
        else:
            wl["n_test"] = args.instances
            wl["n_train"] = min(wl["n_train"], 4 * args.instances)
        wl["label"] += f" [reduced to {args.instances} instances]"
    if wl.get("kind"):
        return run_batch(args, rank, world, local_rank, wl, lib, rfm, dist)
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

    names = family_names(lib)
    # warm-up; the last warm-up step is profiled per family to pick the dominant kernel
    info = None
    for wi in range(args.warmup):
        if wi == args.warmup - 1:
            lib.rfm_profile_enable((1 << len(names)) - 1)
        _, c, info = one()
    fam_ms = read_families(lib, rfm, names)
    lib.rfm_profile_enable(0)
    dom_fams, mask = pick_dominant(fam_ms, names, wl["precision"])

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
    dom_ms, dom_cnt, dom_work = read_dominant(lib, rfm, names, dom_fams)
    lib.rfm_profile_enable(0)
    value, max_s = job_throughput(sum(times) / 1e3, args.steps, dist, "cuda")
    if dist:
        dist.barrier()

    # accuracy of the last solve: against the manufactured solution and, where
    # a stored whole oracle solve of this instance exists, against the oracle
    X = W.eval_grid(desc)
    u = gp.rfm_eval(c, torch.as_tensor(X, device="cuda")).cpu().numpy()
    from oracle.problem import Problem as OProblem  # exact solution formula only
    ue = OProblem(desc).exact(X)
    acc = {"status": STATUS[info["status"]], "final_resid": info["final_resid"],
           "rel_l2_vs_exact": float(np.linalg.norm(u - ue) / np.linalg.norm(ue)),
           "outer_iters": info["outer_iters"], "n_jac": info["n_jac"], "lsqr_iters_total": info["lsqr_iters_total"]}
    ref = stored_oracle_solve(args, wl)
    gate_ok = info["status"] == 0
    if ref is not None:
        rel_o = float(np.linalg.norm(u - ref["u"]) / np.linalg.norm(ref["u"]))
        same = (info["outer_iters"] == int(ref["outer_iters"]) and info["n_jac"] == int(ref["n_jac"])
                and info["lsqr_iters_total"] == int(np.sum(ref["lsqr_iters"])))
        acc.update({"rel_l2_vs_oracle": rel_o, "oracle_counts": {
            "outer_iters": int(ref["outer_iters"]), "n_jac": int(ref["n_jac"]),
            "lsqr_iters_total": int(np.sum(ref["lsqr_iters"]))}, "counts_equal_oracle": same})
        gate_ok = gate_ok and rel_o <= GATE_REL_L2
    acc["gate"] = {"requires": f"status OK and rel-L2 vs the stored FP64 oracle solve <= {GATE_REL_L2:g}"
                               if ref is not None else "status OK (no stored oracle solve of this instance)",
                   "passed": bool(gate_ok)}

    # end to end through the public API from host memory
    e2e_times = []
    c0_host = torch.zeros(gp.n, dtype=torch.float64).pin_memory()
    out_host = torch.empty(gp.n, dtype=torch.float64).pin_memory()
    for _ in range(1 if wl.get("large") else max(1, min(args.steps, 3))):
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
    roof = roofline(dom_fams, dom_ms, dom_cnt, dom_work, (args.workload, wl["precision"]))
    line = {
        "metric": METRIC, "value": value if gate_ok else None, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * max_s / steps_per_rank, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["label"], "solver": wl["solver"], "parallelism": "replicas" if world > 1 else "1gpu",
                   "precision": PRECISION_NAMES[wl["precision"]],
                   "l2": "flushed (512 MiB write) between timed steps"},
        "accuracy": acc,
        "phase_ms": {k: info[k] for k in ("t_assemble", "t_sketch", "t_qr", "t_lsqr", "t_linesearch", "t_total")},
        "kernel_ms_warmup_step": {k: round(v, 3) for k, v in fam_ms.items() if v > 0},
        "roofline": roof,
        "gpu_launches": int(launches),
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": 8 * gp.n, "d2h_bytes_per_step": 8 * gp.n,
                "includes": "problem creation + H2D c0 + solve + D2H c"},
        "clocks": clk.summary(),
    }
    if not gate_ok:
        line["value_ungated"] = value
    if wl.get("forms") and args.forms != "off" and world == 1:
        line["forms"] = forms_record(args, wl, rfm, line, info)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, budget_s=args.cpu_budget, info=info)
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


STATUS = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ENOCONV", "ERANK", "ENONFINITE", "ETIMEOUT"]
GATE_REL_L2 = 1e-6
GOLDEN = os.path.join(ROOT, "tests", "golden")


def stored_oracle_solve(args, wl):
    """The stored whole oracle solve of this workload's instance (written by
    tests/golden/make_c2_ipn_oracle.py, which calls only the oracle), or None."""
    name = wl.get("oracle_npz")
    if not name or not os.path.exists(os.path.join(GOLDEN, name)):
        return None
    return np.load(os.path.join(GOLDEN, name))


def forms_record(args, wl, rfm, line, info):
    """The metric's comparison on this GPU: plain FP64 IPN against each form
    (mixed precision, batching, learned warm start).  Each entry is two timed
    runs of the same instances that differ only in the option named, with the
    accuracy of both.  The plain FP64 solve of the headline instance runs only
    if the run stays within the wall-clock budget (--budget seconds since the
    start); its projected duration is recorded either way."""
    import torch
    from paper_2510_04170_gb300 import warmstart
    out = {}
    # -- mixed precision: the headline instance in plain FP64
    ph = info
    est = (8.5 * ph["t_qr"] + 3.0 * ph["t_sketch"] + (ph["t_total"] - ph["t_qr"] - ph["t_sketch"])) / 1e3
    elapsed = time.time() - T_START
    mixed = {"solves_per_s": line["value"] if line["value"] is not None else line.get("value_ungated"),
             "rel_l2_vs_oracle": line["accuracy"].get("rel_l2_vs_oracle")}
    rec = {"mixed_solves_per_s": mixed["solves_per_s"], "mixed_rel_l2_vs_oracle": mixed["rel_l2_vs_oracle"],
           "plain_projected_s": est}
    if args.forms == "on" or elapsed + est <= args.budget:
        import torch as _t
        stream = _t.cuda.Stream()
        with _t.cuda.stream(stream):
            gp = rfm.Problem(wl["desc"], stream=stream)
        opts0 = dict(wl["opts"], precision=0)
        a = _t.cuda.Event(enable_timing=True)
        b = _t.cuda.Event(enable_timing=True)
        with _t.cuda.stream(stream):
            a.record(stream)
            c, inf0 = gp.rfm_ipn_solve(opts0)
            b.record(stream)
        b.synchronize()
        t_plain = a.elapsed_time(b) / 1e3
        X = W.eval_grid(wl["desc"])
        u = gp.rfm_eval(c, _t.as_tensor(X, device="cuda")).cpu().numpy()
        ref = stored_oracle_solve(args, wl)
        rec.update({"plain_solves_per_s": 1.0 / t_plain, "plain_status": STATUS[inf0["status"]],
                    "plain_counts": [inf0["outer_iters"], inf0["n_jac"], inf0["lsqr_iters_total"]],
                    "gain": mixed["solves_per_s"] * t_plain if mixed["solves_per_s"] else None})
        if ref is not None:
            rec["plain_rel_l2_vs_oracle"] = float(np.linalg.norm(u - ref["u"]) / np.linalg.norm(ref["u"]))
        gp.close()
    else:
        rec["plain"] = (f"skipped: {elapsed:.0f} s elapsed + {est:.0f} s projected exceeds the "
                        f"{args.budget:.0f} s budget")
    out["mixed_precision"] = rec
    # -- batching: the same instances on one stream vs eight (tensor-core QR)
    descs = [d for i, d in enumerate(W.config_c4_instances(64, seed=1)) if i % 3 != 2][:args.forms_instances]
    res = {}
    for streams in (1, 8):
        b = rfm.Batch(descs, streams=streams)
        b.solve(W.solve_opts(precision=2, max_outer=1))  # graphs, buffers, first-touch
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cs, infos, _ = b.solve(W.solve_opts(precision=2))
        torch.cuda.synchronize()
        res[streams] = (len(descs) / (time.perf_counter() - t0), cs, infos, b)
    dev = max(float(torch.linalg.norm(a - z) / torch.linalg.norm(z)) for a, z in zip(res[8][1], res[1][1]))
    out["batching"] = {"instances": f"{len(descs)} C4 instances with 2 or 3 subdomains per axis, M = 128/256",
                       "single_stream_solves_per_s": res[1][0], "batched_8_streams_solves_per_s": res[8][0],
                       "gain": res[8][0] / res[1][0], "max_rel_diff_c_batched_vs_single": dev}
    for r in res.values():
        r[3].close()
    # -- learned warm start: zero start vs the network's prediction
    ptrain = warmstart.sample_params(args.forms_train, 1)
    ptest = warmstart.sample_params(args.forms_instances, 10001)
    bt = rfm.Batch([warmstart.family_desc(p) for p in ptrain], streams=8)
    ctrain, _, _ = bt.solve(W.solve_opts(precision=2))
    bt.close()
    ws = warmstart.train_warm_start(ptrain, torch.stack(ctrain), warmstart.family_desc(ptrain[0]))
    del ctrain
    bz = rfm.Batch([warmstart.family_desc(p) for p in ptest], streams=8)
    params = torch.as_tensor(ptest, device="cuda")
    bz.solve(W.solve_opts(precision=2, max_outer=1))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cz, iz, _ = bz.solve(W.solve_opts(precision=2))
    torch.cuda.synchronize()
    tz = time.perf_counter() - t0
    t0 = time.perf_counter()
    c0 = ws.predict(params)
    cw, iw, _ = bz.solve(W.solve_opts(precision=2), c0=[c0[i] for i in range(len(ptest))])
    torch.cuda.synchronize()
    tw = time.perf_counter() - t0
    rel = []
    for d, gp, a, z in zip(bz.descs, bz.problems, cw, cz):
        Xe = torch.as_tensor(W.eval_grid(d, per_axis=4), device="cuda")
        ua, uz = gp.rfm_eval(a, Xe), gp.rfm_eval(z, Xe)
        rel.append(float(torch.linalg.norm(ua - uz) / torch.linalg.norm(uz)))
    out["learned_warm_start"] = {
        "instances": f"{len(ptest)} held-out instances of the C5 family (n = 4,096), network trained on "
                     f"{len(ptrain)} solver outputs", "zero_start_solves_per_s": len(ptest) / tz,
        "warm_start_solves_per_s": len(ptest) / tw, "gain": tz / tw, "prediction_included": True,
        "n_jac_mean_zero": float(np.mean([i["n_jac"] for i in iz])),
        "n_jac_mean_warm": float(np.mean([i["n_jac"] for i in iw])),
        "rel_l2_warm_vs_zero_max": max(rel)}
    bz.close()
    return out


# ------------------------------------------------------------------ oracle
def _threads():
    from oracle import timing
    return timing.threads()


def oracle_projection(wl, outer_iters, lsqr_iters, qr_cols=1024):
    """The oracle's timing model (oracle.timing.projection) for a workload."""
    from oracle import timing
    return timing.projection(wl["desc"], wl["opts"], outer_iters, lsqr_iters, qr_cols)


def oracle_counts(wl, info=None):
    """Outer and LSQR iterations of the oracle's own solve of this instance
    (stored whole solve), else those of the GPU solve."""
    ref = stored_oracle_solve(None, wl)
    if ref is not None:
        return int(ref["outer_iters"]), int(np.sum(ref["lsqr_iters"])), "the stored oracle solve"
    if info is not None:
        return info["outer_iters"], info["lsqr_iters_total"], "the GPU solve"
    return 4, 137, "assumed"


def calibration(wl):
    """measured / projected seconds of one whole oracle solve of this
    instance on the machine that measured it (tests/golden/c2_oracle_timing.json,
    written by tests/golden/calibrate_c2_oracle_model.py), or None."""
    name = wl.get("oracle_timing")
    path = os.path.join(GOLDEN, name) if name else None
    if not path or not os.path.exists(path):
        return None
    return json.load(open(path))


def projected_baseline(wl, info=None, qr_cols=1024):
    """Oracle seconds per solve from its timing model on this host, scaled by
    the model's calibration against a whole measured oracle solve."""
    it, ls, src = oracle_counts(wl, info)
    per, sample, t_sample = oracle_projection(wl, it, ls, qr_cols=qr_cols)
    cal = calibration(wl)
    factor = cal["measured_wall_s"] / cal["projected_s"] if cal else 1.0
    extra = {"projected_seconds_per_solve": per, "counts_from": src}
    if cal:
        extra["calibration"] = {"factor": factor, **cal}
    return per * factor, sample, t_sample, extra


def cpu_baseline(wl, budget_s=15.0, info=None):
    """The oracle as it stands, timed on the host cores on a bounded sample."""
    from oracle import newton
    from oracle.problem import Problem as OProblem
    desc, opts = wl["desc"], wl["opts"]
    if wl.get("large"):
        per, sample, _, extra = projected_baseline(wl, info)
        return {"value": 1.0 / per, "unit": "solves/s", "cores": _threads(), "kind": "oracle", "sample": sample,
                **extra}
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
    if wl.get("kind"):
        # each step: the oracle projected per instance shape (IT 4 and 100 LSQR
        # steps per instance assumed; the GPU arm reports the measured counts)
        if wl["kind"] == "batch":
            descs = wl["descs"]
        else:
            from paper_2510_04170_gb300 import warmstart as _ws
            descs = [_ws.family_desc(p) for p in _ws.sample_params(wl["n_test"], 10001)]
        fake = [{"outer_iters": 4, "lsqr_iters_total": 100}] * len(descs)
        per = []
        for i in range(args.warmup + args.steps):
            cb = batch_cpu_baseline(wl, descs, fake)
            if i >= args.warmup:
                per.append(len(descs) / cb["value"])  # projected seconds per step (all instances)
        v = len(descs) / statistics.median(per)
        el = sum(per)
        sample = "per step: " + cb["sample"]
    elif wl.get("large"):
        # each step: one bounded sample of the oracle's steps (the same model as
        # the cpu_baseline leg of the GPU arm), projected to a solve; the step
        # lasts as long as its sample, so a step is that fraction of a solve
        per, spent = [], []
        for i in range(args.warmup + args.steps):
            p_, sample, t_s, extra = projected_baseline(wl)
            if i >= args.warmup:
                per.append(p_)
                spent.append(t_s)
        v = 1.0 / statistics.median(per)
        el = sum(spent)
        sample = ("per step: " + sample + f"; each step is {statistics.median(spent) / statistics.median(per):.2e} "
                  "of a solve")
    else:
        op = OProblem(wl["desc"])
        fn = getattr(newton, wl["solver"])
        for _ in range(args.warmup):
            fn(op, wl["opts"])
        t0 = time.perf_counter()
        for _ in range(args.steps):
            fn(op, wl["opts"])
        el = time.perf_counter() - t0
        v = args.steps / el
        sample = f"{args.steps} complete oracle solves"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["label"], "solver": wl["solver"]},
        "cpu_baseline": {"value": v, "unit": "solves/s", "cores": _threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--precision", type=int, default=None)
    ap.add_argument("--solver", default=None, choices=[None, "ipn", "amipn"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--instances", type=int, default=None,
                    help="c4/c5: use only this many instances (functional runs; the label says so)")
    ap.add_argument("--forms", default="auto", choices=["auto", "on", "off"],
                    help="c2: add the plain-vs-forms comparison (auto: the plain FP64 solve only within --budget)")
    ap.add_argument("--budget", type=float, default=1650.0, help="wall-clock seconds for --forms auto")
    ap.add_argument("--forms-instances", type=int, default=16)
    ap.add_argument("--forms-train", type=int, default=128)
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 2 if args.workload == "c2" else 10
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
