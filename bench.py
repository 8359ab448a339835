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


def roofline(dom_fams, dom_ms, dom_cnt, dom_work):
    """Roofline entry of the dominant kernel family from its CUDA-event time,
    launch count and the algorithmic work the library recorded per launch."""
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    roof = None
    bound = BOUND.get(dom_fams[0])
    if bound and dom_ms > 0 and dom_work > 0:
        rate = dom_work / (dom_ms / 1e3)
        common = {"traffic": None, "kernel": "+".join(dom_fams), "launches": dom_cnt,
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
        "roofline": roofline(dom_fams, dom_ms, dom_cnt, dom_work),
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
    roof = roofline(dom_fams, dom_ms, dom_cnt, dom_work)
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
        line["cpu_baseline"] = cpu_baseline(wl, budget_s=args.cpu_budget, info=info)
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


def oracle_projection(wl, outer_iters, lsqr_iters, qr_cols=4096):
    """Projected time of one oracle solve of a workload too large to run whole:
    each oracle step is timed on a sample at the workload's sizes and scaled
    by its operation count (assembly per row, Gaussian sketch per column
    block, Householder QR per flop 2 n^2 (s - n/3), triangular solve per n^2,
    block products per nonzero), with the iteration counts of the solve.
    Returns (seconds per solve, sample description, seconds spent sampling)."""
    import numpy as np
    from oracle import assemble as asm
    from oracle import linalg as la
    from oracle import philox
    from oracle.problem import Problem as OProblem
    t_all = time.perf_counter()
    desc, opts = wl["desc"], wl["opts"]
    op = OProblem(desc)
    n, m, W_ = op.n, op.m, op.W
    s = opts["sketch_rows"] or int(math.ceil(opts["gamma"] * n))
    c = np.zeros(n)
    rng = np.random.default_rng(0)
    # assembly of F and J: 2048 sampled rows
    rows = np.sort(rng.choice(m, 2048, replace=False))
    t0 = time.perf_counter()
    asm.assemble_rows(op, c, rows)
    t_asm = (time.perf_counter() - t0) * m / rows.size
    if opts.get("sketch_kind", "count") == "gauss":
        # Gaussian sketch of one column block (generation + product), times G blocks
        blk_rows = np.nonzero((op.re0 == 0) | (op.re1 == 0))[0]
        Jb = rng.standard_normal((blk_rows.size, W_))
        t0 = time.perf_counter()
        S = philox.gaussian_sketch(s, blk_rows, 0, desc["seed"])
        S @ Jb
        t_sk = (time.perf_counter() - t0) * op.G
        del S
    else:
        # count sketch: the oracle adds dense rows of J; 2048 rows x 1024 columns, scaled to m x n
        Jc = rng.standard_normal((2048, 1024))
        t0 = time.perf_counter()
        la.count_sketch(Jc, 4096, 0, desc["seed"])
        t_sk = (time.perf_counter() - t0) * (m / 2048) * (n / 1024)
    # Householder QR = per-column panel work (one s x 64 panel factorised)
    # plus the blocked trailing update, 2 n^2 (s - n/3) flops at the rate of
    # the oracle's own trailing-update products (V^T A, A -= V W) measured on
    # an s x 64 by s x qr_cols sample
    B = rng.standard_normal((s, 64))
    t0 = time.perf_counter()
    la.qr_r_blocked(B, nb=64)
    t_col = (time.perf_counter() - t0) / 64
    V = rng.standard_normal((s, 64))
    A = rng.standard_normal((s, qr_cols))
    t0 = time.perf_counter()
    Wm = V.T @ A
    A -= V @ Wm
    rate = 4.0 * s * 64 * qr_cols / (time.perf_counter() - t0)
    del B, V, A, Wm
    t_qr = n * t_col + 2.0 * n * n * (s - n / 3.0) / rate
    # triangular solve (n^2) and block product J x (nnz) per LSQR iteration
    nt = 8192
    Rs = np.triu(rng.standard_normal((nt, nt))) + nt * np.eye(nt)
    t0 = time.perf_counter()
    la.solve_upper(Rs, rng.standard_normal(nt))
    t_tr = (time.perf_counter() - t0) * (n / nt) ** 2
    Jr = rng.standard_normal((4096, W_))
    xr = rng.standard_normal(W_)
    t0 = time.perf_counter()
    for _ in range(4):
        Jr @ xr
    t_mv = (time.perf_counter() - t0) / 4 * (m + op.m_iface) / 4096
    t_it = 2 * t_tr + 2 * t_mv
    # line search: about 19 residual evaluations per Newton step, each ~ an assembly
    t_ls = 19 * t_asm * 0.5
    per_solve = outer_iters * (t_asm + t_sk + t_qr + t_ls) + lsqr_iters * t_it
    sk = (f"Gaussian sketch of 1 of {op.G} column blocks" if opts.get("sketch_kind", "count") == "gauss"
          else "count sketch of 2048 x 1024")
    sample = (f"oracle steps timed on samples and scaled by operation counts: assembly of 2048 rows, "
              f"{sk}, Householder panel {s}x64 and "
              f"trailing-update product {s}x64 by {s}x{qr_cols}, R solve n=8192, 4096-row block product; {outer_iters} outer and "
              f"{lsqr_iters} LSQR iterations")
    return per_solve, sample, time.perf_counter() - t_all


def cpu_baseline(wl, budget_s=15.0, info=None):
    """The oracle as it stands, timed on the host cores on a bounded sample."""
    from oracle import newton
    from oracle.problem import Problem as OProblem
    desc, opts = wl["desc"], wl["opts"]
    if wl.get("large"):
        per, sample, _ = oracle_projection(wl, info["outer_iters"], info["lsqr_iters_total"])
        return {"value": 1.0 / per, "unit": "solves/s", "cores": _threads(), "kind": "oracle", "sample": sample,
                "projected_seconds_per_solve": per}
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
        # each step: one bounded sample of the oracle's steps, projected to a solve
        # (iteration counts of the GPU solve of this workload: IT 4, 137 LSQR steps)
        per = []
        for i in range(args.warmup + args.steps):
            p_, sample, _ = oracle_projection(wl, 4, 137, qr_cols=2048)
            if i >= args.warmup:
                per.append(p_)
        v = 1.0 / statistics.median(per)
        el = sum(per)
        sample = "per step: " + sample
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
