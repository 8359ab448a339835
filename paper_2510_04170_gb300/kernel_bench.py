"""Micro-benchmarks of single hot-path kernels, for profiling and roofline
checks (run under ncu or plain):

  python -m paper_2510_04170_gb300.kernel_bench qr --s 32768 --n 1024 [--tc]
  python -m paper_2510_04170_gb300.kernel_bench gemm --M 128 --N 32768 --K 65536
  python -m paper_2510_04170_gb300.kernel_bench sketch --workload c2 --precision 1

Prints one JSON line with the CUDA-event time and the algorithmic rate."""
import argparse
import json
import os
import sys

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2510_04170_gb300 import build, rfm  # noqa: E402


def _time(fn, reps=1):
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["qr", "gemm", "sketch", "trsv"])
    ap.add_argument("--s", type=int, default=32768)
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--M", type=int, default=128)
    ap.add_argument("--N", type=int, default=32768)
    ap.add_argument("--K", type=int, default=65536)
    ap.add_argument("--tc", action="store_true")
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--precision", type=int, default=1)
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--prof", action="store_true", help="report per-kernel-family CUDA-event times")
    a = ap.parse_args()
    build.build()
    lib = rfm.load()
    lib.rfm_profile_enable.argtypes = [rfm.ctypes.c_int]
    lib.rfm_profile_name.restype = rfm.ctypes.c_char_p
    nfam = lib.rfm_profile_count()
    torch.manual_seed(0)
    out = {"what": a.what}
    if a.what == "qr":
        A0 = torch.randn(a.n, a.s, dtype=torch.float64, device="cuda")
        fn = rfm.rfm_householder_r_tc if a.tc else rfm.rfm_householder_r
        A = A0.clone()
        fn(A, a.s, a.n)  # warm-up
        A = A0.clone()
        if a.prof:
            lib.rfm_profile_enable((1 << nfam) - 1)
        ms = _time(lambda: fn(A, a.s, a.n))
        fl = 2.0 * a.n * a.n * (a.s - a.n / 3.0)
        out.update(s=a.s, n=a.n, tc=a.tc, ms=ms, fp64_equiv_tflops=fl / ms / 1e9)
    elif a.what == "gemm":
        A = torch.randn(a.K, a.M, dtype=torch.float64, device="cuda")
        B = torch.randn(a.N, a.K, dtype=torch.float64, device="cuda")
        rfm.rfm_emulated_dgemm(A, B)
        if a.prof:
            lib.rfm_profile_enable((1 << nfam) - 1)
        ms = _time(lambda: rfm.rfm_emulated_dgemm(A, B), a.reps)
        fl = 2.0 * a.M * a.N * a.K
        out.update(M=a.M, N=a.N, K=a.K, ms=ms, fp64_equiv_tflops=fl / ms / 1e9,
                   bf16_pair_tflops=36 * fl / ms / 1e9)
    elif a.what == "trsv":
        import rfm_workloads as W
        desc = {"c2": W.config_c2, "c1": W.config_c1,
                "n16k": lambda: W.problem(3, (4, 4, 4), 256, (6, 6, 6), (3, 3, 3), (3, 3, 3))}[a.workload]()
        gp = rfm.Problem(desc)
        n = gp.n
        R = torch.randn(n, n, dtype=torch.float64, device="cuda").triu_() / n ** 0.5
        R.diagonal().add_(2.0)
        gp.rfm_set_r(R.T.contiguous())  # column-major
        del R
        b = torch.randn(n, dtype=torch.float64, device="cuda")
        gp.rfm_trsv(b, 0)
        if a.prof:
            lib.rfm_profile_enable((1 << nfam) - 1)
        ms0 = _time(lambda: gp.rfm_trsv(b, 0), a.reps)
        ms1 = _time(lambda: gp.rfm_trsv(b, 1), a.reps)
        byts = 8.0 * n * (n + 1) / 2
        out.update(n=n, ms_upper=ms0, ms_upper_t=ms1, gbs_upper=byts / ms0 / 1e6, gbs_upper_t=byts / ms1 / 1e6)
    else:
        import rfm_workloads as W
        desc = {"c2": W.config_c2, "c1": W.config_c1}[a.workload]()
        gp = rfm.Problem(desc)
        c = torch.zeros(gp.n, dtype=torch.float64, device="cuda")
        gp.rfm_assemble(c)
        gp.rfm_set_precision(a.precision)
        s = 65536 if a.workload == "c2" else 2 * gp.n
        gp.rfm_sketch("gauss", s, 0, copy_out=False)
        if a.prof:
            lib.rfm_profile_enable((1 << nfam) - 1)
        ms = _time(lambda: gp.rfm_sketch("gauss", s, 1, copy_out=False))
        nnz = gp.m * gp.W + gp.m_iface * gp.W
        out.update(workload=a.workload, precision=a.precision, s=s, ms=ms,
                   fp64_equiv_tflops=2.0 * s * nnz / ms / 1e9)
    if a.prof:
        fam = {}
        for i in range(nfam):
            ms, cnt = rfm.ctypes.c_double(), rfm.ctypes.c_int64()
            lib.rfm_profile_read(i, rfm.ctypes.byref(ms), rfm.ctypes.byref(cnt))
            if cnt.value:
                fam[lib.rfm_profile_name(i).decode()] = [round(ms.value, 3), cnt.value]
        out["families_ms_launches"] = fam
    print(json.dumps(out))


if __name__ == "__main__":
    main()
