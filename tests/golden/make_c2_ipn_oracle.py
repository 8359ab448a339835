"""Writes c2_ipn_oracle.npz: the oracle's IPN solve (Alg. 1) of the 3D
benchmark instance -Lap u + u^3 = f on [0,1]^3 with 4x4x4 subdomains, M = 512
(n = 32,768 unknowns, m = 124,416 rows) and a Gaussian sketch of 65,536 rows,
from u_0 = 0, with the paper's solver settings (Sec. 6).  Stores the
solution's values on the evaluation grid (10 points per axis per subdomain,
64,000 points), the outer iterations, Jacobian evaluations, LSQR steps and
line-search steps per outer iteration, the final residual norm, and the wall
time of the solve with the core count and CPU model it ran on.

Calls only the oracle, in its memory-lean form (oracle.lean: block Jacobian,
column-block sketch, in-place QR; about 35 GB of host memory at the peak), and
takes one to two hours on an 8-core CPU.

    python tests/golden/make_c2_ipn_oracle.py [workers]
"""
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import rfm_workloads as W  # noqa: E402
from oracle import lean, newton  # noqa: E402
from oracle.problem import Problem  # noqa: E402


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def _timed(name, fn, t0):
    def run(*a, **k):
        t = time.time()
        out = fn(*a, **k)
        print(f"[{time.time() - t0:8.1f} s]   {name}: {time.time() - t:.1f} s", flush=True)
        return out
    return run


def main():
    workers = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    desc = W.config_c2()
    opts = W.opts_c2()
    t0 = time.time()
    op = Problem(desc)
    lean.gaussian_sketch_blocks = _timed("sketch", lean.gaussian_sketch_blocks, t0)
    lean.qr_r_lapack = _timed("qr", lean.qr_r_lapack, t0)

    def log(k, info):
        print(f"[{time.time() - t0:8.1f} s] outer {k + 1}: alpha {info.alphas[-1]:.6g} "
              f"lsqr {info.lsqr_iters[-1]} resid {info.final_resid:.6e}", flush=True)

    c, info = newton.ipn(op, opts, lean=True, workers=workers, log=log)
    wall = time.time() - t0
    X = W.eval_grid(desc)
    u = newton.evaluate(op, c, X)
    ue = op.exact(X)
    print(f"wall {wall:.1f} s, IT {info.outer_iters}, NJ {info.n_jac}, LSQR {sum(info.lsqr_iters)}, "
          f"rel-L2 vs exact {newton.rel_l2(u, ue):.3e}", flush=True)
    np.savez_compressed(os.path.join(HERE, "c2_ipn_oracle.npz"), u=u, outer_iters=info.outer_iters,
                        n_jac=info.n_jac, lsqr_iters=np.array(info.lsqr_iters), alphas=np.array(info.alphas),
                        final_resid=info.final_resid, wall_s=wall, cores=os.cpu_count() or 1,
                        workers=workers, cpu=cpu_model(), machine=platform.machine())


if __name__ == "__main__":
    main()
