"""Writes operators_oracle.npz: the oracle's IPN (Alg. 1) and AMIPN (Alg. 2,
m_max = 3) solves of the three further 3D operators of the paper on [0,1]^3
with 2x2x2 subdomains, M = 100 features per subdomain (n = 800), 8^3 interior
points and 8 x 8 points per face, count sketch gamma = 3, from u_0 = 0:
  kind 4  Lap u - 100 u + 10 cosh(u) = f      (Sec. 6.2, nonlinear Helmholtz)
  kind 5  -div((1 + u^2) grad u) = f          (Sec. 3.2 benchmark)
  kind 6  -div((1 + |grad u|^2) grad u) = f   (Sec. 6.2, strongly nonlinear)
Stores, per kind and solver, u on the evaluation grid (4 points per axis per
subdomain), the outer iterations, Jacobian evaluations and LSQR steps.  Calls
only the oracle; a few minutes on a CPU.

    python tests/golden/make_operators_oracle.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import rfm_workloads as W  # noqa: E402
from oracle import newton  # noqa: E402
from oracle.problem import Problem  # noqa: E402


def main():
    out = {}
    for kind in (4, 5, 6):
        desc = W.operator_small(kind)
        op = Problem(desc)
        X = W.eval_grid(desc, per_axis=4)
        for solver in ("ipn", "amipn"):
            c, info = getattr(newton, solver)(op, W.solve_opts())
            key = f"k{kind}_{solver}"
            out[key + "_u"] = newton.evaluate(op, c, X)
            out[key + "_outer_iters"] = info.outer_iters
            out[key + "_n_jac"] = info.n_jac
            out[key + "_lsqr_iters"] = np.array(info.lsqr_iters)
            print(key, info.outer_iters, info.n_jac, info.lsqr_iters,
                  newton.rel_l2(out[key + "_u"], op.exact(X)), flush=True)
    np.savez_compressed(os.path.join(HERE, "operators_oracle.npz"), **out)


if __name__ == "__main__":
    main()
