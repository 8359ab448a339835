"""Writes grayscott_oracle.npz: the oracle's IPN (Alg. 1) and AMIPN (Alg. 2,
inner cap m_max = 5) solves of a steady Gray-Scott system (two fields, the
equations of the 3D Gray-Scott benchmark with constant diffusion eps_u =
2e-3, eps_v = 1e-3, F = 0.04, k = 0.06 and the paper's manufactured u, v of
Sec. 6.2) on [0,1]^3 with 2x2x2 subdomains, M = 64 features per field
(n = 1,024), 12^3 interior points and 6x6 points per face, count sketch
gamma = 3, from u_0 = 0.  Stores, per solver, both fields on the evaluation
grid (10 points per axis per subdomain), the outer iterations, Jacobian
evaluations and LSQR steps.  Calls only the oracle; a few minutes on a CPU.

    python tests/golden/make_grayscott_oracle.py
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
    desc = W.grayscott_small()
    op = Problem(desc)
    X = W.eval_grid(desc)
    out = {}
    for solver in ("ipn", "amipn"):
        c, info = getattr(newton, solver)(op, W.solve_opts(m_max=5))
        out[f"{solver}_u"] = newton.evaluate(op, c, X)
        out[f"{solver}_outer_iters"] = info.outer_iters
        out[f"{solver}_n_jac"] = info.n_jac
        out[f"{solver}_lsqr_iters"] = np.array(info.lsqr_iters)
        out[f"{solver}_final_resid"] = info.final_resid
        print(solver, info.outer_iters, info.n_jac, info.lsqr_iters, info.final_resid, flush=True)
    np.savez_compressed(os.path.join(HERE, "grayscott_oracle.npz"), **out)


if __name__ == "__main__":
    main()
