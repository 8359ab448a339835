"""Writes ball_oracle.npz: the oracle's AMIPN (Alg. 2, m_max = 3) and IPN
(Alg. 1) solves of the diffusion-reaction equation on the unit ball of Sec.
6.2, -div((1 + u^2) grad u) + u^3 - u + e^u = f with u* = |x|^2 prod sin(pi
x_d): the cube [-1,1]^3 in 2x2x2 subdomains, M = 100 features per subdomain
(n = 800), 10^3 grid points per subdomain and 10 x 10 per interface (those
inside the ball kept), 2,000 Dirichlet points on the sphere by the Fibonacci
spiral, count sketch gamma = 3, from u_0 = 0.  Stores, per solver, u at 2,000
seeded points inside the ball, the outer iterations, Jacobian evaluations
and LSQR steps.  Calls only the oracle; about a minute on a CPU.

    python tests/golden/make_ball_oracle.py
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
    desc = W.ball(100, 10, 2000)
    op = Problem(desc)
    X = W.ball_points(2000, seed=5)
    out = {"X": X}
    for solver in ("amipn", "ipn"):
        c, info = getattr(newton, solver)(op, W.solve_opts())
        out[f"{solver}_u"] = newton.evaluate(op, c, X)
        out[f"{solver}_outer_iters"] = info.outer_iters
        out[f"{solver}_n_jac"] = info.n_jac
        out[f"{solver}_lsqr_iters"] = np.array(info.lsqr_iters)
        print(solver, info.outer_iters, info.n_jac, info.lsqr_iters,
              newton.rel_l2(out[f"{solver}_u"], op.exact(X)), flush=True)
    np.savez_compressed(os.path.join(HERE, "ball_oracle.npz"), **out)


if __name__ == "__main__":
    main()
