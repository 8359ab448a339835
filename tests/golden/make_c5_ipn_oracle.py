"""Writes c5_ipn_oracle.npz: the oracle's IPN solve (Alg. 1) of one instance
of the C5 family at its full size (2x2x2 subdomains, M = 512, n = 4,096,
count sketch gamma = 3), with kappa = 3, A = 1.2, q = 2, and the solution's
values on the evaluation grid (10 points per axis per subdomain).  Calls only
the oracle; takes a few minutes on a CPU.

    python tests/golden/make_c5_ipn_oracle.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import rfm_workloads as W  # noqa: E402
from oracle import newton  # noqa: E402
from oracle.problem import Problem  # noqa: E402

PARAMS = (3.0, 1.2, 2.0)


def main():
    desc = W.config_c5(*PARAMS)
    op = Problem(desc)
    c, info = newton.ipn(op, W.solve_opts())
    X = W.eval_grid(desc)
    u = newton.evaluate(op, c, X)
    np.savez_compressed(os.path.join(HERE, "c5_ipn_oracle.npz"), params=np.array(PARAMS), u=u,
                        outer_iters=info.outer_iters, n_jac=info.n_jac, lsqr_iters=np.array(info.lsqr_iters),
                        final_resid=info.final_resid)


if __name__ == "__main__":
    main()
