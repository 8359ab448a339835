"""Timing model of the oracle for instances too large to solve whole on the
host within a benchmark run.

Each oracle step is timed on a bounded sample at the instance's sizes and
scaled by its operation count: assembly per row, Gaussian sketch per column
block (count sketch per row), the Householder QR at the flop rate (2 n^2
(s - n/3)) of the oracle's own QR routine on an s x 1024 sample, triangular
solves per n^2, block products per nonzero, and about 19
residual evaluations per line search; the iteration counts of a solve
complete the model.  A whole oracle solve measured on one machine calibrates
the model there (tests/golden/make_c2_ipn_oracle.py measures the solve and
tests/golden/calibrate_c2_oracle_model.py stores the ratio).

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
import math
import os
import time

import numpy as np

from . import assemble as asm
from . import lean
from . import linalg as la
from . import philox
from .problem import Problem


def threads():
    """BLAS threads the oracle's products use (the host's cores when the
    thread pools cannot be inspected)."""
    try:
        from threadpoolctl import threadpool_info
        return max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        return os.cpu_count()


def projection(desc, opts, outer_iters, lsqr_iters, qr_cols=1024):
    """Projected seconds of one oracle solve of `desc` with solver options
    `opts`, `outer_iters` Jacobian evaluations and `lsqr_iters` LSQR steps in
    total.  Returns (seconds per solve, sample description, seconds spent
    sampling)."""
    t_all = time.perf_counter()
    op = Problem(desc)
    n, m, W_ = op.n, op.m, op.W
    s = opts["sketch_rows"] or int(math.ceil(opts["gamma"] * n))
    c = np.zeros(n)
    rng = np.random.default_rng(0)
    # assembly of F and J: 2048 sampled rows
    rows = np.sort(rng.choice(m, min(2048, m), replace=False))
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
    # Householder QR: the oracle's routine (LAPACK geqrf, lean.qr_r_lapack) on
    # an s x qr_cols sample, scaled by the flop count 2 n^2 (s - n/3)
    qc = min(qr_cols, n)
    B = np.asfortranarray(rng.standard_normal((s, qc)))
    t0 = time.perf_counter()
    lean.qr_r_lapack(B)
    rate = 2.0 * qc * qc * (s - qc / 3.0) / (time.perf_counter() - t0)
    del B
    t_qr = 2.0 * n * n * (s - n / 3.0) / rate
    # triangular solve (n^2) and block product J x (nnz) per LSQR iteration
    nt = min(8192, n)
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
    sample = (f"oracle steps timed on samples and scaled by operation counts: assembly of {rows.size} rows, "
              f"{sk}, Householder QR of {s}x{qc}, "
              f"R solve n={nt}, 4096-row block product; {outer_iters} outer and {lsqr_iters} LSQR iterations")
    return per_solve, sample, time.perf_counter() - t_all
