"""Memory-lean forms of the oracle's linearisation for full-size instances.

The dense forms in `assemble`, `linalg` and `newton` hold J as an m x n array
and draw the Gaussian sketch S_k as one s x m array; at the 3D benchmark size
(n = 32,768, m = 124,416, s = 65,536) those alone would take 33 GB and 65 GB.
This module computes the same quantities without either array:

* J is kept in the block form that the assembly produces row by row (Alg. 3,
  Sec. 5): each row's primary block (the W = fields*M columns of subdomain
  e0) and, for interface rows, the secondary block (subdomain e1).  J x and
  J^T u are the block sums of the dense products.
* The row scale lambda_i = c / max_j |J_ij| (Sec. 5) is taken over both blocks
  of a row, as in `assemble.row_scale`.
* The sketch B = S_k J (Sec. 4.1) is formed one column block at a time:
  B[:, cols(e)] = S_k[:, rows(e)] J[rows(e), cols(e)], where rows(e) are the
  rows whose primary or secondary block is subdomain e (every other row is
  zero in those columns).  S_k's entries for those rows are drawn by the same
  definition as `philox.gaussian_sketch`, a range of sketch rows at a time,
  optionally in a pool of worker processes.  The count sketch adds
  sigma(i) J[i, :] to row h(i) of B in increasing i, as `linalg.count_sketch`.
* The Householder QR without pivoting (Sec. 4.1, R as `linalg.normalise_r`
  fixes it) is LAPACK's geqrf, the routine behind numpy.linalg.qr, in numpy's
  64-bit-index build (s * n exceeds 2^31 at full size).  This library routine
  serves as one step and computes the factorisation that
  `qr_r_blocked_inplace` writes out: `linalg.qr_r_blocked`'s algorithm in
  place, with the compact-WY trailing update done a range of columns at a
  time.  The two are pinned to each other, and geqrf to the textbook
  definition, by the oracle's tests.
* R is held in row-major and column-major copies so that both triangular
  solves of `linalg` read contiguous memory.

None of this changes what is computed; each function is checked against its
dense counterpart on small instances by the oracle's pin tests.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
import os

import numpy as np

from . import assemble as asm
from . import linalg as la
from . import philox


class BlockJacobian:
    """Row-scaled J in block form with its residual and row scales."""

    def __init__(self, prob, c, C=100.0, chunk=8192):
        m, W = prob.m, prob.W
        self.prob = prob
        self.F = np.zeros(m)
        self.Jp = np.zeros((m, W))
        self.lam = np.ones(m)
        self.e0 = prob.re0.astype(np.int64)
        self.e1 = prob.re1.astype(np.int64)
        self.sec = np.nonzero(self.e1 >= 0)[0]          # rows with a secondary block
        self.Js = np.zeros((self.sec.size, W))
        pos = np.full(m, -1, dtype=np.int64)
        pos[self.sec] = np.arange(self.sec.size)
        for s0 in range(0, m, chunk):
            rows = np.arange(s0, min(m, s0 + chunk))
            Fr, Jp, Js, e0, e1 = asm.assemble_rows(prob, c, rows)
            lam = asm.row_scale(Jp, Js, C)
            self.F[rows] = Fr
            self.lam[rows] = lam
            self.Jp[rows] = lam[:, None] * Jp
            t = np.nonzero(e1 >= 0)[0]
            if t.size:
                self.Js[pos[rows[t]]] = lam[t, None] * Js[t]
        # rows touching each column block, in increasing row order
        G = prob.G
        self.rows_of = []
        for e in range(G):
            self.rows_of.append(np.nonzero((self.e0 == e) | (self.e1 == e))[0])
        self._pos = pos

    def block_rows(self, e):
        """Rows touching subdomain e's columns and J restricted to them."""
        rows = self.rows_of[e]
        Jb = np.empty((rows.size, self.prob.W))
        prim = self.e0[rows] == e
        Jb[prim] = self.Jp[rows[prim]]
        if (~prim).any():
            Jb[~prim] = self.Js[self._pos[rows[~prim]]]
        return rows, Jb

    def matvec(self, x, chunk=8192):
        """J x."""
        W = self.prob.W
        xb = x.reshape(self.prob.G, W)
        y = np.empty(self.prob.m)
        for s0 in range(0, y.size, chunk):
            r = slice(s0, min(y.size, s0 + chunk))
            y[r] = np.einsum("rw,rw->r", self.Jp[r], xb[self.e0[r]])
        if self.sec.size:
            y[self.sec] += np.einsum("rw,rw->r", self.Js, xb[self.e1[self.sec]])
        return y

    def rmatvec(self, u):
        """J^T u."""
        out = np.zeros((self.prob.G, self.prob.W))
        for e in range(self.prob.G):
            rows, Jb = self.block_rows(e)
            out[e] = Jb.T @ u[rows]
        return out.reshape(-1)


# ------------------------------------------------------------------ sketch
def count_sketch_blocks(J, s, kJ, seed):
    """B = S_k J for the count sketch, column-major [s, n]."""
    prob = J.prob
    W = prob.W
    h, sig = philox.count_sketch_hash(prob.m, s, kJ, seed)
    B = np.zeros((s, prob.n), order="F")
    for i in range(prob.m):
        e = J.e0[i]
        B[h[i], e * W:(e + 1) * W] += sig[i] * J.Jp[i]
        if J.e1[i] >= 0:
            e = J.e1[i]
            B[h[i], e * W:(e + 1) * W] += sig[i] * J.Js[J._pos[i]]
    return B


def _gauss_task(args):
    r0, r1, rows, Jb, kJ, seed = args
    return philox.gaussian_sketch_range(r0, r1, rows, kJ, seed) @ Jb


def gaussian_sketch_blocks(J, s, kJ, seed, workers=0, rchunk=8192):
    """B = S_k J for the Gaussian sketch, column-major [s, n], one column
    block and one range of sketch rows at a time.  workers > 1 spreads the
    ranges over that many spawned processes (each with one BLAS thread)."""
    prob = J.prob
    W = prob.W
    B = np.zeros((s, prob.n), order="F")
    tasks, keys = [], []
    for e in range(prob.G):
        rows, Jb = J.block_rows(e)
        for r0 in range(0, s, rchunk):
            r1 = min(s, r0 + rchunk)
            tasks.append((r0, r1, rows, Jb, kJ, seed))
            keys.append((e, r0, r1))
    if workers and workers > 1:
        import multiprocessing as mp
        saved = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS")}
        os.environ["OPENBLAS_NUM_THREADS"] = "1"
        os.environ["OMP_NUM_THREADS"] = "1"
        try:
            with mp.get_context("spawn").Pool(workers) as pool:
                for (e, r0, r1), blk in zip(keys, pool.imap(_gauss_task, tasks, chunksize=1)):
                    B[r0:r1, e * W:(e + 1) * W] = blk
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
    else:
        for (e, r0, r1), t in zip(keys, tasks):
            B[r0:r1, e * W:(e + 1) * W] = _gauss_task(t)
    return B


# ------------------------------------------------------------------ QR
def qr_r_blocked_inplace(A, nb=64, chunk=2048):
    """linalg.qr_r_blocked on A (overwritten; column-major is fastest), the
    trailing update A[j0:, c] -= V (T^T (V^T A[j0:, c])) applied `chunk`
    columns at a time.  Returns (R, rank_flag) like linalg.normalise_r."""
    s, n = A.shape
    for j0 in range(0, n, nb):
        j1 = min(n, j0 + nb)
        w_ = j1 - j0
        V = np.zeros((s - j0, w_))
        taus = np.zeros(w_)
        for jj in range(w_):
            j = j0 + jj
            v, tau, beta = la.house(A[j:, j])
            if tau != 0.0 and j + 1 < j1:
                w = v @ A[j:, j + 1:j1]
                # tau * (v_r w_k) as in linalg.qr_r_blocked, formed column-major
                # (np.outer(w, v).T) to match A's layout
                A[j:, j + 1:j1] -= tau * np.outer(w, v).T
            A[j, j] = beta
            A[j + 1:, j] = 0.0
            V[jj:, jj] = v
            taus[jj] = tau
        if j1 < n:
            T = np.zeros((w_, w_))
            for jj in range(w_):
                T[jj, jj] = taus[jj]
                if jj:
                    T[:jj, jj] = -taus[jj] * (T[:jj, :jj] @ (V[:, :jj].T @ V[:, jj]))
            for c0 in range(j1, n, chunk):
                c1 = min(n, c0 + chunk)
                Wm = V.T @ A[j0:, c0:c1]
                A[j0:, c0:c1] -= V @ (T.T @ Wm)
    return la.normalise_r(A[:n, :n])


def qr_r_lapack(A):
    """R of the Householder QR of A (s >= n) by LAPACK geqrf, normalised
    like linalg.normalise_r; returns (R, rank_flag).  A is overwritten: the
    in-place geqrf gufunc behind numpy.linalg.qr is called directly, so the
    full-size sketch (17 GB) is not copied first; numpy.linalg.qr (which
    copies) is the fallback where that gufunc is absent."""
    s, n = A.shape
    try:
        from numpy.linalg import _umath_linalg
        raw = _umath_linalg.qr_r_raw
    except (ImportError, AttributeError):
        raw = None
    if raw is not None:
        raw(A, signature="d->d")
        R = np.triu(A[:n, :n])
    else:
        R = np.linalg.qr(A, mode="r")[:n, :n]
    return la.normalise_r(R)


class LeanLin:
    """The linearisation of `newton._Lin` (scaled J, row scale lambda,
    preconditioner R) in the lean forms above."""

    def __init__(self, prob, opts, c, kJ, workers=0, qr="lapack"):
        from . import newton
        self.Jb = BlockJacobian(prob, c, opts["row_scale_c"])
        self.lam = self.Jb.lam
        s = newton.sketch_rows(prob, opts)
        seed = prob.desc["seed"]
        if opts["sketch_kind"] == "gauss":
            B = gaussian_sketch_blocks(self.Jb, s, kJ, seed, workers)
        else:
            B = count_sketch_blocks(self.Jb, s, kJ, seed)
        R, self.rank_flag = qr_r_lapack(B) if qr == "lapack" else qr_r_blocked_inplace(B)
        del B
        self.Rc = np.ascontiguousarray(R)
        self.Rf = np.asfortranarray(R)
        del R

    def direction(self, rhs, opts, n):
        Jb, Rc, Rf = self.Jb, self.Rc, self.Rf
        mv = lambda v: Jb.matvec(la.solve_upper(Rc, v))
        rmv = lambda u: la.solve_upper_t(Rf, Jb.rmatvec(u))
        lim = opts.get("lsqr_max_iter", 0) or 2 * n
        eta = opts["eta"]
        res = la.lsqr(mv, rmv, rhs, n, eta, eta, opts.get("conlim", 1e8), lim)
        return la.solve_upper(Rc, res.x), res
