"""Pins of the oracle's memory-lean forms (block Jacobian, column-block
sketch, in-place blocked QR) against the dense forms they restate, on small
instances where both fit.  The lean forms are what the full-size 3D oracle
solve runs, so each must compute the dense quantity up to rounding order."""
import numpy as np

import rfm_workloads as W
from oracle import assemble as asm
from oracle import lean
from oracle import linalg as la
from oracle import newton, philox
from oracle.problem import Problem

U = 2.0 ** -53


def _small(kind=0, fields=1):
    return Problem(W.small_3d(M=24, q=5, qf=4, pde_kind=kind, fields=fields))


def test_block_jacobian_equals_dense():
    for kind, fields in ((0, 1), (1, 2), (2, 1)):
        p = _small(kind, fields)
        c = W.random_coeffs(p.n, seed=3, scale=0.1)
        Fs, Js, lam = asm.scaled_system(p, c)
        Jb = lean.BlockJacobian(p, c)
        assert np.array_equal(Jb.lam, lam)
        assert np.array_equal(Jb.lam * Jb.F, Fs)
        x = np.random.default_rng(1).standard_normal(p.n)
        u = np.random.default_rng(2).standard_normal(p.m)
        y = Jb.matvec(x)
        assert np.max(np.abs(y - Js @ x)) <= 4 * p.W * U * np.max(np.abs(Js) @ np.abs(x))
        z = Jb.rmatvec(u)
        assert np.max(np.abs(z - Js.T @ u)) <= 4 * p.m * U * np.max(np.abs(Js.T) @ np.abs(u))
        # the block rows reproduce J's columns exactly
        for e in (0, p.G - 1):
            rows, Jblk = Jb.block_rows(e)
            dense = Js[:, e * p.W:(e + 1) * p.W]
            assert np.array_equal(Jblk, dense[rows])
            other = np.setdiff1d(np.arange(p.m), rows)
            assert not np.any(dense[other])


def test_sketch_range_rows_are_rows_of_the_sketch():
    rows = np.arange(30) + 101
    S = philox.gaussian_sketch(64, rows, 1, 20251004)
    assert np.array_equal(philox.gaussian_sketch_range(16, 40, rows, 1, 20251004), S[16:40])


def test_lean_sketches_equal_dense():
    p = _small()
    c = W.random_coeffs(p.n, seed=4, scale=0.1)
    _, Js, _ = asm.scaled_system(p, c)
    Jb = lean.BlockJacobian(p, c)
    seed = p.desc["seed"]
    s = 2 * p.n
    Bd = la.count_sketch(Js, s, 1, seed)
    Bl = lean.count_sketch_blocks(Jb, s, 1, seed)
    assert np.array_equal(Bd, Bl)  # same terms added in the same order
    Sd = la.gaussian_sketch_matrix(s, p.m, 2, seed)
    Bd = Sd @ Js
    bound = 2 * p.m * U * (np.abs(Sd) @ np.abs(Js))
    for workers, rchunk in ((0, 128), (0, s), (2, 96)):
        Bl = lean.gaussian_sketch_blocks(Jb, s, 2, seed, workers=workers, rchunk=rchunk)
        assert np.all(np.abs(Bl - Bd) <= bound)


def test_inplace_blocked_qr_equals_blocked_qr():
    rng = np.random.default_rng(6)
    B = rng.standard_normal((300, 150)) @ np.diag(np.logspace(0, 6, 150))
    R1, f1 = la.qr_r_blocked(B, nb=16)
    A = np.asfortranarray(B.copy())
    R2, f2 = lean.qr_r_blocked_inplace(A, nb=16, chunk=40)
    assert f1 == f2
    assert np.max(np.abs(R1 - R2)) <= 1e-13 * np.abs(R1).max()
    # and the Gram identity of the factorisation
    G = B.T @ B
    assert np.max(np.abs(R2.T @ R2 - G)) <= 1e-12 * np.abs(G).max()


def test_lapack_qr_equals_blocked_qr():
    """geqrf (the full-size oracle's QR) and the written-out blocked
    Householder QR give the same normalised R within the FP64 bound, the same
    rank flag, and R^T R = B^T B; a rank-deficient B sets the flag on both."""
    rng = np.random.default_rng(7)
    B = rng.standard_normal((300, 150)) @ np.diag(np.logspace(0, 6, 150))
    R1, f1 = lean.qr_r_blocked_inplace(np.asfortranarray(B.copy()), nb=16, chunk=40)
    R2, f2 = lean.qr_r_lapack(np.asfortranarray(B.copy()))
    assert f1 == f2 and not f2
    assert np.all(np.diag(R2) > 0) and np.array_equal(R2, np.triu(R2))
    assert np.max(np.abs(R1 - R2)) <= 1e-13 * np.abs(R1).max()
    G = B.T @ B
    assert np.max(np.abs(R2.T @ R2 - G)) <= 1e-12 * np.abs(G).max()
    D = B.copy()
    D[:, 7] = D[:, 3]
    _, fd1 = lean.qr_r_blocked_inplace(np.asfortranarray(D.copy()), nb=16, chunk=40)
    _, fd2 = lean.qr_r_lapack(np.asfortranarray(D.copy()))
    assert fd1 and fd2


def test_lean_solves_equal_dense_solves():
    for kind, sk, solver in ((0, "gauss", "ipn"), (0, "count", "amipn"), (1, "count", "ipn")):
        p = _small(kind, 2 if kind == 1 else 1)
        opts = W.solve_opts(sketch_kind=sk, max_outer=6)
        c1, i1 = getattr(newton, solver)(p, opts)
        c2, i2 = getattr(newton, solver)(p, opts, lean=True)
        assert (i1.outer_iters, i1.n_jac, i1.lsqr_iters) == (i2.outer_iters, i2.n_jac, i2.lsqr_iters)
        X = W.eval_grid(p.desc, per_axis=4)
        assert newton.rel_l2(newton.evaluate(p, c2, X), newton.evaluate(p, c1, X)) < 1e-10
