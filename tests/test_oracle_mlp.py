"""Pins of the warm-start oracle (oracle/mlp.py) against facts fixed outside
it: central finite differences, the closed form of Adam's first step, and the
function-space meaning of the feature-Gram metric."""
import numpy as np
import pytest

import rfm_workloads as W
from oracle import mlp
from oracle import newton
from oracle.problem import Problem


def _net(seed=3, din=3, H=7, dout=12, B=5):
    rng = np.random.default_rng(seed)
    w = mlp.init_params(din, H, dout, seed) + 0.05 * rng.standard_normal(mlp.layout(din, H, dout)[2])
    x = rng.uniform(-1, 1, (B, din))
    t = rng.standard_normal((B, dout))
    return w, x, t, (din, H, dout)


def _spd_blocks(nb, g, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((nb, g, g))
    return np.einsum("kij,klj->kil", A, A) / g + 0.1 * np.eye(g)


@pytest.mark.parametrize("metric", ["identity", "blocks"])
def test_gradient_matches_finite_differences(metric):
    w, x, t, dims = _net()
    G, gblk = (None, 0) if metric == "identity" else (_spd_blocks(3, 4, 7), 4)
    L, g = mlp.loss_and_grad(w, x, t, *dims, G=G, gblk=gblk, quantise=False)
    off, sizes, total = mlp.layout(*dims)
    live = np.concatenate([np.arange(o, o + s) for o, s in zip(off, sizes)])
    h = 1e-6
    fd = np.zeros(total)
    for i in live:
        e = np.zeros(total)
        e[i] = h
        fd[i] = (mlp.loss_and_grad(w + e, x, t, *dims, G=G, gblk=gblk, quantise=False)[0]
                 - mlp.loss_and_grad(w - e, x, t, *dims, G=G, gblk=gblk, quantise=False)[0]) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-7 * max(1.0, np.max(np.abs(g)))
    pad = np.setdiff1d(np.arange(total), live)
    assert np.all(g[pad] == 0)


def test_loss_identity_metric_is_mean_square():
    w, x, t, dims = _net()
    _, _, y = mlp.forward(w, x, *dims, quantise=False)
    L, _ = mlp.loss_and_grad(w, x, t, *dims, quantise=False)
    assert L == pytest.approx(np.mean((y - t) ** 2) * 1.0, rel=1e-13)


def test_straight_through_gradient_close_to_exact():
    w, x, t, dims = _net(din=3, H=32, dout=64, B=16)
    _, g0 = mlp.loss_and_grad(w, x, t, *dims, quantise=False)
    _, g1 = mlp.loss_and_grad(w, x, t, *dims, quantise=True)
    assert np.linalg.norm(g1 - g0) <= 3e-2 * np.linalg.norm(g0)


def test_adam_first_step_is_signed_lr():
    rng = np.random.default_rng(1)
    w = rng.standard_normal(50)
    g = rng.standard_normal(50)
    w1, m, v = mlp.adam_step(w, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    # m_hat = g, v_hat = g^2: the step is lr * g / (|g| + eps)
    assert np.allclose(w1, w - 1e-3 * np.sign(g), rtol=0, atol=1e-3 * 1e-8 / np.min(np.abs(g)) + 1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_init_is_glorot_uniform():
    din, H, dout = 3, 256, 512
    w = mlp.init_params(din, H, dout, 11)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(w, din, H, dout)
    for Wl, fi, fo in ((W1, din, H), (W2, H, H), (W3, H, dout)):
        s = np.sqrt(6.0 / (fi + fo))
        assert np.max(np.abs(Wl)) <= s * (1 + 1e-6)
        assert np.var(Wl) == pytest.approx(s * s / 3.0, rel=0.1)
        assert np.all(Wl.astype(np.float32) == Wl)
    assert not np.any(b1) and not np.any(b2) and not np.any(b3)
    assert np.array_equal(w, mlp.init_params(din, H, dout, 11))
    assert not np.array_equal(w, mlp.init_params(din, H, dout, 12))


def test_gram_quadratic_form_is_mean_square_of_function():
    desc = W.small_2d()
    prob = Problem(desc)
    X = W.eval_grid(desc, per_axis=7)
    e = newton.owner(prob, X)
    order = np.argsort(e, kind="stable")
    Xs = X[order]
    starts = np.concatenate([[0], np.cumsum(np.bincount(e, minlength=prob.G))])
    Gm = mlp.feature_gram(prob, Xs, starts)
    r = np.random.default_rng(5).standard_normal(prob.n)
    quad = sum(r[k * prob.M:(k + 1) * prob.M] @ Gm[k] @ r[k * prob.M:(k + 1) * prob.M] for k in range(Gm.shape[0]))
    u = newton.evaluate(prob, r, X)
    assert quad == pytest.approx(np.mean(np.sum(u * u, axis=1)), rel=1e-12)


def _basis_case(N=6):
    desc = W.small_2d(M=16)
    prob = Problem(desc)
    C = np.random.default_rng(9).standard_normal((N, prob.n))
    X = W.eval_grid(desc, per_axis=6)
    return prob, C, X


def test_function_basis_diag_matches_lapack_pivoted_qr():
    import scipy.linalg as sla
    prob, C, X = _basis_case()
    mean, U, Z, diag = mlp.function_basis(prob, C, X, tol=1e-9)
    V = mlp.snapshot_values(prob, C - C.mean(axis=0), X)
    _, Rl, piv = sla.qr(V, mode="economic", pivoting=True)
    # centring leaves N - 1 independent snapshots
    assert len(diag) == C.shape[0] - 1
    assert np.allclose(diag, np.abs(np.diag(Rl))[:len(diag)], rtol=1e-10, atol=0)
    assert np.allclose(mean, C.mean(axis=0), rtol=0, atol=1e-15)


def test_function_basis_orthonormal_and_reconstructs():
    prob, C, X = _basis_case()
    mean, U, Z, _ = mlp.function_basis(prob, C, X, tol=1e-9)
    Q = mlp.snapshot_values(prob, U, X)
    assert np.allclose(Q.T @ Q, np.eye(U.shape[0]), atol=1e-10)
    resid = mlp.snapshot_values(prob, C - mean - Z @ U, X)
    scale = np.linalg.norm(mlp.snapshot_values(prob, C - mean, X), axis=0)
    assert np.all(np.linalg.norm(resid, axis=0) <= 1e-10 * scale)


def test_function_basis_detects_rank():
    # centring removes one dimension: N snapshots span at most N - 1 after
    # subtracting their mean; one snapshot built from three others removes one more
    prob, C, X = _basis_case(N=7)
    C[-1] = C[0] + C[1] - C[2]
    _, U, Z, _ = mlp.function_basis(prob, C, X, tol=1e-9)
    assert U.shape[0] == 5 and Z.shape == (7, 5)
