"""Parity of the tensor-core (emulated FP64) paths with the FP64 oracle:
precision 1 = Gaussian sketch S J on the bf16 tensor cores, precision 2 =
also the QR trailing update.  Tolerances are those of the FP64 paths."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import rfm_workloads as W  # noqa: E402
from oracle import assemble as asm  # noqa: E402
from oracle import linalg as la  # noqa: E402
from oracle import newton, philox  # noqa: E402
from oracle.problem import Problem as OProblem  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_04170_gb300 import build
    build.build()


def G():
    from paper_2510_04170_gb300 import rfm
    return rfm


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


RAGGED = W.small_3d(M=37, nsub=(3, 2, 2), q=4, qf=3)   # n = 444: four 128-column blocks, the last ragged


def _system(desc, seed=4):
    op = OProblem(desc)
    gp = G().Problem(desc)
    c = W.random_coeffs(op.n, seed=seed, scale=0.5)
    F, lam = gp.rfm_assemble(dev(c))
    Fo, Jo = asm.assemble(op, c)
    return op, gp, host(lam)[:, None] * Jo


@pytest.mark.parametrize("desc", [W.config_c1(), RAGGED])
def test_tensor_core_gaussian_sketch(desc):
    op, gp, J = _system(desc)
    s = 2 * op.n + 130
    s += s % 2
    gp.rfm_set_precision(1)
    B = host(gp.rfm_sketch("gauss", s, 3)).T
    S = philox.gaussian_sketch(s, np.arange(op.m), 3, desc["seed"])
    Bo = S @ J
    bound = 2.3e-16 * op.m * (np.abs(S) @ np.abs(J))
    assert np.all(np.abs(B - Bo) <= bound)


@pytest.mark.parametrize("kind", ["count", "gauss"])
def test_tensor_core_qr(kind):
    op, gp, J = _system(RAGGED)
    s = 3 * op.n
    gp.rfm_set_precision(2)
    B = host(gp.rfm_sketch(kind, s, 1)).T
    R, flag = gp.rfm_qr()
    R = host(R).T
    Ro, _ = la.qr_r_blocked(B)
    assert np.all(np.diag(R) > 0)
    cond = np.linalg.cond(Ro)
    nrm = np.linalg.norm(B)
    assert np.linalg.norm(R - Ro) / nrm <= 1e-15 * cond * np.sqrt(op.n) + 1e-13
    assert np.abs(R.T @ R - B.T @ B).max() <= 1e-14 * s * nrm ** 2


@pytest.mark.parametrize("precision", [1, 2])
def test_tensor_core_solve_parity(precision):
    desc = W.small_3d(M=40, nsub=(2, 2, 2), q=6, qf=5)
    opts = W.solve_opts(sketch_kind="gauss", sketch_rows=2 * 320 + 64, precision=precision)
    op = OProblem(desc)
    gp = G().Problem(desc)
    c, info = gp.rfm_ipn_solve(opts)
    co, info_o = newton.ipn(op, opts)
    assert info["status"] == 0
    assert info["outer_iters"] == info_o.outer_iters and info["n_jac"] == info_o.n_jac
    X = W.eval_grid(desc)
    u = host(gp.rfm_eval(c, dev(X)))
    assert newton.rel_l2(u, newton.evaluate(op, co, X)) <= 1e-7


def test_tensor_core_c1_amipn_parity():
    desc = W.config_c1()
    opts = W.solve_opts(precision=2)
    op = OProblem(desc)
    gp = G().Problem(desc)
    c, info = gp.rfm_amipn_solve(opts)
    co, info_o = newton.amipn(op, opts)
    assert info["outer_iters"] == info_o.outer_iters and info["n_jac"] == info_o.n_jac
    X = W.eval_grid(desc)
    u = host(gp.rfm_eval(c, dev(X)))
    assert newton.rel_l2(u, newton.evaluate(op, co, X)) <= 1e-7


def _matrix(s, n, cond, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((s, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return U @ np.diag(np.logspace(0, -np.log10(cond), n)) @ V.T


@pytest.mark.parametrize("s,n,cond", [(300, 97, 1e8), (1000, 300, 1e12), (2000, 640, 1e6), (257, 257, 1e4)])
def test_tensor_core_householder_matches_oracle(s, n, cond):
    B = _matrix(s, n, cond, seed=n + 1)
    R, flag = G().rfm_householder_r_tc(dev(B.T.copy()), s, n)
    R = host(R).T
    Ro, _ = la.qr_r_blocked(B, nb=32)
    assert not flag and np.all(np.diag(R) > 0)
    nrm = np.linalg.norm(B)
    assert np.linalg.norm(R - Ro) / nrm <= 1e-15 * cond * np.sqrt(n) + 1e-13
    assert np.abs(R.T @ R - B.T @ B).max() <= 1e-14 * s * nrm ** 2
