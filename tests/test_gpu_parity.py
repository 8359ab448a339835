"""GPU-vs-oracle parity of every hot-path step, called through the C ABI.

Tolerances (floating point, FP64 on both sides):
  * features, points, count-sketch buckets: bit-exact;
  * J and F entries: |gpu - oracle| <= 1e-12 * max_j |J_ij| per row (the rows
    are scaled to max 100, so 1e-10 absolute);
  * sketch, QR, triangular solves, LSQR: bounds from the FP64 error analysis
    of each operation (stated per test);
  * solves: equal IT and NJ, relative L2 distance of u at evaluation points
    <= 1e-7.
"""
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


CASES = {
    "2d_small": W.small_2d(),
    "2d_c1": W.config_c1(),
    "3d_small": W.small_3d(),
    "3d_ragged": W.small_3d(M=37, nsub=(3, 2, 2), q=4, qf=3),
    "3d_kind2": W.small_3d(pde_kind=2, pde_params=[3.0]),
    "3d_kind3": W.small_3d(pde_kind=3, pde_params=[2.0, 1.5, 2.0]),
    "3d_grayscott": W.small_3d(pde_kind=1, fields=2, M=20),
    "3d_helmholtz": W.small_3d(pde_kind=4, M=20),
    "3d_quasilinear": W.small_3d(pde_kind=5, M=20),
    "3d_strongly_nonlinear": W.small_3d(pde_kind=6, M=20),
    "3d_ball": W.ball(20, 7, 300),
}


@pytest.mark.parametrize("name", list(CASES))
def test_features_and_points_bit_exact(name):
    desc = CASES[name]
    op = OProblem(desc)
    gp = G().Problem(desc)
    assert (gp.m, gp.n, gp.m_int, gp.m_iface) == (op.m, op.n, op.m_int, op.m_iface)
    f = host(gp.rfm_get_features()).reshape(op.G, op.fields, op.M, 4)
    assert np.array_equal(f[..., : op.d + 1], op.feats)
    pts = host(gp.rfm_get_points())[:, : op.d]
    assert np.array_equal(pts, op.rx)


@pytest.mark.parametrize("name", list(CASES))
def test_assembly_matches_oracle(name):
    desc = CASES[name]
    op = OProblem(desc)
    gp = G().Problem(desc)
    c = W.random_coeffs(op.n, seed=3, scale=0.5)
    F, lam = gp.rfm_assemble(dev(c))
    Jp, Js, blk = gp.rfm_get_jacobian()
    Fo, Jpo, Jso, e0, e1 = asm.assemble_rows(op, c, np.arange(op.m))
    lamo = asm.row_scale(Jpo, Jso)
    blk = host(blk)
    assert np.array_equal(blk[:, 0], e0) and np.array_equal(blk[:, 1], e1)
    lam = host(lam)
    assert np.allclose(lam, lamo, rtol=1e-12, atol=0)
    Jp, Js = host(Jp), host(Js)
    tol = 1e-12 * 100.0
    assert np.max(np.abs(Jp - lamo[:, None] * Jpo)) <= tol
    if op.m_iface:
        sl = slice(op.m_int, op.m_int + op.m_iface)
        assert np.max(np.abs(Js - (lamo[:, None] * Jso)[sl])) <= tol
    Fs = lamo * Fo
    assert np.max(np.abs(host(F) - Fs)) <= 1e-12 * max(1.0, np.abs(Fs).max())
    # residual-only path with the stored scales
    Fr, nrm = gp.rfm_residual(dev(c))
    assert np.max(np.abs(host(Fr) - Fs)) <= 1e-12 * max(1.0, np.abs(Fs).max())
    assert abs(nrm - np.linalg.norm(Fs)) <= 1e-12 * np.linalg.norm(Fs)


def _dense(op, gp, c):
    F, lam = gp.rfm_assemble(dev(c))
    Fo, Jo = asm.assemble(op, c)
    lamo = host(lam)
    return lamo[:, None] * Jo


@pytest.mark.parametrize("name", ["2d_c1", "3d_ragged", "3d_grayscott"])
def test_jacobian_matvecs(name):
    desc = CASES[name]
    op = OProblem(desc)
    gp = G().Problem(desc)
    J = _dense(op, gp, W.random_coeffs(op.n, seed=4, scale=0.5))
    x = W.random_coeffs(op.n, seed=5)
    y = W.random_coeffs(op.m, seed=6)
    bound = lambda A, v: 1e-14 * 64 * (np.abs(A) @ np.abs(v)).max()
    assert np.max(np.abs(host(gp.rfm_jmv(dev(x), 0)) - J @ x)) <= bound(J, x)
    assert np.max(np.abs(host(gp.rfm_jmv(dev(y), 1)) - J.T @ y)) <= bound(J.T, y)


@pytest.mark.parametrize("name", ["2d_c1", "3d_ragged", "3d_grayscott"])
def test_count_sketch(name):
    desc = CASES[name]
    op = OProblem(desc)
    gp = G().Problem(desc)
    J = _dense(op, gp, W.random_coeffs(op.n, seed=4, scale=0.5))
    s = 3 * op.n + 5
    B = host(gp.rfm_sketch("count", s, 2)).T
    Bo = la.count_sketch(J, s, 2, desc["seed"])
    assert np.max(np.abs(B - Bo)) <= 1e-12 * 100 * 4


@pytest.mark.parametrize("name", ["2d_c1", "3d_ragged"])
def test_gaussian_sketch(name):
    desc = CASES[name]
    op = OProblem(desc)
    gp = G().Problem(desc)
    J = _dense(op, gp, W.random_coeffs(op.n, seed=4, scale=0.5))
    s = 2 * op.n + 130
    s += s % 2
    B = host(gp.rfm_sketch("gauss", s, 1)).T
    S = philox.gaussian_sketch(s, np.arange(op.m), 1, desc["seed"])
    Bo = S @ J
    # FP64 GEMM bound: K u |S||J|
    bound = 2.3e-16 * op.m * (np.abs(S) @ np.abs(J))
    assert np.all(np.abs(B - Bo) <= bound + 1e-300)


def _test_matrix(s, n, cond, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((s, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return U @ np.diag(np.logspace(0, -np.log10(cond), n)) @ V.T


@pytest.mark.parametrize("s,n,cond", [(100, 40, 1e3), (300, 97, 1e8), (1000, 300, 1e12), (257, 257, 1e4),
                                      (4100, 130, 1e6)])
def test_householder_r_matches_oracle(s, n, cond):
    B = _test_matrix(s, n, cond, seed=n)
    A = dev(B.T.copy())  # (n, s) row-major == s x n column-major
    R, flag = G().rfm_householder_r(A, s, n)
    R = host(R).T
    Ro, flo = la.qr_r_blocked(B, nb=32)
    assert not flag and not flo
    assert np.all(np.diag(R) > 0)
    nrm = np.linalg.norm(B)
    # both backward stable: agreement of R to ~u * cond(B) relative (perturbation bound of R)
    assert np.linalg.norm(R - Ro) / nrm <= 1e-15 * cond * np.sqrt(n) + 1e-13
    # R^T R reproduces the Gram matrix to FP64 backward error
    G_ = B.T @ B
    assert np.abs(R.T @ R - G_).max() <= 1e-14 * s * nrm ** 2


def test_qr_rank_floor_flag():
    B = np.zeros((64, 20))
    B[:, :15] = np.random.default_rng(1).standard_normal((64, 15))
    R, flag = G().rfm_householder_r(dev(B.T.copy()), 64, 20)
    assert flag
    R = host(R).T
    assert np.all(np.diag(R)[15:] == pytest.approx(1e-14 * np.diag(R)[:15].max()))


def _with_oracle_r(name, kind="count"):
    desc = CASES[name]
    op = OProblem(desc)
    gp = G().Problem(desc)
    c = W.random_coeffs(op.n, seed=9, scale=0.3)
    J = _dense(op, gp, c)
    s = 3 * op.n
    B = la.count_sketch(J, s, 0, desc["seed"])
    R, _ = la.qr_r_blocked(B)
    gp.rfm_set_r(dev(R.T.copy()))
    return op, gp, J, R, c


@pytest.mark.parametrize("name", ["2d_c1", "3d_ragged"])
def test_triangular_solves(name):
    op, gp, J, R, c = _with_oracle_r(name)
    b = W.random_coeffs(op.n, seed=10)
    x = host(gp.rfm_trsv(dev(b), 0))
    xo = la.solve_upper(R, b)
    cond = np.linalg.cond(R)
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-15 * cond * op.n
    z = host(gp.rfm_trsv(dev(b), 1))
    zo = la.solve_upper_t(R, b)
    assert np.linalg.norm(z - zo) / np.linalg.norm(zo) <= 1e-15 * cond * op.n


@pytest.mark.parametrize("name", ["2d_c1", "3d_ragged"])
def test_lsqr_direction(name):
    op, gp, J, R, c = _with_oracle_r(name)
    b = -host(gp.rfm_assemble(dev(c))[0])
    gp.rfm_set_r(dev(R.T.copy()))
    d, itn, istop = gp.rfm_lsqr(dev(b), eta=1e-6)
    mv = lambda v: J @ la.solve_upper(R, v)
    rmv = lambda u: la.solve_upper_t(R, J.T @ u)
    res = la.lsqr(mv, rmv, b, op.n, 1e-6, 1e-6, 1e8, 2 * op.n)
    do = la.solve_upper(R, res.x)
    assert itn == res.itn and istop == res.istop
    # The direction only has to agree well below the inner tolerance eta = 1e-6
    # (Alg. 1 step 3): rounding differences of the two FP64 implementations,
    # amplified by kappa(R) (~1e10 for C1) in the R solves and over the Krylov
    # steps, must stay 10x below eta in the J-norm.
    assert np.linalg.norm(J @ (host(d) - do)) <= 1e-7 * np.linalg.norm(J @ do)


@pytest.mark.parametrize("name", ["2d_c1", "3d_small", "3d_grayscott", "3d_helmholtz", "3d_quasilinear",
                                  "3d_strongly_nonlinear", "3d_ball"])
def test_linesearch(name):
    desc = CASES[name]
    op = OProblem(desc)
    gp = G().Problem(desc)
    c = W.random_coeffs(op.n, seed=12, scale=0.1)
    d = W.random_coeffs(op.n, seed=13, scale=0.05)
    F, lam = gp.rfm_assemble(dev(c))
    lamo = host(lam)
    f0 = float(np.linalg.norm(host(F)))
    a, fb = gp.rfm_linesearch(dev(c), dev(d), f0)
    ao, fo, _ = newton.golden_section(lambda t: newton.scaled_norm(op, lamo, c + t * d), f0)
    assert a == ao
    assert abs(fb - fo) <= 1e-12 * fo


def test_eval_matches_oracle():
    for name in ("2d_c1", "3d_ragged", "3d_grayscott"):
        desc = CASES[name]
        op = OProblem(desc)
        gp = G().Problem(desc)
        c = W.random_coeffs(op.n, seed=14)
        X = W.random_points(desc, 3000, seed=15)
        u = host(gp.rfm_eval(dev(c), dev(X)))
        uo = newton.evaluate(op, c, X)
        assert np.max(np.abs(u - uo)) <= 1e-13 * np.abs(c).sum() / op.G
    empty = gp.rfm_eval(dev(c), torch.zeros(0, 3, dtype=torch.float64, device="cuda"))
    assert empty.shape[0] == 0


@pytest.mark.parametrize("solver", ["ipn", "amipn"])
def test_c1_solve_parity(solver):
    desc = W.config_c1()
    op = OProblem(desc)
    gp = G().Problem(desc)
    opts = W.solve_opts()
    c, info = getattr(gp, f"rfm_{solver}_solve")(opts)
    co, info_o = getattr(newton, solver)(op, opts)
    assert info["status"] == 0
    assert info["outer_iters"] == info_o.outer_iters and info["n_jac"] == info_o.n_jac
    X = W.eval_grid(desc)
    u = host(gp.rfm_eval(c, dev(X)))
    uo = newton.evaluate(op, co, X)
    assert newton.rel_l2(u, uo) <= 1e-7
    assert newton.rel_l2(u[:, 0], op.exact(X)[:, 0]) <= 1e-6


def test_invalid_descriptions_are_rejected():
    rfm = G()
    bad = W.with_(W.small_2d(), M=0)
    with pytest.raises(rfm.RfmError) as e:
        rfm.Problem(bad)
    assert e.value.status == rfm.RFM_EINVAL
    with pytest.raises(rfm.RfmError):
        rfm.Problem(W.with_(W.small_3d(), fields=2))   # two fields only for Gray-Scott
    with pytest.raises(rfm.RfmError):
        rfm.Problem(W.small_2d(pde_kind=5))            # kinds 4-7 are three-dimensional
    with pytest.raises(rfm.RfmError):
        rfm.Problem(W.small_3d(pde_kind=8, pde_params=[0.0]))


def test_set_rhs_replaces_source_and_boundary_data():
    """rfm_set_rhs: the residual with data f + delta (interior) and g + delta
    (boundary) is the manufactured-data residual minus lambda * delta; the
    interface rows keep zero data."""
    desc = CASES["3d_ragged"]
    op = OProblem(desc)
    gp = G().Problem(desc)
    c = W.random_coeffs(op.n, seed=3, scale=0.5)
    F, lam = gp.rfm_assemble(dev(c))
    Fo = asm.residual(op, c)
    rhs0 = np.zeros(op.m)
    rhs0[: op.m_int] = op.source(op.rx[: op.m_int], 0)
    rhs0[op.m_int + op.m_iface:] = op.boundary_data(op.rx[op.m_int + op.m_iface:], 0)
    delta = np.random.default_rng(21).standard_normal(op.m)
    gp.rfm_set_rhs(dev(rhs0 + delta))
    Fr, _ = gp.rfm_residual(dev(c))
    lamo = host(lam)
    expect = lamo * Fo - lamo * delta
    expect[op.m_int:op.m_int + op.m_iface] = lamo[op.m_int:op.m_int + op.m_iface] * Fo[op.m_int:op.m_int + op.m_iface]
    assert np.max(np.abs(host(Fr) - expect)) <= 1e-12 * max(1.0, np.abs(expect).max())
