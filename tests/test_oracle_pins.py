"""Pins of the CPU oracle to facts outside itself: published known-answer
vectors, closed forms, finite differences, library routines, the paper's row
count formulas (Sec. 3.2) and manufactured-solution convergence (Sec. 6.1)."""
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.stats

import rfm_workloads as W
from oracle import assemble as asm
from oracle import linalg as la
from oracle import newton, philox
from oracle.problem import Problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    n = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(t, 16) for t in line.split()]
        out = philox.philox4x32_10(*w[:6])
        assert [int(o) for o in out] == w[6:]
        n += 1
    assert n == 3


def test_uniform53_range_and_resolution():
    assert philox.uniform53(0, 0) == 0.0
    top = philox.uniform53(0xFFFFFFFF, 0xFFFFFFFF)
    assert top == 1.0 - 2.0 ** -53
    x0, x1, _, _ = philox.philox4x32_10(0, np.arange(100000), 0, 0, 1, 2)
    u = philox.uniform53(x0, x1)
    assert u.min() >= 0 and u.max() < 1
    assert abs(u.mean() - 0.5) < 0.005
    assert np.all(u * 2.0 ** 53 == np.floor(u * 2.0 ** 53))


def test_round_bf16_matches_torch_on_float32_inputs():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(200000) * 4).astype(np.float32).astype(np.float64)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(philox.round_bf16(x), ref)


def test_round_bf16_ties_to_even_and_bits():
    one = 1.0
    ulp = 2.0 ** -7
    assert philox.round_bf16(np.array([one + ulp / 2]))[0] == one            # tie -> even (1.0)
    assert philox.round_bf16(np.array([one + 3 * ulp / 2]))[0] == one + 2 * ulp  # tie -> even
    assert philox.round_bf16(np.array([one + ulp / 2 + 2.0 ** -40]))[0] == one + ulp
    x = np.random.default_rng(1).standard_normal(10000)
    r = philox.round_bf16(x)
    m, e = np.frexp(r)
    assert np.all(m * 256 == np.round(m * 256))
    assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -8)


def test_features_uniform_range():
    f = philox.features(8, 1, 512, 3, 1.0, W.FEATURE_SEED)
    assert f.shape == (8, 1, 512, 4)
    assert f.min() >= -1.0 and f.max() <= 1.0
    assert abs(f.mean()) < 0.02
    # U[-1,1] variance 1/3
    assert abs(f.var() - 1.0 / 3.0) < 0.01
    ks = scipy.stats.kstest(f.reshape(-1), scipy.stats.uniform(loc=-1, scale=2).cdf)
    assert ks.pvalue > 1e-3


def test_gaussian_sketch_distribution():
    S = philox.gaussian_sketch(512, np.arange(200), 0, W.FEATURE_SEED)
    q = S * 16.0
    assert np.array_equal(q, np.rint(q)) and np.abs(q).max() <= 137   # one 8-bit digit on the 2^-4 grid
    assert np.array_equal(S, philox.round_bf16(S))                     # hence also exact in bf16
    z = S.reshape(-1)
    # rounding to 2^-4 adds variance 1/(12*256)
    assert abs(z.mean()) < 0.01 and abs(z.var() - (1.0 + 1.0 / 3072)) < 0.02
    jitter = np.random.default_rng(0).uniform(-1.0 / 32, 1.0 / 32, z.size)
    ks = scipy.stats.kstest(z + jitter, scipy.stats.norm(scale=np.sqrt(1 + 1.0 / 1536)).cdf)
    assert ks.pvalue > 1e-3
    # a fresh sketch for every Jacobian evaluation
    S1 = philox.gaussian_sketch(512, np.arange(200), 1, W.FEATURE_SEED)
    assert not np.array_equal(S, S1)


def test_count_sketch_hash_uniform():
    h, sg = philox.count_sketch_hash(300000, 1000, 0, W.FEATURE_SEED)
    assert h.min() >= 0 and h.max() < 1000
    counts = np.bincount(h, minlength=1000)
    chi = scipy.stats.chisquare(counts)
    assert chi.pvalue > 1e-4
    assert abs(sg.mean()) < 0.01 and set(np.unique(sg)) == {-1.0, 1.0}


def test_row_counts_match_paper_formulas_3d():
    # Sec. 3.2: m = Q_I + Q_b + Q_c with Q_b = 2(NxNy QxQy + NxNz QxQz + NyNz QyQz)
    # and Q_c = 2((Nx-1)NyNz QyQz + (Ny-1)NxNz QxQz + (Nz-1)NxNy QxQy).
    Nx, Ny, Nz, q, qf = 3, 2, 4, 4, 3
    p = Problem(W.problem(3, (Nx, Ny, Nz), 8, (q, q, q), (qf, qf, qf), (qf, qf, qf)))
    QI = Nx * Ny * Nz * q ** 3
    Qb = 2 * (Nx * Ny * qf * qf + Nx * Nz * qf * qf + Ny * Nz * qf * qf)
    Qc = 2 * ((Nx - 1) * Ny * Nz + (Ny - 1) * Nx * Nz + (Nz - 1) * Nx * Ny) * qf * qf
    assert (p.m_int, p.m_bdy, p.m_iface) == (QI, Qb, Qc)


def test_row_counts_benchmark_configs():
    p = Problem(W.config_c1())
    assert (p.m, p.m_int, p.m_bdy, p.m_iface, p.n) == (1920, 1600, 160, 160, 400)


def test_points_on_grid_and_faces():
    p = Problem(W.config_c1())
    # interior grid includes subdomain endpoints (Sec. 3.2: uniformly spaced including endpoints)
    Xi = p.rx[: p.m_int]
    assert np.isclose(Xi.min(), 0.0) and np.isclose(Xi.max(), 1.0)
    assert np.sum(np.isclose(Xi[:, 0], 0.5)) == 2 * 2 * 20  # both sides of the x-interface
    Xc = p.rx[p.m_int:p.m_int + p.m_iface]
    ax = p.raxis[p.m_int:p.m_int + p.m_iface]
    assert np.all(Xc[np.arange(Xc.shape[0]), ax] == 0.5)
    Xb = p.rx[p.m_int + p.m_iface:]
    onb = (Xb == 0.0) | (Xb == 1.0)
    assert np.all(onb.any(axis=1))


def _fd_feature_check(prob):
    rng = np.random.default_rng(5)
    e = rng.integers(0, prob.G, 20)
    X = prob.mu[e] + prob.sigma[e] * rng.uniform(-0.9, 0.9, (20, prob.d))
    phi, grad, lap = asm.feature_values(prob, e, X)
    h = 1e-4
    lap_fd = np.zeros_like(phi)
    for b in range(prob.d):
        dX = np.zeros_like(X); dX[:, b] = h
        pp, _, _ = asm.feature_values(prob, e, X + dX)
        pm, _, _ = asm.feature_values(prob, e, X - dX)
        g_fd = (pp - pm) / (2 * h)
        assert np.max(np.abs(g_fd - grad[..., b])) < 1e-6 * max(1, np.abs(grad).max())
        lap_fd += (pp - 2 * phi + pm) / h ** 2
    assert np.max(np.abs(lap_fd - lap)) < 1e-4 * max(1, np.abs(lap).max())
    # phi is exactly tanh(k . l(x) + b) for one feature, computed by hand
    kb = prob.feats[e[0], 0, 3]
    z = sum(kb[b] * (X[0, b] - prob.mu[e[0], b]) / prob.sigma[e[0], b] for b in range(prob.d)) + kb[prob.d]
    assert abs(math.tanh(z) - phi[0, 0, 3]) < 1e-15


def test_feature_derivatives_match_finite_differences():
    _fd_feature_check(Problem(W.small_3d()))
    _fd_feature_check(Problem(W.small_2d()))


@pytest.mark.parametrize("desc", [W.small_2d(), W.small_3d(),
                                  W.small_3d(pde_kind=2, pde_params=[3.0]),
                                  W.small_3d(pde_kind=1, fields=2, M=16),
                                  W.small_3d(pde_kind=3, pde_params=[2.0, 1.5, 2.0])])
def test_jacobian_matches_finite_differences(desc):
    p = Problem(desc)
    c = W.random_coeffs(p.n, seed=2, scale=0.3)
    F, J = asm.assemble(p, c)
    rng = np.random.default_rng(4)
    for _ in range(3):
        dv = rng.standard_normal(p.n)
        h = 1e-5
        fd = (asm.residual(p, c + h * dv) - asm.residual(p, c - h * dv)) / (2 * h)
        assert np.max(np.abs(fd - J @ dv)) < 1e-6 * np.abs(J @ dv).max()


def test_linear_rows_are_exactly_linear():
    p = Problem(W.small_3d())
    c = W.random_coeffs(p.n, seed=3)
    F, J = asm.assemble(p, c)
    lin = slice(p.m_int, p.m)
    g = np.zeros(p.m)
    g[p.m_int + p.m_iface:] = asm.residual(p, np.zeros(p.n))[p.m_int + p.m_iface:]
    assert np.allclose(F[lin], (J @ c + g)[lin], rtol=0, atol=1e-12)


def _fd_laplacian(fun, X, h=1e-3):
    out = np.zeros(X.shape[0])
    for b in range(X.shape[1]):
        dX = np.zeros_like(X); dX[:, b] = h
        out += (fun(X + dX) - 2 * fun(X) + fun(X - dX)) / h ** 2
    return out


def test_manufactured_sources_satisfy_the_pde():
    rng = np.random.default_rng(8)
    X = rng.uniform(0.1, 0.9, (50, 3))
    # kind 0: -Lap u + u^3
    p = Problem(W.small_3d())
    u = lambda Y: p.exact(Y)[:, 0]
    assert np.allclose(p.source(X, 0), -_fd_laplacian(u, X) + u(X) ** 3, atol=2e-5)
    # kind 2: -div(a grad u) + kappa u^3, by a flux-form finite difference
    p2 = Problem(W.small_3d(pde_kind=2, pde_params=[3.0]))
    a = lambda Y: 1 + 0.5 * np.sin(2 * np.pi * Y[:, 0])
    u2 = lambda Y: p2.exact(Y)[:, 0]
    h = 1e-3
    div = np.zeros(X.shape[0])
    for b in range(3):
        e = np.zeros(3); e[b] = h / 2
        E = np.zeros(3); E[b] = h
        div += (a(X + e) * (u2(X + E) - u2(X)) - a(X - e) * (u2(X) - u2(X - E))) / h ** 2
    assert np.allclose(p2.source(X, 0), -div + 3.0 * u2(X) ** 3, atol=2e-5)
    # kind 1: Gray-Scott with constant diffusion
    p3 = Problem(W.small_3d(pde_kind=1, fields=2, M=8))
    eu, ev, F, k = p3.params[:4]
    uu = lambda Y: p3.exact(Y)[:, 0]
    vv = lambda Y: p3.exact(Y)[:, 1]
    U, V = uu(X), vv(X)
    assert np.allclose(p3.source(X, 0), -eu * _fd_laplacian(uu, X) + U * V * V - F * (1 - U), atol=1e-6)
    assert np.allclose(p3.source(X, 1), -ev * _fd_laplacian(vv, X) - U * V * V + (F + k) * V, atol=1e-6)


def test_row_scaling_invariant():
    p = Problem(W.config_c1())
    c = W.random_coeffs(p.n, seed=9)
    Fs, Js, lam = asm.scaled_system(p, c)
    assert np.allclose(np.abs(Js).max(axis=1), 100.0, rtol=1e-15)


def test_count_sketch_scatter_matches_explicit_matrix():
    rng = np.random.default_rng(1)
    J = rng.standard_normal((300, 20))
    h, sg = philox.count_sketch_hash(300, 50, 3, 99)
    S = np.zeros((50, 300))
    S[h, np.arange(300)] = sg            # one +-1 per column of S_k (Sec. 4.1)
    assert np.allclose(la.count_sketch(J, 50, 3, 99), S @ J, atol=1e-13)


def _signed_r_lapack(B):
    R = np.linalg.qr(B, mode="r")
    return R * np.sign(np.diag(R))[:, None]


@pytest.mark.parametrize("shape,cond", [((60, 20), 1e2), ((90, 33), 1e10), ((7, 7), 1e3)])
def test_householder_qr_against_lapack(shape, cond):
    rng = np.random.default_rng(11)
    U, _ = np.linalg.qr(rng.standard_normal((shape[0], shape[1])))
    V, _ = np.linalg.qr(rng.standard_normal((shape[1], shape[1])))
    B = U @ np.diag(np.logspace(0, -np.log10(cond), shape[1])) @ V.T
    Ru, f1 = la.qr_r_unblocked(B)
    Rb, f2 = la.qr_r_blocked(B, nb=8)
    Rl = _signed_r_lapack(B)
    assert np.all(np.diag(Ru) > 0) and not f1 and not f2
    nrm = np.linalg.norm(B)
    assert np.linalg.norm(Ru - Rl) / nrm < 1e-13 * cond ** 0.5 + 1e-14
    assert np.linalg.norm(Rb - Ru) / nrm < 1e-14 * shape[0]
    # R^T R = B^T B (Gram matrix in extended precision)
    G = B.astype(np.longdouble).T @ B.astype(np.longdouble)
    assert float(np.abs(Ru.T.astype(np.longdouble) @ Ru - G).max()) < 1e-14 * shape[0] * nrm ** 2


def test_qr_rank_floor():
    B = np.zeros((10, 4)); B[:, :3] = np.random.default_rng(0).standard_normal((10, 3))
    R, flag = la.qr_r_unblocked(B)
    assert flag and R[3, 3] == pytest.approx(1e-14 * np.diag(R)[:3].max())


def test_triangular_solves_against_scipy():
    rng = np.random.default_rng(2)
    R = np.triu(rng.standard_normal((40, 40))) + 10 * np.eye(40)
    b = rng.standard_normal(40)
    assert np.allclose(la.solve_upper(R, b), scipy.linalg.solve_triangular(R, b), rtol=1e-13)
    assert np.allclose(la.solve_upper_t(R, b), scipy.linalg.solve_triangular(R, b, trans="T"), rtol=1e-13)


def test_lsqr_against_direct_least_squares():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((200, 30)) @ np.diag(np.linspace(1, 3, 30))
    b = rng.standard_normal(200)
    res = la.lsqr(lambda v: A @ v, lambda u: A.T @ u, b, 30, 1e-12, 1e-12, 1e8, 200)
    x = np.linalg.lstsq(A, b, rcond=None)[0]
    assert res.istop in (1, 2)
    assert np.linalg.norm(res.x - x) / np.linalg.norm(x) < 1e-9
    # consistent system: converges by S1, and in exact arithmetic within n steps
    bc = A @ rng.standard_normal(30)
    res = la.lsqr(lambda v: A @ v, lambda u: A.T @ u, bc, 30, 1e-10, 1e-10, 1e8, 200)
    assert res.istop == 1 and res.itn <= 31
    # the reported residual norm is the true one
    assert abs(res.normr - np.linalg.norm(bc - A @ res.x)) < 1e-8 * np.linalg.norm(bc)


def test_golden_section_finds_minimum_and_rejects_ascent():
    a, fa, cnt = newton.golden_section(lambda t: (t - 0.3) ** 2 + 1, 1.09)
    assert abs(a - 0.3) < 1e-3 and cnt == 18
    a, fa, _ = newton.golden_section(lambda t: 1 + t, 1.0)
    assert a == 0.0 and fa == 1.0
    a, fa, _ = newton.golden_section(lambda t: 2 - t, 2.0)
    assert a == 1.0 and fa == 1.0
    a, fa, _ = newton.golden_section(lambda t: 1.0, 2.0)       # flat: ties -> largest alpha
    assert a == 1.0


def test_preconditioned_jacobian_is_well_conditioned():
    # Sec. 4.1: kappa(J R^-1) <= sqrt((1+eps)/(1-eps)) with high probability,
    # independent of kappa(J).
    p = Problem(W.config_c1())
    c = W.random_coeffs(p.n, seed=1, scale=0.1)
    for kind in ("count", "gauss"):
        opts = W.solve_opts(sketch_kind=kind, sketch_rows=1200)
        lin = newton._Lin(p, opts, c, 0)
        sv = np.linalg.svd(lin.J, compute_uv=False)
        assert sv[0] / sv[-1] > 1e6
        P = scipy.linalg.solve_triangular(lin.R, np.eye(p.n))
        sv2 = np.linalg.svd(lin.J @ P, compute_uv=False)
        assert sv2[0] / sv2[-1] < 10.0


def test_ipn_matches_dense_gauss_newton_on_tiny_problem():
    """Same Newton loop with the LSQR step replaced by a direct dense
    least-squares solve: same iteration count, same solution."""
    p = Problem(W.small_2d(M=12, q=6))
    opts = W.solve_opts(eta=1e-12)
    c, info = newton.ipn(p, opts)
    cg = np.zeros(p.n)
    for k in range(50):
        Fs, Js, lam = asm.scaled_system(p, cg)
        d = np.linalg.lstsq(Js, -Fs, rcond=None)[0]
        f0 = np.linalg.norm(Fs)
        alpha, f1, _ = newton.golden_section(lambda a: newton.scaled_norm(p, lam, cg + a * d), f0)
        cg = cg + alpha * d
        if abs(f1 - f0) < opts["eps"]:
            break
    assert info.outer_iters == k + 1
    X = W.eval_grid(p.desc)
    assert newton.rel_l2(newton.evaluate(p, c, X), newton.evaluate(p, cg, X)) < 1e-8


def test_c1_manufactured_solution_converges():
    """2D -Lap u + u^3 = f (the 2D analogue of Sec. 6.1): IPN and AMIPN reach
    relative L2 error below 1e-6 with few outer iterations; AMIPN needs fewer
    Jacobian evaluations (Sec. 4.2)."""
    d = W.config_c1()
    p = Problem(d)
    X = W.eval_grid(d)
    ue = p.exact(X)
    c, info = newton.ipn(p, W.solve_opts())
    assert newton.rel_l2(newton.evaluate(p, c, X), ue) < 1e-6
    assert 2 <= info.outer_iters <= 8 and info.n_jac == info.outer_iters
    c2, info2 = newton.amipn(p, W.solve_opts())
    assert newton.rel_l2(newton.evaluate(p, c2, X), ue) < 1e-6
    assert info2.n_jac < info.n_jac
    assert max(info.lsqr_iters) < 100


def test_gaussian_sketch_rows_are_rows_of_the_sketch():
    """The few-rows form used at full sizes draws the same entries."""
    from oracle import philox as _ph
    rows = np.arange(40) + 777
    S = _ph.gaussian_sketch(96, rows, 2, 20251004)
    pick = np.array([0, 1, 2, 33, 95, 64])
    assert np.array_equal(_ph.gaussian_sketch_rows(pick, rows, 2, 20251004), S[pick])


def test_amipn_as_printed_keeps_a_stale_jacobian():
    """Alg. 2 recomputes the preconditioned Jacobian only when the inner loop
    runs to m_max; an early inner stop keeps it.  On a steady Gray-Scott system
    from u_0 = 0 the inner loop stops early with the Jacobian of u_0 and the
    outer test then ends the solve on that one Jacobian, well short of what
    IPN (a fresh Jacobian every step) reaches.  The GPU solver shows the same
    behaviour at full size; this records the reading."""
    from oracle import newton as _nt
    desc = W.small_3d(pde_kind=1, fields=2, M=20)
    op = Problem(desc)
    X = W.eval_grid(desc, per_axis=4)
    ue = op.exact(X)
    err = {}
    nj = {}
    for solver in ("amipn", "ipn"):
        c, info = getattr(_nt, solver)(op, W.solve_opts(m_max=5))
        u = _nt.evaluate(op, c, X)
        err[solver] = np.linalg.norm(u - ue) / np.linalg.norm(ue)
        nj[solver] = info.n_jac
    assert nj["amipn"] == 1 and nj["ipn"] > 5
    assert err["amipn"] > 2 * err["ipn"]
