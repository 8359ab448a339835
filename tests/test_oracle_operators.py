"""Pins of the oracle's further operators of the paper (Sec. 3.2 and Sec.
6.2): the nonlinear Helmholtz equation Lap u - 100 u + 10 cosh u = f (kind
4), the quasi-linear -div((1 + u^2) grad u) = f (kind 5), the strongly
nonlinear -div((1 + |grad u|^2) grad u) = f (kind 6) and the unit-ball
diffusion-reaction -div((1 + u^2) grad u) + u^3 - u + e^u = f (kind 7), with
the unit-ball geometry (masked grids, Fibonacci boundary points).

Each closed form is checked against something it does not share code with:
the Jacobian against central differences of the residual, the manufactured
sources against finite differences of the manufactured solution in flux
(divergence) form, the hand-written gradients and Hessians of the
manufactured solutions and of the features against finite differences, and
boundary rows against the exact solution."""
import numpy as np
import pytest

import rfm_workloads as W
from oracle import assemble as asm
from oracle.problem import Problem

KINDS = (4, 5, 6, 7)


@pytest.mark.parametrize("kind", KINDS)
def test_jacobian_matches_finite_differences(kind):
    p = Problem(W.small_3d(pde_kind=kind, M=20))
    c = W.random_coeffs(p.n, seed=2, scale=0.3)
    F, J = asm.assemble(p, c)
    rng = np.random.default_rng(4)
    for _ in range(3):
        dv = rng.standard_normal(p.n)
        h = 1e-5
        fd = (asm.residual(p, c + h * dv) - asm.residual(p, c - h * dv)) / (2 * h)
        assert np.max(np.abs(fd - J @ dv)) < 1e-6 * np.abs(J @ dv).max()


def test_feature_hessian_matches_finite_differences():
    p = Problem(W.small_3d(M=12))
    rng = np.random.default_rng(5)
    e = rng.integers(0, p.G, 10)
    X = p.mu[e] + p.sigma[e] * rng.uniform(-0.9, 0.9, (10, 3))
    H = asm.feature_hessian(p, e, X)
    h = 1e-5
    for b in range(3):
        dX = np.zeros_like(X)
        dX[:, b] = h
        gp = asm.feature_values(p, e, X + dX)[1]
        gm = asm.feature_values(p, e, X - dX)[1]
        fd = (gp - gm) / (2 * h)  # d/dx_b of grad phi: column b of the Hessian
        assert np.max(np.abs(fd - H[..., :, b])) < 1e-7 * max(1.0, np.abs(H).max())
    # the trace is the Laplacian of feature_values
    lap = asm.feature_values(p, e, X)[2]
    assert np.allclose(np.trace(H, axis1=-2, axis2=-1), lap, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("kind", KINDS)
def test_exact_jet_matches_finite_differences(kind):
    p = Problem(W.small_3d(pde_kind=kind, M=8))
    X = np.random.default_rng(6).uniform(0.05, 0.95, (40, 3))
    u, g, H = p.exact_jet(X)
    assert np.array_equal(p.exact(X)[:, 0], u)
    h = 1e-5
    for b in range(3):
        dX = np.zeros_like(X)
        dX[:, b] = h
        up, gp, _ = p.exact_jet(X + dX)
        um, gm, _ = p.exact_jet(X - dX)
        assert np.max(np.abs((up - um) / (2 * h) - g[:, b])) < 1e-8 * max(1.0, np.abs(g).max())
        assert np.max(np.abs((gp - gm) / (2 * h) - H[:, :, b])) < 1e-7 * max(1.0, np.abs(H).max())
    assert np.allclose(H, np.swapaxes(H, 1, 2), rtol=0, atol=1e-12)


def _u(p):
    return lambda Y: p.exact(Y)[:, 0]


def _grad_fd(u, Y, h):
    out = np.zeros_like(Y)
    for b in range(3):
        dY = np.zeros_like(Y)
        dY[:, b] = h
        out[:, b] = (u(Y + dY) - u(Y - dY)) / (2 * h)
    return out


def _div_fd(flux, X, h):
    """sum_b d/dx_b of flux(Y)[:, b] by central differences."""
    out = np.zeros(X.shape[0])
    for b in range(3):
        dX = np.zeros_like(X)
        dX[:, b] = h
        out += (flux(X + dX)[:, b] - flux(X - dX)[:, b]) / (2 * h)
    return out


def test_manufactured_sources_satisfy_the_pdes():
    X = np.random.default_rng(8).uniform(0.1, 0.9, (60, 3))
    h = 2e-3
    # kind 4: Lap u - 100 u + 10 cosh u, Laplacian by the 7-point difference
    p = Problem(W.small_3d(pde_kind=4, M=8))
    u = _u(p)
    lap = np.zeros(X.shape[0])
    for b in range(3):
        dX = np.zeros_like(X)
        dX[:, b] = h
        lap += (u(X + dX) - 2 * u(X) + u(X - dX)) / h ** 2
    ref = lap - 100.0 * u(X) + 10.0 * np.cosh(u(X))
    f = p.source(X, 0)
    assert np.max(np.abs(f - ref)) < 1e-4 * np.abs(ref).max()
    # kind 5: -div((1 + u^2) grad u) in flux form
    p = Problem(W.small_3d(pde_kind=5, M=8))
    u = _u(p)
    flux = lambda Y: (1.0 + u(Y) ** 2)[:, None] * _grad_fd(u, Y, h)
    ref = -_div_fd(flux, X, h)
    f = p.source(X, 0)
    assert np.max(np.abs(f - ref)) < 1e-4 * np.abs(ref).max()
    # kind 6: -div((1 + |grad u|^2) grad u) in flux form
    p = Problem(W.small_3d(pde_kind=6, M=8))
    u = _u(p)

    def flux6(Y):
        g = _grad_fd(u, Y, h)
        return (1.0 + np.sum(g * g, axis=1))[:, None] * g

    ref = -_div_fd(flux6, X, h)
    f = p.source(X, 0)
    assert np.max(np.abs(f - ref)) < 1e-4 * np.abs(ref).max()
    # kind 7: kind 5's flux form plus the reaction u^3 - u + e^u
    p = Problem(W.small_3d(pde_kind=7, M=8))
    u = _u(p)
    flux = lambda Y: (1.0 + u(Y) ** 2)[:, None] * _grad_fd(u, Y, h)
    ref = -_div_fd(flux, X, h) + u(X) ** 3 - u(X) + np.exp(u(X))
    f = p.source(X, 0)
    assert np.max(np.abs(f - ref)) < 1e-4 * np.abs(ref).max()


def test_fibonacci_points_cover_the_sphere_evenly():
    from oracle.problem import fibonacci_sphere
    N = 4000
    F = fibonacci_sphere(N)
    assert np.max(np.abs(np.linalg.norm(F, axis=1) - 1.0)) < 1e-15
    # equal-area property: every octant holds about N / 8 points, and the
    # z-coordinates are uniform on (-1, 1) (Archimedes: equal z-bands, equal area)
    octant = (F[:, 0] > 0) * 4 + (F[:, 1] > 0) * 2 + (F[:, 2] > 0)
    counts = np.bincount(octant, minlength=8)
    assert np.all(np.abs(counts - N / 8) < 0.03 * N / 8)
    assert np.allclose(np.sort(F[:, 2]), np.linspace(1 - 1 / N, -1 + 1 / N, N)[::-1])
    # no two points closer than a fraction of the mean spacing sqrt(4 pi / N)
    from scipy.spatial import cKDTree
    d, _ = cKDTree(F).query(F, k=2)
    assert d[:, 1].min() > 0.5 * np.sqrt(4 * np.pi / N)


def test_ball_rows():
    d = W.ball(20, 7, 500)
    p = Problem(d)
    r2 = np.sum(p.rx ** 2, axis=1)
    interior = slice(0, p.m_int + p.m_iface)
    assert np.all(r2[interior] < 1.0)
    assert p.m_bdy == 500 and np.allclose(r2[p.m_int + p.m_iface:], 1.0, rtol=0, atol=1e-15)
    # every row lies in (the closure of) its subdomain
    lo = p.mu[p.re0] - p.sigma[p.re0]
    hi = p.mu[p.re0] + p.sigma[p.re0]
    assert np.all((p.rx >= lo - 1e-15) & (p.rx <= hi + 1e-15))
    # the same grids as the box layout, minus the points outside the ball
    box = Problem(W.with_(d, geometry="box"))
    kept = np.sum(np.sum(box.rx[:box.m_int] ** 2, axis=1) < 1.0)
    assert kept == p.m_int


@pytest.mark.parametrize("kind", KINDS)
def test_ipn_converges_to_the_manufactured_solution(kind):
    """IPN (Alg. 1) from u_0 = 0 on a coarse discretisation reaches the
    manufactured solution to a few percent (the paper's finer settings reach
    1e-5 and below, Sec. 6.2): the source, boundary data and Jacobian are
    consistent with one PDE.  Kinds 4-6 on the unit cube (2x2x2 subdomains,
    M = 40, 6^3 points); kind 7 on its own domain, the unit ball (2x2x2
    subdomains, M = 80, 8 points per axis, 800 boundary points): on the cube
    with M = 40 its Gauss-Newton iteration still converges, but only linearly
    (full steps, shrinking LSQR counts) and not within 30 steps."""
    from oracle import newton
    if kind == 7:
        d = W.ball(80, 8, 800)
        X = W.ball_points(500, 3)
    else:
        d = W.problem(3, (2, 2, 2), 40, (6, 6, 6), (6, 6, 6), (6, 6, 6), pde_kind=kind)
        X = W.eval_grid(d, per_axis=4)
    p = Problem(d)
    c, info = newton.ipn(p, W.solve_opts(max_outer=30))
    assert info.outer_iters < 30
    assert newton.rel_l2(newton.evaluate(p, c, X), p.exact(X)) < 0.1
