"""Seeded synthetic workloads for the RFM nonlinear-solver hot path.

This module holds *inputs only*: problem descriptors (domain box, subdomain
grid, features per subdomain, collocation counts, seeds, PDE selector and its
parameters), solver options, and seeded random vectors / query points used by
tests and the benchmark.  It holds none of the method's arithmetic; both the
CUDA library and the CPU oracle interpret these descriptors independently.

Problem families (the paper's experiments, Sec. 6; configuration sizes are
those of the configurations C1-C5 below):

  pde_kind 0  -Lap u + u^3 = f,  u* = prod sin(pi x_d)       (Sec. 6.1, Eq. 6.1)
  pde_kind 1  steady Gray-Scott, two fields u, v              (Sec. 6.2, Gray-Scott
              system), constant diffusion eps_u, eps_v
  pde_kind 2  -div(a grad u) + kappa u^3 = f, a = 1 + 0.5 sin(2 pi x),
              u* = prod sin(pi x_d)
  pde_kind 3  same operator as kind 2 with source A prod sin(q pi x_d) and
              homogeneous Dirichlet data (no closed-form solution)
  pde_kind 4  Lap u - 100 u + 10 cosh(u) = f on [0,1]^3, u* = (2 + |x|^2) prod sin(pi x_d)
              (Sec. 6.2, nonlinear Helmholtz equation)
  pde_kind 5  -div((1 + u^2) grad u) = f on [0,1]^3, u* = (x+y+z) sin(pi x) sin(pi y) cos(pi z)
              (Sec. 3.2 benchmark)
  pde_kind 6  -div((1 + |grad u|^2) grad u) = f on [0,1]^3,
              u* = sin(x(1-x)) sin(y(1-y)) e^(z+1/2)  (Sec. 6.2, strongly nonlinear)
  pde_kind 7  -div((1 + u^2) grad u) + u^3 - u + e^u = f on the unit ball,
              u* = |x|^2 prod sin(pi x_d)  (Sec. 6.2, diffusion-reaction on the ball:
              geometry "ball", the cube [-1,1]^3 in subdomains, collocation points
              inside the ball kept, Dirichlet rows at n_sphere Fibonacci points)
"""
from __future__ import annotations

import copy

import numpy as np

FEATURE_SEED = 20251004

# pde_params layout per kind (8 doubles):
#   kind 0: [cubic coefficient]
#   kind 1: [eps_u, eps_v, F, k]
#   kind 2: [kappa]
#   kind 3: [kappa, amplitude A, frequency q]
#   kind 4: [coefficient of u (-100), coefficient of cosh u (10)]
#   kinds 5, 6: none


def problem(dim, nsub, M, q_int, q_bdy, q_iface, *, fields=1, lo=None, hi=None,
            cont_order=2, feat_range=1.0, seed=FEATURE_SEED, pde_kind=0,
            pde_params=None):
    lo = tuple(lo) if lo is not None else (0.0,) * dim
    hi = tuple(hi) if hi is not None else (1.0,) * dim
    params = list(pde_params) if pde_params is not None else _default_params(pde_kind)
    params = (params + [0.0] * 8)[:8]
    return dict(dim=dim, lo=lo, hi=hi, nsub=tuple(nsub), M=M, fields=fields,
                q_int=tuple(q_int), q_bdy=tuple(q_bdy), q_iface=tuple(q_iface),
                cont_order=cont_order, feat_range=feat_range, seed=seed,
                pde_kind=pde_kind, pde_params=tuple(float(p) for p in params))


def _default_params(kind):
    return {0: [1.0], 1: [2e-3, 1e-3, 0.04, 0.06], 2: [1.0], 3: [1.0, 1.0, 1.0], 4: [-100.0, 10.0],
            5: [], 6: [], 7: []}[kind]


def solve_opts(**kw):
    """Solver options; defaults are the paper's settings (Sec. 6: gamma=3,
    eta=1e-6, eps=1e-10, tau_rel=1e-3, m_max=3; row scale c=100, Sec. 5)."""
    o = dict(sketch_kind="count", gamma=3.0, sketch_rows=0, eta=1e-6, eps=1e-10,
             max_outer=50, m_max=3, tau_rel=1e-3, row_scale_c=100.0,
             lsqr_max_iter=0, conlim=1e8, precision=0)
    o.update(kw)
    return o


# ---- the five benchmark configurations ----------------------------------

def config_c1():
    """2D -Lap u + u^3, 2x2 subdomains, M=100, 20x20 interior grid per
    subdomain, 20 points per subdomain edge on the boundary (40 per domain
    side) and per interface; count sketch gamma=3."""
    return problem(2, (2, 2), 100, (20, 20), (20, 20), (20, 20))


def config_c2():
    """3D -Lap u + u^3, 4x4x4 subdomains, M=512 (n=32,768), 12^3 interior
    points and 6x6 points per face; Gaussian sketch with 65,536 rows."""
    return problem(3, (4, 4, 4), 512, (12, 12, 12), (6, 6, 6), (6, 6, 6))


def opts_c2(**kw):
    return solve_opts(sketch_kind="gauss", sketch_rows=65536, **kw)


def config_c3():
    """3D steady Gray-Scott, two fields, 4x4x4 subdomains, M=256 per field."""
    return problem(3, (4, 4, 4), 256, (12, 12, 12), (6, 6, 6), (6, 6, 6),
                   fields=2, pde_kind=1)


def grayscott_small():
    """The Gray-Scott system of config_c3 at 2x2x2 subdomains and M=64 per
    field (n=1,024), small enough for whole oracle solves."""
    return problem(3, (2, 2, 2), 64, (12, 12, 12), (6, 6, 6), (6, 6, 6),
                   fields=2, pde_kind=1)


def paper_3d(kind, M, q=20):
    """The 3D examples of Sec. 6.2 (and the Sec. 3.2 benchmark) at the paper's
    settings: 2x2x2 subdomains, q^3 interior points and q x q points per face,
    M features per subdomain (the paper's J)."""
    return problem(3, (2, 2, 2), M, (q, q, q), (q, q, q), (q, q, q), pde_kind=kind)


def operator_small(kind):
    """Kinds 4-6 at 2x2x2 subdomains, M = 100 (n = 800), 8^3 interior points
    and 8 x 8 per face: whole oracle solves take under a minute."""
    return problem(3, (2, 2, 2), 100, (8, 8, 8), (8, 8, 8), (8, 8, 8), pde_kind=kind)


def ball(M, q, n_sphere, nsub=(2, 2, 2)):
    """Unit-ball diffusion-reaction (kind 7): [-1,1]^3 in nsub subdomains, q^3
    grid points per subdomain and q x q per interface (those inside the ball
    kept), n_sphere Fibonacci points on the sphere."""
    d = problem(3, nsub, M, (q, q, q), (q, q, q), (q, q, q), lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0),
                pde_kind=7)
    d.update(geometry="ball", n_sphere=int(n_sphere))
    return d


def config_c5(kappa=1.0, amp=1.0, freq=1.0):
    """Learned-warm-start family: 2x2x2 subdomains, M=512 (n=4,096)."""
    return problem(3, (2, 2, 2), 512, (12, 12, 12), (6, 6, 6), (6, 6, 6),
                   pde_kind=3, pde_params=[kappa, amp, freq])


def config_c4_instances(count=64, seed=1):
    """Batched family: instance i uses g=2+(i mod 3) subdomains per axis and
    M=128 when floor(i/3) is even else 256; kappa ~ U[0.1, 10] from a seeded
    generator.  All instances share one feature seed."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        g = 2 + (i % 3)
        M = 128 if (i // 3) % 2 == 0 else 256
        kappa = float(rng.uniform(0.1, 10.0))
        out.append(problem(3, (g, g, g), M, (12, 12, 12), (6, 6, 6), (6, 6, 6),
                           pde_kind=2, pde_params=[kappa]))
    return out


def small_2d(M=24, nsub=(2, 2), q=8, seed=FEATURE_SEED, pde_kind=0):
    return problem(2, nsub, M, (q, q), (q, q), (q, q), seed=seed, pde_kind=pde_kind)


def small_3d(M=32, nsub=(2, 2, 2), q=5, qf=4, seed=FEATURE_SEED, pde_kind=0, fields=1,
             pde_params=None):
    return problem(3, nsub, M, (q, q, q), (qf, qf, qf), (qf, qf, qf), seed=seed,
                   pde_kind=pde_kind, fields=fields, pde_params=pde_params)


def with_(desc, **kw):
    d = copy.deepcopy(desc)
    d.update(kw)
    return d


# ---- seeded vectors and query points -------------------------------------

def random_coeffs(n, seed=7, scale=1.0):
    return np.random.default_rng(seed).standard_normal(n) * scale


def random_points(desc, count, seed=11):
    rng = np.random.default_rng(seed)
    d = desc["dim"]
    lo = np.array(desc["lo"][:d]); hi = np.array(desc["hi"][:d])
    return lo + (hi - lo) * rng.random((count, d))


def ball_points(count, seed=5):
    """`count` seeded uniform points inside the unit ball (rejection from the cube)."""
    rng = np.random.default_rng(seed)
    out = []
    while sum(len(o) for o in out) < count:
        P = rng.uniform(-1.0, 1.0, (2 * count, 3))
        out.append(P[np.sum(P * P, axis=1) < 1.0])
    return np.concatenate(out)[:count]


def eval_grid(desc, per_axis=10):
    """Cell-centred grid with `per_axis` points per subdomain per axis; no
    point lies on an interface."""
    d = desc["dim"]
    axes = []
    for b in range(d):
        N = desc["nsub"][b] * per_axis
        lo, hi = desc["lo"][b], desc["hi"][b]
        axes.append(lo + (hi - lo) * (np.arange(N) + 0.5) / N)
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([m.reshape(-1) for m in mesh], axis=1)
