"""Residual F(u) and Jacobian J(u) of the RFM nonlinear least-squares system.

Follows Alg. 3 steps 1-4 (interior rows lambda*L(phi)u + mu*N(phi u) - f,
continuity rows A_con u, boundary rows A_bdy u - b_bdy, stacked as Eq. 5.13),
the Jacobian in block form (Sec. 5, J = [lambda A_int + mu dg/du; A_con;
A_bdy]) and the row rescaling lambda_{k,i} = c / max_j |J_ij| with c = 100
(Sec. 5, after Eq. 5.14).

The features are phi = tanh(z), z = k . l_e(x) + b, l_e(x) = (x - mu_e) /
sigma_e (Sec. 2.2, Eq. 2.6), with the analytic derivatives
    d phi / d x_b       = (1 - t^2) k_b / sigma_b
    d^2 phi / d x_b^2   = -2 t (1 - t^2) (k_b / sigma_b)^2 ,   t = tanh(z).

Operators (pde_kind):
  0  F = -Lap u + p0 u^3 - f                 J = -Lap phi + 3 p0 u^2 phi
  4  F = Lap u + p0 u + p1 cosh(u) - f        J = Lap phi + (p0 + p1 sinh u) phi
     (nonlinear Helmholtz of Sec. 6.2, p0 = -100, p1 = 10)
  5  F = -div((1 + u^2) grad u) - f = -(1 + u^2) Lap u - 2 u |grad u|^2 - f
     J = -(1 + u^2) Lap phi - (2 u Lap u + 2 |grad u|^2) phi - 4 u grad u . grad phi
     (Sec. 3.2 benchmark)
  6  F = -div((1 + |grad u|^2) grad u) - f = -(1 + |g|^2) Lap u - 2 g^T H g - f
     J = -(1 + |g|^2) Lap phi - 2 Lap u (g . grad phi) - 4 grad phi . H g - 2 g^T Hess(phi) g
     (strongly nonlinear example of Sec. 6.2; g = grad u, H = Hess u)
  7  kind 5 plus the reaction u^3 - u + e^u (unit-ball example of Sec. 6.2)
  2,3 F = -a Lap u - a_x u_x + kap u^3 - f    J = -a Lap phi - a_x phi_x + 3 kap u^2 phi
      with a = 1 + 0.5 sin(2 pi x), a_x = pi cos(2 pi x)
  1  (Gray-Scott, fields u, v)
     F_u = -eps_u Lap u + u v^2 - F (1 - u) - f_u
     F_v = -eps_v Lap v - u v^2 + (F + k) v - f_v
     dF_u/dc_u = -eps_u Lap phi + (v^2 + F) phi   dF_u/dc_v = 2 u v phi
     dF_v/dc_u = -v^2 phi                        dF_v/dc_v = -eps_v Lap phi - 2 u v phi + (F + k) phi

A row is returned as a primary block (columns of subdomain e0, width W =
fields*M) and, for interface rows, a secondary block (subdomain e1).

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
import math

import numpy as np


def feature_values(prob, e_arr, X):
    """phi, grad phi [.., d], Lap phi for every feature of the subdomains
    e_arr at the points X.  Shapes (r, fields, M) and (r, fields, M, d)."""
    d = prob.d
    mu = prob.mu[e_arr]
    sg = prob.sigma[e_arr]
    L = (X - mu) / sg
    K = prob.feats[e_arr, :, :, :d]
    B = prob.feats[e_arr, :, :, d]
    Z = L[:, 0, None, None] * K[..., 0]
    for b in range(1, d):
        Z = Z + L[:, b, None, None] * K[..., b]
    Z = Z + B
    T = np.tanh(Z)
    S1 = 1.0 - T * T
    ks = K / sg[:, None, None, :]
    grad = S1[..., None] * ks
    lap = np.zeros_like(T)
    for b in range(d):
        lap = lap + (-2.0 * T * S1) * ks[..., b] ** 2
    return T, grad, lap


def feature_hessian(prob, e_arr, X):
    """Second derivatives d^2 phi / dx_a dx_b = -2 t (1 - t^2) (k_a / sigma_a)
    (k_b / sigma_b) of every feature, shape (r, fields, M, d, d)."""
    d = prob.d
    sg = prob.sigma[e_arr]
    L = (X - prob.mu[e_arr]) / sg
    K = prob.feats[e_arr, :, :, :d]
    Z = prob.feats[e_arr, :, :, d].copy()
    for b in range(d):
        Z = Z + L[:, b, None, None] * K[..., b]
    T = np.tanh(Z)
    ks = K / sg[:, None, None, :]
    return (-2.0 * T * (1.0 - T * T))[..., None, None] * ks[..., :, None] * ks[..., None, :]


def _coef_block(prob, c, e_arr):
    return c.reshape(prob.G, prob.fields, prob.M)[e_arr]


def assemble_rows(prob, c, rows, want_jacobian=True):
    """Unscaled F_i and Jacobian row blocks for the given row indices.
    Returns F [r], Jp [r, W], Js [r, W], e0 [r], e1 [r] (e1 = -1 if none)."""
    rows = np.asarray(rows, dtype=np.int64)
    r = rows.size
    W, M, fields = prob.W, prob.M, prob.fields
    F = np.zeros(r)
    Jp = np.zeros((r, W)) if want_jacobian else None
    Js = np.zeros((r, W)) if want_jacobian else None
    kind = prob.rkind[rows]; e0 = prob.re0[rows]; e1 = prob.re1[rows]
    X = prob.rx[rows]; fld = prob.rfield[rows]; ax = prob.raxis[rows]; so = prob.rsord[rows]
    p = prob.params
    # interior rows
    sel = np.nonzero(kind == 0)[0]
    if sel.size:
        phi, grad, lap = feature_values(prob, e0[sel], X[sel])
        cb = _coef_block(prob, c, e0[sel])
        u = np.einsum("rfm,rfm->rf", phi, cb)
        lu = np.einsum("rfm,rfm->rf", lap, cb)
        Xs = X[sel]
        fs = fld[sel]
        src = np.zeros(sel.size)
        for f in range(fields):
            t = fs == f
            if t.any():
                src[t] = prob.source(Xs[t], f)
        k = prob.kind
        if k == 0:
            F[sel] = -lu[:, 0] + p[0] * u[:, 0] ** 3 - src
            if want_jacobian:
                Jp[sel, :M] = -lap[:, 0] + 3.0 * p[0] * (u[:, 0] ** 2)[:, None] * phi[:, 0]
        elif k in (2, 3):
            a = 1.0 + 0.5 * np.sin(2 * math.pi * Xs[:, 0])
            a_x = math.pi * np.cos(2 * math.pi * Xs[:, 0])
            ux = np.einsum("rm,rm->r", grad[:, 0, :, 0], cb[:, 0])
            kap = p[0]
            F[sel] = -a * lu[:, 0] - a_x * ux + kap * u[:, 0] ** 3 - src
            if want_jacobian:
                Jp[sel, :M] = (-a[:, None] * lap[:, 0] - a_x[:, None] * grad[:, 0, :, 0]
                               + 3.0 * kap * (u[:, 0] ** 2)[:, None] * phi[:, 0])
        elif k == 1:
            eu, ev, Fc, kk = p[0], p[1], p[2], p[3]
            uu, vv = u[:, 0], u[:, 1]
            t0 = fs == 0
            t1 = ~t0
            Fu = -eu * lu[:, 0] + uu * vv * vv - Fc * (1.0 - uu) - src
            Fv = -ev * lu[:, 1] - uu * vv * vv + (Fc + kk) * vv - src
            F[sel[t0]] = Fu[t0]
            F[sel[t1]] = Fv[t1]
            if want_jacobian:
                Ju_u = -eu * lap[:, 0] + (vv * vv + Fc)[:, None] * phi[:, 0]
                Ju_v = (2.0 * uu * vv)[:, None] * phi[:, 1]
                Jv_u = -(vv * vv)[:, None] * phi[:, 0]
                Jv_v = -ev * lap[:, 1] + (-2.0 * uu * vv + (Fc + kk))[:, None] * phi[:, 1]
                Jp[sel[t0], :M] = Ju_u[t0]; Jp[sel[t0], M:] = Ju_v[t0]
                Jp[sel[t1], :M] = Jv_u[t1]; Jp[sel[t1], M:] = Jv_v[t1]
        elif k in (4, 5, 6, 7):
            # 3D examples of Sec. 6.2 (one field), from the 2-jet of u at the point
            phi0, grad0, lap0 = phi[:, 0], grad[:, 0], lap[:, 0]
            cb0 = cb[:, 0]
            uu = u[:, 0]
            lu0 = lu[:, 0]
            gu = np.einsum("rmb,rm->rb", grad0, cb0)           # grad u
            gg = np.einsum("rb,rb->r", gu, gu)                  # |grad u|^2
            if k == 4:
                # Lap u + p0 u + p1 cosh(u) = f
                F[sel] = lu0 + p[0] * uu + p[1] * np.cosh(uu) - src
                if want_jacobian:
                    Jp[sel, :M] = lap0 + (p[0] + p[1] * np.sinh(uu))[:, None] * phi0
            elif k in (5, 7):
                # -div((1 + u^2) grad u) = -(1 + u^2) Lap u - 2 u |grad u|^2,
                # kind 7 adds the reaction u^3 - u + e^u (unit-ball example)
                F[sel] = -(1.0 + uu * uu) * lu0 - 2.0 * uu * gg - src
                if k == 7:
                    F[sel] += uu ** 3 - uu + np.exp(uu)
                if want_jacobian:
                    gphi = np.einsum("rmb,rb->rm", grad0, gu)       # grad u . grad phi_j
                    react = 3.0 * uu * uu - 1.0 + np.exp(uu) if k == 7 else 0.0 * uu
                    Jp[sel, :M] = (-(1.0 + uu * uu)[:, None] * lap0
                                   - (2.0 * uu * lu0 + 2.0 * gg - react)[:, None] * phi0
                                   - (4.0 * uu)[:, None] * gphi)
            else:
                # -div((1 + |grad u|^2) grad u) = -(1 + |g|^2) Lap u - 2 g^T H g
                hess0 = feature_hessian(prob, e0[sel], X[sel])[:, 0]       # (r, M, d, d)
                Hu = np.einsum("rmab,rm->rab", hess0, cb0)
                Hg = np.einsum("rab,rb->ra", Hu, gu)
                gHg = np.einsum("ra,ra->r", gu, Hg)
                F[sel] = -(1.0 + gg) * lu0 - 2.0 * gHg - src
                if want_jacobian:
                    gphi = np.einsum("rmb,rb->rm", grad0, gu)
                    hphi = np.einsum("rmb,rb->rm", grad0, Hg)          # grad phi_j . H g
                    gHphig = np.einsum("ra,rmab,rb->rm", gu, hess0, gu)
                    Jp[sel, :M] = (-(1.0 + gg)[:, None] * lap0 - (2.0 * lu0)[:, None] * gphi
                                   - 4.0 * hphi - 2.0 * gHphig)
        else:
            raise ValueError(k)
    # interface rows: [d^s phi_e0 | -d^s phi_e1] on the row's field
    sel = np.nonzero(kind == 1)[0]
    if sel.size:
        for side, es in ((0, e0[sel]), (1, e1[sel])):
            phi, grad, _ = feature_values(prob, es, X[sel])
            sgn = 1.0 if side == 0 else -1.0
            cb = _coef_block(prob, c, es)
            for j, i in enumerate(sel):
                f = fld[i]
                vals = phi[j, f] if so[i] == 0 else grad[j, f, :, ax[i]]
                F[i] += sgn * np.dot(vals, cb[j, f])
                if want_jacobian:
                    (Jp if side == 0 else Js)[i, f * M:(f + 1) * M] = sgn * vals
    # boundary rows: phi_e0 on the row's field, minus g
    sel = np.nonzero(kind == 2)[0]
    if sel.size:
        phi, _, _ = feature_values(prob, e0[sel], X[sel])
        cb = _coef_block(prob, c, e0[sel])
        for f in range(fields):
            t = np.nonzero(fld[sel] == f)[0]
            if t.size == 0:
                continue
            ii = sel[t]
            g = prob.boundary_data(X[ii], f)
            F[ii] = np.einsum("rm,rm->r", phi[t, f], cb[t, f]) - g
            if want_jacobian:
                Jp[ii, f * M:(f + 1) * M] = phi[t, f]
    return F, Jp, Js, e0, e1


def row_scale(Jp, Js, C=100.0):
    """lambda_i = C / max_j |J_ij| over the whole row; a zero row keeps 1."""
    mx = np.abs(Jp).max(axis=1)
    if Js is not None:
        mx = np.maximum(mx, np.abs(Js).max(axis=1))
    lam = np.ones_like(mx)
    nz = mx > 0
    lam[nz] = C / mx[nz]
    return lam


def assemble(prob, c, chunk=4096):
    """Unscaled F [m] and dense J [m, n] (small problems only)."""
    m, n, W = prob.m, prob.n, prob.W
    F = np.zeros(m)
    J = np.zeros((m, n))
    for s in range(0, m, chunk):
        rows = np.arange(s, min(m, s + chunk))
        Fr, Jp, Js, e0, e1 = assemble_rows(prob, c, rows)
        F[rows] = Fr
        for j, i in enumerate(rows):
            J[i, e0[j] * W:(e0[j] + 1) * W] = Jp[j]
            if e1[j] >= 0:
                J[i, e1[j] * W:(e1[j] + 1) * W] = Js[j]
    return F, J


def residual(prob, c, chunk=8192):
    """Unscaled F(c) [m]."""
    F = np.zeros(prob.m)
    for s in range(0, prob.m, chunk):
        rows = np.arange(s, min(prob.m, s + chunk))
        F[rows] = assemble_rows(prob, c, rows, want_jacobian=False)[0]
    return F


def scaled_system(prob, c, C=100.0):
    """Row-scaled (F, J, lambda) at c (Sec. 5 rescaling)."""
    F, J = assemble(prob, c)
    lam = np.ones(prob.m)
    mx = np.abs(J).max(axis=1)
    nz = mx > 0
    lam[nz] = C / mx[nz]
    return lam * F, lam[:, None] * J, lam
