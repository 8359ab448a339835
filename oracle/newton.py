"""Golden-section line search, IPN (Alg. 1), AMIPN (Alg. 2) and evaluation.

Readings of points the paper leaves open (each also listed in the design notes):
* Line search (Alg. 1, "golden-section search such that ||F(u + alpha d)||
  sufficiently decreases"): phi(alpha) = ||W F(u + alpha d)|| on [0, 1];
  golden-section steps until the bracket is at most 1e-3 (17 interior
  evaluations), plus alpha = 1.  The step is the evaluated alpha with the
  smallest phi (values within a relative 1e-12 of the minimum count as ties and
  the largest alpha wins); if no evaluated phi is below phi(0) the step is 0.
* The row scale W = diag(lambda_k) is recomputed at each Jacobian evaluation
  and used for every residual norm until the next one (Sec. 5 defines
  lambda_{k,i} per Newton iteration k).
* Initial guess u_0 = 0, at most K = 50 outer iterations.
* The sketch S_k is drawn afresh for the k-th Jacobian evaluation.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
import math

import numpy as np

from . import assemble as asm
from . import linalg as la

GOLD = (math.sqrt(5.0) - 1.0) / 2.0


def golden_section(phi, f0, tol=1e-3):
    a, b = 0.0, 1.0
    x1 = b - GOLD * (b - a)
    x2 = a + GOLD * (b - a)
    f1, f2 = phi(x1), phi(x2)
    pts = [(x1, f1), (x2, f2)]
    while b - a > tol:
        if f1 < f2:
            b, x2, f2 = x2, x1, f1
            x1 = b - GOLD * (b - a)
            f1 = phi(x1)
            pts.append((x1, f1))
        else:
            a, x1, f1 = x1, x2, f2
            x2 = a + GOLD * (b - a)
            f2 = phi(x2)
            pts.append((x2, f2))
    pts.append((1.0, phi(1.0)))
    fmin = min(f for _, f in pts)
    best = max(x for x, f in pts if f <= fmin * (1.0 + 1e-12))
    fbest = min(f for x, f in pts if x == best)
    if not fbest < f0:
        return 0.0, f0, len(pts)
    return best, fbest, len(pts)


def sketch_rows(prob, opts):
    if opts.get("sketch_rows", 0):
        s = int(opts["sketch_rows"])
    else:
        s = int(math.ceil(opts["gamma"] * prob.n))
    if opts["sketch_kind"] == "gauss" and s % 2:
        s += 1
    return s


class Info:
    def __init__(self):
        self.outer_iters = 0
        self.n_jac = 0
        self.lsqr_iters = []
        self.alphas = []
        self.final_resid = float("nan")
        self.rank_flag = False


class _Lin:
    """Scaled Jacobian, row scale and preconditioner R at one point."""

    def __init__(self, prob, opts, c, kJ, blocked=True):
        C = opts["row_scale_c"]
        F, J = asm.assemble(prob, c)
        mx = np.abs(J).max(axis=1)
        lam = np.ones(prob.m)
        lam[mx > 0] = C / mx[mx > 0]
        self.lam = lam
        self.J = lam[:, None] * J
        s = sketch_rows(prob, opts)
        seed = prob.desc["seed"]
        if opts["sketch_kind"] == "gauss":
            B = la.gaussian_sketch(self.J, s, kJ, seed)
        else:
            B = la.count_sketch(self.J, s, kJ, seed)
        self.B = B
        qr = la.qr_r_blocked if blocked else la.qr_r_unblocked
        self.R, self.rank_flag = qr(B)

    def direction(self, rhs, opts, n):
        R, J = self.R, self.J
        mv = lambda v: J @ la.solve_upper(R, v)
        rmv = lambda u: la.solve_upper_t(R, J.T @ u)
        lim = opts.get("lsqr_max_iter", 0) or 2 * n
        eta = opts["eta"]
        res = la.lsqr(mv, rmv, rhs, n, eta, eta, opts.get("conlim", 1e8), lim)
        return la.solve_upper(R, res.x), res


def scaled_norm(prob, lam, c):
    return float(np.linalg.norm(lam * asm.residual(prob, c)))


def _make_lin(prob, opts, c, kJ, blocked, lean, workers):
    if lean:
        from .lean import LeanLin
        return LeanLin(prob, opts, c, kJ, workers)
    return _Lin(prob, opts, c, kJ, blocked)


def ipn(prob, opts, c0=None, blocked=True, lean=False, workers=0, log=None):
    """Algorithm 1 (IPN).  lean=True keeps J in block form and forms the
    sketch and QR without dense m x n or s x m arrays (oracle.lean); workers
    spreads the Gaussian sketch over that many processes; log(k, info) is
    called after each outer iteration."""
    n = prob.n
    c = np.zeros(n) if c0 is None else np.array(c0, dtype=np.float64)
    info = Info()
    for k in range(int(opts["max_outer"])):
        lin = _make_lin(prob, opts, c, k, blocked, lean, workers)
        info.n_jac += 1
        info.rank_flag |= lin.rank_flag
        f0 = scaled_norm(prob, lin.lam, c)
        d, res = lin.direction(-lin.lam * asm.residual(prob, c), opts, n)
        info.lsqr_iters.append(res.itn)
        alpha, f1, _ = golden_section(lambda a: scaled_norm(prob, lin.lam, c + a * d), f0)
        info.alphas.append(alpha)
        c = c + alpha * d
        info.outer_iters = k + 1
        info.final_resid = f1
        if log is not None:
            log(k, info)
        if abs(f1 - f0) < opts["eps"]:
            break
    return c, info


def amipn(prob, opts, c0=None, blocked=True, lean=False, workers=0, log=None):
    """Algorithm 2 (AMIPN): one Jacobian and preconditioner per outer
    iteration, up to m_max inner steps reusing them, early stop when
    ||F_{k,i+1} - F_{k,i}|| < tau_rel ||F_{k,0}||; the Jacobian is recomputed
    only when the inner loop ran to m_max."""
    n = prob.n
    c = np.zeros(n) if c0 is None else np.array(c0, dtype=np.float64)
    info = Info()
    kJ = 0
    lin = _make_lin(prob, opts, c, kJ, blocked, lean, workers)
    info.n_jac = 1
    info.rank_flag |= lin.rank_flag
    for k in range(int(opts["max_outer"])):
        z = c
        Fk0 = -lin.lam * asm.residual(prob, c)
        nk0 = float(np.linalg.norm(Fk0))
        Fprev = Fk0
        flag = True
        for i in range(int(opts["m_max"])):
            d, res = lin.direction(Fprev, opts, n)
            info.lsqr_iters.append(res.itn)
            f0 = float(np.linalg.norm(Fprev))
            alpha, _, _ = golden_section(lambda a: scaled_norm(prob, lin.lam, z + a * d), f0)
            info.alphas.append(alpha)
            z = z + alpha * d
            Fnew = -lin.lam * asm.residual(prob, z)
            stop = float(np.linalg.norm(Fnew - Fprev)) < opts["tau_rel"] * nk0
            Fprev = Fnew
            if stop:
                flag = False
                break
        c = z
        info.outer_iters = k + 1
        nk1 = float(np.linalg.norm(Fprev))
        info.final_resid = nk1
        if log is not None:
            log(k, info)
        if abs(nk1 - nk0) < opts["eps"]:
            break
        if flag:
            kJ += 1
            lin = _make_lin(prob, opts, c, kJ, blocked, lean, workers)
            info.n_jac += 1
            info.rank_flag |= lin.rank_flag
    return c, info


def owner(prob, X):
    e = np.zeros(X.shape[0], dtype=np.int64)
    for b in range(prob.d):
        t = np.floor((X[:, b] - prob.lo[b]) / (prob.hi[b] - prob.lo[b]) * prob.N[b]).astype(np.int64)
        t = np.clip(t, 0, prob.N[b] - 1)
        e = e * prob.N[b] + t
    return e


def evaluate(prob, c, X):
    """u_n(x) = sum_j c_ej phi_ej(x) on the owning subdomain e (indicator
    partition of unity psi^a, Sec. 2.2).  Returns [npts, fields]."""
    e = owner(prob, X)
    out = np.zeros((X.shape[0], prob.fields))
    for s in range(0, X.shape[0], 4096):
        sl = slice(s, s + 4096)
        phi, _, _ = asm.feature_values(prob, e[sl], X[sl])
        cb = c.reshape(prob.G, prob.fields, prob.M)[e[sl]]
        out[sl] = np.einsum("rfm,rfm->rf", phi, cb)
    return out


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
