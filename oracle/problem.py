"""Geometry, collocation rows and manufactured data of the RFM discretisation.

Follows Sec. 2.2 (subdomains Omega_i, affine map l_i(x) = (x - mu_i)/sigma_i,
indicator partition of unity psi^a, tanh features phi_ij) and Sec. 5 (uniform
collocation grids including endpoints, interface continuity rows C^0..C^{k-1},
Eqs. con:1-3, and Dirichlet boundary rows, Eqs. bdy:1-3).  Row counts reproduce
Sec. 3.2's formulas m = Q_I + Q_b + Q_c.

Row order (a reading; the paper does not fix one):
  1. interior rows: subdomain e (lexicographic, axis 0 slowest), field f,
     grid point (lexicographic, axis 0 slowest);
  2. interface rows: normal axis a = 0..d-1; left subdomain e (lexicographic)
     with a right neighbour along a; field f; derivative order s = 0..k-1;
     face point (remaining axes lexicographic);
  3. boundary rows: axis a = 0..d-1; side lo then hi; subdomain e touching it
     (lexicographic); field f; face point.
Unknowns are ordered subdomain-major, then field, then feature.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
import math

import numpy as np

from . import philox


def fibonacci_sphere(count):
    """`count` points spread uniformly over the unit sphere by the Fibonacci
    (golden-angle) spiral: z_i = 1 - (2 i + 1) / count, radius sqrt(1 - z_i^2),
    azimuth i * pi (3 - sqrt 5)."""
    ga = math.pi * (3.0 - math.sqrt(5.0))
    out = np.zeros((count, 3))
    for i in range(count):
        z = 1.0 - (2.0 * i + 1.0) / count
        r = math.sqrt(1.0 - z * z)
        th = i * ga
        out[i] = (r * math.cos(th), r * math.sin(th), z)
    return out


class Problem:
    def __init__(self, desc):
        self.desc = desc
        d = self.d = int(desc["dim"])
        self.N = [int(x) for x in desc["nsub"][:d]]
        self.G = int(np.prod(self.N))
        self.M = int(desc["M"])
        self.fields = int(desc["fields"])
        self.W = self.fields * self.M
        self.n = self.G * self.W
        self.lo = [float(x) for x in desc["lo"][:d]]
        self.hi = [float(x) for x in desc["hi"][:d]]
        self.kind = int(desc["pde_kind"])
        self.params = [float(p) for p in desc["pde_params"]]
        self.cont = int(desc["cont_order"])
        # breakpoints X_b[j] = lo + (hi - lo) * j / N, ends exact
        self.X = []
        for b in range(d):
            xs = [self.lo[b] + ((self.hi[b] - self.lo[b]) * j) / self.N[b] for j in range(self.N[b] + 1)]
            xs[0], xs[-1] = self.lo[b], self.hi[b]
            self.X.append(xs)
        self.idx = np.array([self.sub_index(e) for e in range(self.G)], dtype=np.int64).reshape(self.G, d)
        self.mu = np.array([[0.5 * (self.X[b][i[b]] + self.X[b][i[b] + 1]) for b in range(d)] for i in self.idx])
        self.sigma = np.array([[0.5 * (self.X[b][i[b] + 1] - self.X[b][i[b]]) for b in range(d)] for i in self.idx])
        self.feats = philox.features(self.G, self.fields, self.M, d, float(desc["feat_range"]), desc["seed"])
        self._build_rows()

    # -- indexing ---------------------------------------------------------
    def sub_index(self, e):
        out = []
        for b in reversed(range(self.d)):
            out.append(e % self.N[b])
            e //= self.N[b]
        return tuple(reversed(out))

    def sub_id(self, idx):
        e = 0
        for b in range(self.d):
            e = e * self.N[b] + idx[b]
        return e

    def grid1d(self, b, j, q):
        a, c = self.X[b][j], self.X[b][j + 1]
        pts = [a + ((c - a) * p) / (q - 1) for p in range(q)]
        pts[0], pts[-1] = a, c
        return pts

    # -- rows -------------------------------------------------------------
    def _face_points(self, e, a, qs):
        other = [b for b in range(self.d) if b != a]
        idx = self.idx[e]
        axes = [self.grid1d(b, idx[b], qs[b]) for b in other]
        mesh = np.meshgrid(*axes, indexing="ij") if axes else []
        cnt = int(np.prod([len(x) for x in axes])) if axes else 1
        P = np.zeros((cnt, self.d))
        for t, b in enumerate(other):
            P[:, b] = mesh[t].reshape(-1)
        return P

    def _build_rows(self):
        d = self.d
        desc = self.desc
        kind, e0, e1, axis, sord, field, side, pts = [], [], [], [], [], [], [], []

        def add(P, k, a0, a1, ax, s, f, sd):
            r = P.shape[0]
            kind.append(np.full(r, k)); e0.append(np.full(r, a0)); e1.append(np.full(r, a1))
            axis.append(np.full(r, ax)); sord.append(np.full(r, s)); field.append(np.full(r, f))
            side.append(np.full(r, sd)); pts.append(P)

        ball = desc.get("geometry", "box") == "ball"
        # inside the ball: (x^2 + y^2) + z^2 < 1, summed in that order
        keep = (lambda P: P[(P[:, 0] * P[:, 0] + P[:, 1] * P[:, 1]) + P[:, 2] * P[:, 2] < 1.0]) if ball \
            else (lambda P: P)
        qi = desc["q_int"]
        for e in range(self.G):
            axes = [self.grid1d(b, self.idx[e][b], qi[b]) for b in range(d)]
            mesh = np.meshgrid(*axes, indexing="ij")
            P = keep(np.stack([m.reshape(-1) for m in mesh], axis=1))
            for f in range(self.fields):
                add(P, 0, e, -1, -1, 0, f, -1)
        self.m_int = sum(p.shape[0] for p in pts)
        for a in range(d):
            for e in range(self.G):
                idx = list(self.idx[e])
                if idx[a] >= self.N[a] - 1:
                    continue
                nb = list(idx); nb[a] += 1
                e2 = self.sub_id(nb)
                P = self._face_points(e, a, desc["q_iface"])
                P[:, a] = self.X[a][idx[a] + 1]
                P = keep(P)
                for f in range(self.fields):
                    for s in range(self.cont):
                        add(P, 1, e, e2, a, s, f, -1)
        self.m_iface = sum(p.shape[0] for p in pts) - self.m_int
        if ball:
            # Dirichlet rows at Fibonacci points of the unit sphere, grouped by
            # the subdomain that contains them (Sec. 6.2, unit-ball example)
            F = fibonacci_sphere(int(desc["n_sphere"]))
            own = np.zeros(F.shape[0], dtype=np.int64)
            for b in range(d):
                t = np.floor((F[:, b] - self.lo[b]) / (self.hi[b] - self.lo[b]) * self.N[b]).astype(np.int64)
                own = own * self.N[b] + np.clip(t, 0, self.N[b] - 1)
            for e in range(self.G):
                sel = np.nonzero(own == e)[0]
                if sel.size:
                    for f in range(self.fields):
                        add(F[sel], 2, e, -1, -1, 0, f, -1)
        for a in range(d if not ball else 0):
            for sd in (0, 1):
                for e in range(self.G):
                    if self.idx[e][a] != (0 if sd == 0 else self.N[a] - 1):
                        continue
                    P = self._face_points(e, a, desc["q_bdy"])
                    P[:, a] = self.lo[a] if sd == 0 else self.hi[a]
                    for f in range(self.fields):
                        add(P, 2, e, -1, a, 0, f, sd)
        cat = np.concatenate
        self.rkind = cat(kind); self.re0 = cat(e0); self.re1 = cat(e1)
        self.raxis = cat(axis); self.rsord = cat(sord); self.rfield = cat(field)
        self.rside = cat(side); self.rx = cat(pts, axis=0)
        self.m = self.rx.shape[0]
        self.m_bdy = self.m - self.m_int - self.m_iface

    # -- manufactured data --------------------------------------------------
    def exact(self, X):
        """Manufactured solution at points X [npts, d] -> [npts, fields]
        (kind 3 has none and returns NaN)."""
        k = self.kind
        S = np.ones(X.shape[0])
        for b in range(self.d):
            S = S * np.sin(math.pi * X[:, b])
        if k in (0, 2):
            return S[:, None]
        if k == 1:
            x, y, z = X[:, 0], X[:, 1], X[:, 2]
            u = np.sin(x * (1 - x)) * np.sin(y * (1 - y)) * np.exp(z)
            return np.stack([u, S], axis=1)
        if k in (4, 5, 6, 7):
            return self.exact_jet(X)[0][:, None]
        return np.full((X.shape[0], 1), np.nan)

    def exact_jet(self, X):
        """Value, gradient [npts, 3] and Hessian [npts, 3, 3] of the manufactured
        solutions of the 3D examples of Sec. 6.2:
          kind 4 (nonlinear Helmholtz)   u = (2 + x^2 + y^2 + z^2) sin(pi x) sin(pi y) sin(pi z)
          kind 5 (Lambda(u) = 1 + u^2)   u = (x + y + z) sin(pi x) sin(pi y) cos(pi z)   (Sec. 3.2)
          kind 6 (Lambda = 1 + |grad u|^2) u = sin(x(1-x)) sin(y(1-y)) e^(z + 1/2)
          kind 7 (unit-ball diffusion-reaction) u = (x^2 + y^2 + z^2) sin(pi x) sin(pi y) sin(pi z)
        Each is a product form; the derivatives are written out by hand."""
        pi = math.pi
        x = [X[:, b] for b in range(3)]
        npts = X.shape[0]
        if self.kind == 6:
            # u = A(x) B(y) C(z), A = sin(x(1-x)), C = e^(z+1/2)
            fs = []
            for b in range(2):
                w = x[b] * (1 - x[b])
                f0 = np.sin(w)
                f1 = np.cos(w) * (1 - 2 * x[b])
                f2 = -np.sin(w) * (1 - 2 * x[b]) ** 2 - 2 * np.cos(w)
                fs.append((f0, f1, f2))
            e = np.exp(x[2] + 0.5)
            fs.append((e, e, e))
            u = fs[0][0] * fs[1][0] * fs[2][0]
            g = np.zeros((npts, 3))
            H = np.zeros((npts, 3, 3))
            for a in range(3):
                for b in range(3):
                    prod = np.ones(npts)
                    for c in range(3):
                        order = (a == c) + (b == c)
                        prod = prod * fs[c][order]
                    H[:, a, b] = prod
                prod = np.ones(npts)
                for c in range(3):
                    prod = prod * fs[c][1 if c == a else 0]
                g[:, a] = prod
            return u, g, H
        # u = r(x) P(x): P a product of sines (and a cosine for kind 5)
        trig = []
        for b in range(3):
            if self.kind == 5 and b == 2:
                trig.append((np.cos(pi * x[b]), -pi * np.sin(pi * x[b]), -pi * pi * np.cos(pi * x[b])))
            else:
                trig.append((np.sin(pi * x[b]), pi * np.cos(pi * x[b]), -pi * pi * np.sin(pi * x[b])))
        P = trig[0][0] * trig[1][0] * trig[2][0]
        dP = np.zeros((npts, 3))
        HP = np.zeros((npts, 3, 3))
        for a in range(3):
            for b in range(3):
                prod = np.ones(npts)
                for c in range(3):
                    prod = prod * trig[c][(a == c) + (b == c)]
                HP[:, a, b] = prod
            prod = np.ones(npts)
            for c in range(3):
                prod = prod * trig[c][1 if c == a else 0]
            dP[:, a] = prod
        if self.kind in (4, 7):
            r = (2.0 if self.kind == 4 else 0.0) + x[0] ** 2 + x[1] ** 2 + x[2] ** 2
            dr = np.stack([2 * x[0], 2 * x[1], 2 * x[2]], axis=1)
            Hr = np.broadcast_to(2.0 * np.eye(3), (npts, 3, 3))
        else:
            r = x[0] + x[1] + x[2]
            dr = np.ones((npts, 3))
            Hr = np.zeros((npts, 3, 3))
        u = r * P
        g = dr * P[:, None] + r[:, None] * dP
        H = (Hr * P[:, None, None] + dr[:, :, None] * dP[:, None, :] + dP[:, :, None] * dr[:, None, :]
             + r[:, None, None] * HP)
        return u, g, H

    def source(self, X, f):
        """Right-hand side f of the PDE for field f at interior points."""
        k, p, d = self.kind, self.params, self.d
        pi = math.pi
        if k == 0:
            u = self.exact(X)[:, 0]
            return d * pi * pi * u + p[0] * u ** 3
        if k == 2:
            u = self.exact(X)[:, 0]
            a = 1.0 + 0.5 * np.sin(2 * pi * X[:, 0])
            ax = pi * np.cos(2 * pi * X[:, 0])
            ux = pi * np.cos(pi * X[:, 0])
            for b in range(1, d):
                ux = ux * np.sin(pi * X[:, b])
            return a * d * pi * pi * u - ax * ux + p[0] * u ** 3
        if k == 3:
            kap, A, q = p[0], p[1], p[2]
            S = np.ones(X.shape[0])
            for b in range(d):
                S = S * np.sin(q * pi * X[:, b])
            return A * S
        if k in (4, 5, 6, 7):
            u, g, H = self.exact_jet(X)
            lap = H[:, 0, 0] + H[:, 1, 1] + H[:, 2, 2]
            if k == 7:  # -div((1 + u^2) grad u) + u^3 - u + e^u
                return (-(1.0 + u * u) * lap - 2.0 * u * np.einsum("ra,ra->r", g, g) + u ** 3 - u + np.exp(u))
            if k == 4:  # Lap u + p0 u + p1 cosh(u) = f
                return lap + p[0] * u + p[1] * np.cosh(u)
            if k == 5:  # -div((1 + u^2) grad u) = -(1 + u^2) Lap u - 2 u |grad u|^2
                return -(1.0 + u * u) * lap - 2.0 * u * np.einsum("ra,ra->r", g, g)
            # -div((1 + |grad u|^2) grad u) = -(1 + |g|^2) Lap u - 2 g^T H g
            gg = np.einsum("ra,ra->r", g, g)
            return -(1.0 + gg) * lap - 2.0 * np.einsum("ra,rab,rb->r", g, H, g)
        if k == 1:
            eu, ev, F, kk = p[0], p[1], p[2], p[3]
            x, y, z = X[:, 0], X[:, 1], X[:, 2]
            # u = sin(x(1-x)) sin(y(1-y)) e^z ; v = sin(pi x) sin(pi y) sin(pi z)
            ax, ay = x * (1 - x), y * (1 - y)
            sx, cx, sy, cy = np.sin(ax), np.cos(ax), np.sin(ay), np.cos(ay)
            ez = np.exp(z)
            u = sx * sy * ez
            uxx = (-sx * (1 - 2 * x) ** 2 - 2 * cx) * sy * ez
            uyy = sx * (-sy * (1 - 2 * y) ** 2 - 2 * cy) * ez
            lap_u = uxx + uyy + u
            v = np.sin(pi * x) * np.sin(pi * y) * np.sin(pi * z)
            lap_v = -3 * pi * pi * v
            if f == 0:
                return -eu * lap_u + u * v * v - F * (1 - u)
            return -ev * lap_v - u * v * v + (F + kk) * v
        raise ValueError(k)

    def boundary_data(self, X, f):
        if self.kind == 3:
            return np.zeros(X.shape[0])
        return self.exact(X)[:, f]
