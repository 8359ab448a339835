"""Sketch, Householder QR, triangular solves and LSQR (Sec. 4.1, Alg. 1).

* Sketch B = S_k J (Sec. 4.1): count sketch (one +-1 per column of S_k,
  never formed) or a Gaussian sketch with bfloat16-exact entries.
* Thin QR B = Q R by Householder reflections without pivoting (textbook
  form: reflector H = I - tau v v^T with v_0 = 1, beta = -sign(alpha) ||x||).
  R is normalised to a positive diagonal, which makes it unique for a
  full-rank B; a diagonal entry below 1e-14 * max_j R_jj is raised to that
  floor (a reading: the paper does not say how rank deficiency is handled).
  A blocked (compact-WY) variant applies the same reflectors panel by panel.
* LSQR of Paige and Saunders (ACM TOMS 8, 1982): Golub-Kahan
  bidiagonalisation with x_0 = 0, no damping, and the stopping rules
    S1  ||r|| <= btol ||b|| + atol ||A|| ||x||
    S2  ||A^T r|| <= atol ||A|| ||r||
    S3  cond(A) >= conlim
  with ||A|| the Frobenius norm of the bidiagonal, ||x|| computed directly and
  cond(A) = ||A|| * sqrt(sum ||w_i / rho_i||^2); atol = btol = eta (Sec. 6).

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
import numpy as np

from . import philox


# ---------------------------------------------------------------- sketch
def count_sketch(J, s, kJ, seed):
    """B = S_k J for the count sketch: row h(i) of B accumulates
    sigma(i) * J[i, :] (rows summed in increasing i)."""
    m = J.shape[0]
    h, sig = philox.count_sketch_hash(m, s, kJ, seed)
    B = np.zeros((s, J.shape[1]))
    for i in range(m):
        B[h[i]] += sig[i] * J[i]
    return B


def gaussian_sketch_matrix(s, m, kJ, seed):
    return philox.gaussian_sketch(s, np.arange(m), kJ, seed)


def gaussian_sketch(J, s, kJ, seed):
    return gaussian_sketch_matrix(s, J.shape[0], kJ, seed) @ J


# ---------------------------------------------------------------- QR
def house(x):
    """Householder vector for x: returns (v, tau, beta) with v[0] = 1 and
    (I - tau v v^T) x = beta e_1."""
    alpha = x[0]
    tail = x[1:]
    sig = float(np.dot(tail, tail))
    v = x.copy()
    v[0] = 1.0
    if sig == 0.0:
        return v, 0.0, alpha
    norm = np.sqrt(alpha * alpha + sig)
    beta = -norm if alpha >= 0 else norm
    v[1:] = tail / (alpha - beta)
    tau = (beta - alpha) / beta
    return v, tau, beta


RANK_FLOOR = 1e-14


def normalise_r(R):
    """Flip rows to a positive diagonal, then floor tiny pivots.
    Returns (R, rank_flag)."""
    R = np.triu(R).copy()
    neg = np.diag(R) < 0
    R[neg, :] *= -1.0
    d = np.diag(R).copy()
    floor = RANK_FLOOR * d.max() if d.size else 0.0
    low = d < floor
    if low.any():
        R[np.nonzero(low)[0], np.nonzero(low)[0]] = floor
    return R, bool(low.any())


def qr_r_unblocked(B):
    """R of B = QR by one Householder reflector per column."""
    A = np.array(B, dtype=np.float64, copy=True)
    s, n = A.shape
    for j in range(n):
        v, tau, beta = house(A[j:, j])
        if tau != 0.0 and j + 1 < n:
            w = v @ A[j:, j + 1:]
            A[j:, j + 1:] -= tau * np.outer(v, w)
        A[j, j] = beta
        A[j + 1:, j] = 0.0
    return normalise_r(A[:n, :n])


def qr_r_blocked(B, nb=64):
    """Same reflectors as qr_r_unblocked, applied to the trailing matrix in
    compact-WY form: Q_panel = I - V T V^T (T upper triangular,
    T_jj = tau_j, T_{:j,j} = -tau_j T_{:j,:j} V_{:,:j}^T v_j)."""
    A = np.array(B, dtype=np.float64, copy=True)
    s, n = A.shape
    for j0 in range(0, n, nb):
        j1 = min(n, j0 + nb)
        w_ = j1 - j0
        V = np.zeros((s - j0, w_))
        taus = np.zeros(w_)
        for jj in range(w_):
            j = j0 + jj
            v, tau, beta = house(A[j:, j])
            if tau != 0.0 and j + 1 < j1:
                w = v @ A[j:, j + 1:j1]
                A[j:, j + 1:j1] -= tau * np.outer(v, w)
            A[j, j] = beta
            A[j + 1:, j] = 0.0
            V[jj:, jj] = v
            taus[jj] = tau
        if j1 < n:
            T = np.zeros((w_, w_))
            for jj in range(w_):
                T[jj, jj] = taus[jj]
                if jj:
                    T[:jj, jj] = -taus[jj] * (T[:jj, :jj] @ (V[:, :jj].T @ V[:, jj]))
            Wm = V.T @ A[j0:, j1:]
            A[j0:, j1:] -= V @ (T.T @ Wm)
    return normalise_r(A[:n, :n])


# ------------------------------------------------------- triangular solves
def solve_upper(R, b):
    """x with R x = b (back substitution)."""
    n = R.shape[0]
    x = np.zeros(n)
    for i in range(n - 1, -1, -1):
        x[i] = (b[i] - np.dot(R[i, i + 1:], x[i + 1:])) / R[i, i]
    return x


def solve_upper_t(R, b):
    """z with R^T z = b (forward substitution on the lower factor R^T)."""
    n = R.shape[0]
    z = np.zeros(n)
    for j in range(n):
        z[j] = (b[j] - np.dot(R[:j, j], z[:j])) / R[j, j]
    return z


# ---------------------------------------------------------------- LSQR
class LsqrResult:
    def __init__(self, x, itn, istop, normr, normar, normA, condA):
        self.x, self.itn, self.istop = x, itn, istop
        self.normr, self.normar, self.normA, self.condA = normr, normar, normA, condA


def lsqr(matvec, rmatvec, b, n, atol, btol, conlim, iter_lim):
    """Paige-Saunders LSQR for min ||A x - b||, x_0 = 0, no damping.
    istop: 0 b = 0 or A^T b = 0, 1 S1, 2 S2, 3 S3, 7 iteration limit."""
    x = np.zeros(n)
    beta = float(np.linalg.norm(b))
    normb = beta
    if beta == 0.0:
        return LsqrResult(x, 0, 0, 0.0, 0.0, 0.0, 0.0)
    u = b / beta
    v = rmatvec(u)
    alpha = float(np.linalg.norm(v))
    if alpha == 0.0:
        return LsqrResult(x, 0, 0, beta, 0.0, 0.0, 0.0)
    v = v / alpha
    w = v.copy()
    phibar, rhobar = beta, alpha
    sumsq = 0.0
    dd = 0.0
    itn, istop = 0, 7
    normr = beta
    normar = alpha * beta
    normA = condA = 0.0
    while itn < iter_lim:
        itn += 1
        # continue the bidiagonalisation
        u = matvec(v) - alpha * u
        beta = float(np.linalg.norm(u))
        if beta > 0.0:
            u = u / beta
        sumsq += alpha * alpha + beta * beta
        v = rmatvec(u) - beta * v
        alpha = float(np.linalg.norm(v))
        if alpha > 0.0:
            v = v / alpha
        # plane rotation eliminating the subdiagonal beta
        rho = float(np.hypot(rhobar, beta))
        c = rhobar / rho
        s = beta / rho
        theta = s * alpha
        rhobar = -c * alpha
        phi = c * phibar
        phibar = s * phibar
        # update x and w
        dk = w / rho
        x = x + phi * dk
        w = v - (theta / rho) * w
        dd += float(np.dot(dk, dk))
        normA = np.sqrt(sumsq)
        condA = normA * np.sqrt(dd)
        normr = phibar
        normar = phibar * alpha * abs(c)
        normx = float(np.linalg.norm(x))
        if normr <= btol * normb + atol * normA * normx:
            istop = 1
        elif normar <= atol * normA * normr:
            istop = 2
        elif condA >= conlim:
            istop = 3
        if istop != 7:
            break
    return LsqrResult(x, itn, istop, normr, normar, normA, condA)
