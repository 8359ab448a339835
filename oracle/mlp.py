"""Learned warm start: the network, its function-space loss and gradient, Adam,
and the feature Gram metric (an addition to the paper's method, which starts
Newton (Alg. 1, Alg. 2) from a fixed guess u_0; here u_0 = Phi c_0 with c_0
predicted from the PDE parameters).

Network  h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = W3 h2 + b3, with x,
the weights and h1, h2 rounded to bfloat16 before each product (the library's
storage format) and everything else in FP64 here.  The backward pass treats the
roundings as the identity (straight-through) and rounds the back-propagated
signals dY and dZ to bfloat16 at the same points as the forward pass does.

Loss  L = (1/B) sum_b r_b^T G r_b, r_b = y_b - t_b, with G block diagonal (one
block per subdomain and field, Sec. 2.2's indicator partition of unity makes
the function-space inner product block diagonal):
    G_(e,f) = (1/N) sum over evaluation points x owned by e of phi_ef(x) phi_ef(x)^T,
so r^T G r = (1/N) sum_x (u_r(x))^2, the mean square of the function u_r = Phi r.
G = None means G = I / n (plain mean square of the coefficients).

Adam (Kingma & Ba, 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps), b1 = 0.9, b2 = 0.999,
eps = 1e-8.

Initialisation: Glorot-uniform weights, W_l[i] = s_l (2u - 1) with u the
53-bit uniform of the Philox4x32-10 draw with counter (4, l, i, 0) and s_l =
sqrt(6 / (fan_in + fan_out)) in single precision; zero biases.

Function-space basis: the snapshots c_j are centred and orthonormalised in
the mean-square inner product of u = Phi c over evaluation points by modified
Gram-Schmidt with column pivoting (largest remaining norm first, Businger and
Golub 1965), the same column operations applied to the coefficient vectors;
the network regresses the coordinates, since the coefficients themselves
cancel by orders of magnitude.

Parity pins: finite differences of the unrounded network, the closed form of
Adam's first step, r^T G r against the mean square of the evaluated function,
|diag R| of the pivoted Gram-Schmidt against LAPACK's pivoted QR, and the
orthonormality and reconstruction properties of the basis.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
import numpy as np

from . import assemble as asm
from .philox import philox4x32_10, round_bf16, seed_key, uniform53

BLOCK = 64  # parameter blocks are padded to a multiple of this many entries


def layout(din, H, dout):
    """Offsets of W1 [H][din], b1 [H], W2 [H][H], b2 [H], W3 [dout][H], b3 [dout]
    in the flat parameter vector, and its length."""
    sizes = [H * din, H, H * H, H, dout * H, dout]
    off, o = [], 0
    for s in sizes:
        off.append(o)
        o += -(-s // BLOCK) * BLOCK
    return off, sizes, o


def unpack(w, din, H, dout):
    off, sizes, _ = layout(din, H, dout)
    blk = [np.asarray(w[o:o + s], dtype=np.float64) for o, s in zip(off, sizes)]
    return (blk[0].reshape(H, din), blk[1], blk[2].reshape(H, H), blk[3], blk[4].reshape(dout, H), blk[5])


def pack(parts, din, H, dout):
    off, sizes, total = layout(din, H, dout)
    w = np.zeros(total)
    for o, s, p in zip(off, sizes, parts):
        w[o:o + s] = np.asarray(p, dtype=np.float64).reshape(-1)
    return w


def init_params(din, H, dout, seed):
    """Glorot-uniform initial parameters (float32 values, returned as doubles)."""
    off, sizes, total = layout(din, H, dout)
    k0, k1 = seed_key(seed)
    w = np.zeros(total)
    fans = [(din, H), (H, H), (H, dout)]
    for l in range(3):
        n = sizes[2 * l]
        scale = np.sqrt(np.float32(6.0) / np.float32(fans[l][0] + fans[l][1]), dtype=np.float32)
        i = np.arange(n, dtype=np.uint64)
        x0, x1, _, _ = philox4x32_10(4, l, i, 0, k0, k1)
        u = (2.0 * uniform53(x0, x1) - 1.0).astype(np.float32)
        w[off[2 * l]:off[2 * l] + n] = (scale * u).astype(np.float32)
    return w


def _q(a, quantise):
    return round_bf16(a) if quantise else np.asarray(a, dtype=np.float64)


def forward(w, x, din, H, dout, quantise=True):
    """Returns (h1, h2, y) for a batch x [B][din]."""
    W1, b1, W2, b2, W3, b3 = unpack(w, din, H, dout)
    xq = _q(x, quantise)
    h1 = np.tanh(xq @ _q(W1, quantise).T + b1)
    h2 = np.tanh(_q(h1, quantise) @ _q(W2, quantise).T + b2)
    y = _q(h2, quantise) @ _q(W3, quantise).T + b3
    return h1, h2, y


def loss_and_grad(w, x, t, din, H, dout, G=None, gblk=0, quantise=True):
    """L and dL/dw (flat, same layout as w) for inputs x [B][din] and targets
    t [B][dout]; G is [dout/gblk][gblk][gblk] or None."""
    B = x.shape[0]
    W1, b1, W2, b2, W3, b3 = unpack(w, din, H, dout)
    h1, h2, y = forward(w, x, din, H, dout, quantise)
    r = y - t
    if G is None:
        Gr = r / dout
    else:
        nb = dout // gblk
        Gr = np.einsum("kij,bkj->bki", np.asarray(G, dtype=np.float64), r.reshape(B, nb, gblk)).reshape(B, dout)
    L = float(np.sum(r * Gr)) / B
    dY = 2.0 * Gr / B
    dYq = _q(dY, quantise)
    gW3 = dYq.T @ _q(h2, quantise)
    gb3 = dY.sum(axis=0)
    dZ2 = (dYq @ _q(W3, quantise)) * (1.0 - h2 * h2)
    dZ2q = _q(dZ2, quantise)
    gW2 = dZ2q.T @ _q(h1, quantise)
    gb2 = dZ2.sum(axis=0)
    dZ1 = (dZ2q @ _q(W2, quantise)) * (1.0 - h1 * h1)
    gW1 = _q(dZ1, quantise).T @ _q(x, quantise)
    gb1 = dZ1.sum(axis=0)
    return L, pack([gW1, gb1, gW2, gb2, gW3, gb3], din, H, dout)


def adam_step(w, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update at step number `step` (1-based); returns (w, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** step)
    vhat = v / (1.0 - b2 ** step)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v


def feature_gram(prob, X, starts):
    """G_(e,f) = (1/N) sum_{x in group e} phi_ef(x) phi_ef(x)^T for points X
    [N][d] grouped by owner (starts: G+1 group boundaries).  Returns
    [G*fields][M][M]."""
    N = X.shape[0]
    out = np.zeros((prob.G * prob.fields, prob.M, prob.M))
    for e in range(prob.G):
        Xe = X[starts[e]:starts[e + 1]]
        if Xe.shape[0] == 0:
            continue
        phi, _, _ = asm.feature_values(prob, np.full(Xe.shape[0], e, dtype=np.int64), Xe)
        for f in range(prob.fields):
            out[e * prob.fields + f] = phi[:, f, :].T @ phi[:, f, :] / N
    return out


def snapshot_values(prob, D, X):
    """Columns u(D_j)(x_q) / sqrt(N) stacked as [len][nsnap] (fields interleaved
    per point), the Euclidean product of two columns being the mean-square
    inner product."""
    from . import newton
    cols = [newton.evaluate(prob, d, X).reshape(-1) for d in D]
    return np.stack(cols, axis=1) / np.sqrt(X.shape[0])


def function_basis(prob, C, X, tol=1e-8):
    """Returns (mean [n], U [rank][n], Z [N][rank], diag R [rank])."""
    C = np.asarray(C, dtype=np.float64)
    N = C.shape[0]
    mean = C.mean(axis=0)
    D = C - mean
    V = snapshot_values(prob, D, X)
    Dc = D.T.copy()  # [n][N]
    rest = list(range(N))
    Z = np.zeros((N, N))
    U, diag = [], []
    norm0 = None
    for k in range(N):
        sq = {j: float(V[:, j] @ V[:, j]) for j in rest[k:]}
        best = max(range(k, N), key=lambda t: (sq[rest[t]], -t))
        rkk = np.sqrt(sq[rest[best]])
        if norm0 is None:
            norm0 = rkk
        if not rkk > tol * norm0 or rkk == 0.0:
            break
        rest[k], rest[best] = rest[best], rest[k]
        p = rest[k]
        V[:, p] /= rkk
        Dc[:, p] /= rkk
        Z[p, k] = rkk
        U.append(Dc[:, p].copy())
        diag.append(rkk)
        for j in rest[k + 1:]:
            r = float(V[:, p] @ V[:, j])
            Z[j, k] = r
            V[:, j] -= r * V[:, p]
            Dc[:, j] -= r * Dc[:, p]
    r = len(U)
    return mean, np.array(U).reshape(r, -1), Z[:, :r], np.array(diag)
