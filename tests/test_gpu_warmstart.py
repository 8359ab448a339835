"""Learned warm start on the GPU (rfm_mlp_*, rfm_feature_gram) against the
oracle (oracle/mlp.py), plus the end-to-end effect on Newton.

Tolerances.  Both sides round the same quantities to bfloat16; the GPU sums
their products in FP32 and takes tanh in FP32, the oracle in FP64.  Almost
every entry therefore agrees to FP32 accuracy; an entry whose FP32 and FP64
values straddle a bfloat16 rounding midpoint (probability ~ 2^-24 / 2^-9 per
entry) rounds to the neighbouring bfloat16, one ulp = 2^-8 relative, and that
propagates.  Where a rounded signal is itself a sum with cancellation (the
metric's G r), its FP32 relative error and with it the flip rate grow, and each
flip moves a whole row of the next weight gradient by ~2^-8 of one term.  The
tests bound every entry, relative to the largest reference entry of its
block: all within 2^-9, and all but a counted 2% within 2^-12 (measured on a
GB300: at most 0.5% of the entries above 2^-12, none above 2^-11); a wrong
index, sign, term or operand moves entries by O(1).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import rfm_workloads as W  # noqa: E402
from oracle import mlp as omlp  # noqa: E402
from oracle import newton  # noqa: E402
from oracle.problem import Problem as OProblem  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_04170_gb300 import build
    build.build()


def R():
    from paper_2510_04170_gb300 import rfm
    return rfm


DIMS = (3, 96, 200)  # ragged against the 64-wide tiles
SEED = 7


def _inputs(B=37, seed=1):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, (B, DIMS[0])).astype(np.float32)
    t = (0.3 * rng.standard_normal((B, DIMS[2]))).astype(np.float32)
    return x, t


def _f32(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def _close(gpu, ref, bulk, flips=0.02, cap=2.0 ** -9):
    """Element by element, relative to the largest reference entry: every
    entry within `cap` (the reach of a few propagated one-ulp bf16 rounding
    flips, 2^-8 each, diluted through the next layer's sum), and all but a
    counted fraction `flips` of the entries within `bulk`."""
    gpu, ref = np.asarray(gpu, np.float64), np.asarray(ref, np.float64)
    scale = max(np.max(np.abs(ref)), 1e-30)
    err = np.abs(gpu - ref) / scale
    assert np.all(err <= cap), (err.max(), cap)
    over = int(np.count_nonzero(err > bulk))
    assert over <= flips * err.size, (over, err.size, bulk)


def test_init_bit_exact():
    net = R().MLP(*DIMS, seed=SEED)
    w, offs = net.params()
    ref_off, _, total = omlp.layout(*DIMS)
    assert offs == ref_off and net.num_params == total
    assert np.array_equal(w.cpu().numpy().astype(np.float64), omlp.init_params(*DIMS, SEED))


def test_forward_parity():
    net = R().MLP(*DIMS, seed=SEED)
    x, _ = _inputs()
    y = net.forward(_f32(x)).cpu().numpy()
    _, _, yref = omlp.forward(omlp.init_params(*DIMS, SEED), x.astype(np.float64), *DIMS)
    _close(y, yref, 2.0 ** -12)


@pytest.mark.parametrize("metric", ["identity", "blocks"])
def test_gradient_parity(metric):
    net = R().MLP(*DIMS, seed=SEED)
    x, t = _inputs()
    if metric == "identity":
        G, gblk, Gt = None, 0, None
    else:
        gblk = 40
        rng = np.random.default_rng(3)
        A = rng.standard_normal((DIMS[2] // gblk, gblk, gblk))
        G = (np.einsum("kij,klj->kil", A, A) / gblk).astype(np.float32)
        Gt = _f32(G)
    g, L = net.gradient(_f32(x), _f32(t), G=Gt, gblk=gblk)
    Lref, gref = omlp.loss_and_grad(omlp.init_params(*DIMS, SEED), x.astype(np.float64), t.astype(np.float64), *DIMS,
                                    G=None if G is None else G.astype(np.float64), gblk=gblk)
    assert L == pytest.approx(Lref, rel=1e-5)
    g = g.cpu().numpy()
    off, sizes, _ = omlp.layout(*DIMS)
    for o, s in zip(off, sizes):
        _close(g[o:o + s], gref[o:o + s], 2.0 ** -12)


def test_adam_first_step_closed_form():
    """One training step from zero moments moves each weight by
    lr * g / (|g| + eps) (Adam's first step: m_hat = g, v_hat = g^2) where the
    oracle gradient is clearly nonzero; the step is insensitive to the
    gradient's own rounding there."""
    net = R().MLP(*DIMS, seed=SEED)
    x, t = _inputs()
    lr = 1e-3
    net.train(_f32(x), _f32(t), 1, lr)
    w1 = net.params()[0].cpu().numpy().astype(np.float64)
    w0 = omlp.init_params(*DIMS, SEED)
    _, gref = omlp.loss_and_grad(w0, x.astype(np.float64), t.astype(np.float64), *DIMS)
    big = np.abs(gref) > 1e-2 * np.max(np.abs(gref))
    step = w1 - w0
    gb = gref[big]
    expect = -lr * gb / (np.abs(gb) + 1e-8)
    assert np.all(np.abs(step[big] - expect) <= 1e-6 * lr + 4 * 2.0 ** -24 * np.abs(w0[big]))
    assert np.all(np.abs(step) <= lr * (1 + 1e-6) + 4 * 2.0 ** -24 * np.abs(w0))


def test_training_reduces_loss():
    """400 Adam steps fit a smooth target the network can represent (the FP64
    oracle reaches 0.3% of the initial loss on the same data)."""
    net = R().MLP(*DIMS, seed=SEED)
    rng = np.random.default_rng(1)
    x = rng.uniform(-1, 1, (64, DIMS[0]))
    P = rng.standard_normal((DIMS[0], 8))
    Q = rng.standard_normal((8, DIMS[2])) / np.sqrt(8)
    t = 0.5 * np.sin(x @ P) @ Q
    _, L0 = net.gradient(_f32(x), _f32(t))
    L = net.train(_f32(x), _f32(t), 400, 2e-3)
    assert L < 0.02 * L0


def test_feature_gram_parity():
    desc = W.small_3d(M=40, nsub=(2, 2, 1))
    gp = R().Problem(desc)
    op = OProblem(desc)
    X = W.eval_grid(desc, per_axis=5)
    e = newton.owner(op, X)
    order = np.argsort(e, kind="stable")
    starts = np.concatenate([[0], np.cumsum(np.bincount(e, minlength=op.G))])
    Gg = R().rfm_feature_gram(gp, torch.as_tensor(X[order], device="cuda"), starts).cpu().numpy()
    Gr = omlp.feature_gram(op, X[order], starts)
    # FP32 sums of at most npts products of |phi| <= 1 scaled by 1/npts
    assert np.max(np.abs(Gg - Gr)) <= 1e-6 * np.max(np.abs(Gr))


def test_function_basis_parity():
    desc = W.small_2d(M=16)
    op = OProblem(desc)
    C = np.random.default_rng(9).standard_normal((7, op.n))
    C[-1] = C[0] + C[1] - C[2]
    X = W.eval_grid(desc, per_axis=6)
    mean, U, Z = R().rfm_function_basis(R().Problem(desc), torch.as_tensor(C, device="cuda"),
                                        torch.as_tensor(X, device="cuda"), tol=1e-9)
    mr, Ur, Zr, _ = omlp.function_basis(op, C, X, tol=1e-9)
    assert U.shape[0] == Ur.shape[0] == 5
    assert np.max(np.abs(mean.cpu().numpy() - mr)) <= 1e-15 * np.max(np.abs(C))
    # same pivots (no near-ties in this data); FP64 Gram-Schmidt differences grow with the conditioning
    assert np.max(np.abs(Z.cpu().numpy() - Zr)) <= 1e-10 * np.max(np.abs(Zr))
    assert np.max(np.abs(U.cpu().numpy() - Ur)) <= 1e-9 * np.max(np.abs(Ur))


def test_basis_combine_definition():
    rng = np.random.default_rng(4)
    n, r, B = 1000, 7, 5
    mean, U = rng.standard_normal(n), rng.standard_normal((r, n))
    y = rng.standard_normal((B, r)).astype(np.float32)
    c = R().rfm_basis_combine(torch.as_tensor(mean, device="cuda"), torch.as_tensor(U, device="cuda"),
                              torch.as_tensor(y, device="cuda"), 0.5).cpu().numpy()
    ref = mean + 0.5 * y.astype(np.float64) @ U
    assert np.max(np.abs(c - ref)) <= 1e-14 * (np.abs(mean) + 0.5 * np.abs(y.astype(np.float64)) @ np.abs(U)).max()


def test_warm_start_reduces_newton_work():
    """Small 2D family of the learned-warm-start workload: on held-out
    parameters the network's u_0 must lie within 10% of the solution, Newton
    from it must need no more Jacobians than from c_0 = 0, and both starts
    must reach the same solution."""
    from paper_2510_04170_gb300 import warmstart

    def base(kappa, amp, freq):
        return W.problem(2, (2, 2), 64, (12, 12), (12, 12), (12, 12), pde_kind=3, pde_params=[kappa, amp, freq])

    out = warmstart.run(n_train=48, n_test=8, solver="ipn", precision=0, steps=2000, base=base)
    m = out["mean"]
    assert m["rel_guess"] < 0.1, m
    assert all(r["nj_warm"] <= r["nj_zero"] for r in out["rows"]), out["rows"]
    assert m["rel_warm_vs_zero"] < 1e-6, m
