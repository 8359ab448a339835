"""Parity at the full C2 size (n = 32,768 unknowns, m = 124,416 rows, Gaussian
sketch s = 65,536) in the configuration the benchmark times (precision 2:
tensor-core sketch and QR update), on outputs the oracle computes one by one
(sampled Jacobian rows, sampled sketch entries) and on properties that hold at
any size (the QR's Gram identity and column norms).  A whole oracle solve at
this size takes hours, so the solve itself is held to the smaller parity
tests and to these step checks."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import rfm_workloads as W  # noqa: E402
from oracle import assemble as asm  # noqa: E402
from oracle import philox  # noqa: E402
from oracle.problem import Problem as OProblem  # noqa: E402

U = 2.0 ** -53


@pytest.fixture(scope="module")
def c2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_04170_gb300 import build, rfm
    build.build()
    desc = W.config_c2()
    gp = rfm.Problem(desc)
    op = OProblem(desc)
    c = W.random_coeffs(op.n, seed=21, scale=1e-2)
    gp.rfm_set_precision(2)
    F, lam = gp.rfm_assemble(torch.as_tensor(c, device="cuda"))
    return desc, gp, op, c, F.cpu().numpy()


def test_sizes_features_points_bit_exact(c2):
    desc, gp, op, c, _ = c2
    assert (gp.m, gp.n, gp.m_int, gp.m_iface) == (op.m, op.n, op.m_int, op.m_iface) == (124416, 32768, op.m_int,
                                                                                          op.m_iface)
    f = gp.rfm_get_features().cpu().numpy().reshape(op.G, op.fields, op.M, 4)
    assert np.array_equal(f[..., : op.d + 1], op.feats)
    pts = gp.rfm_get_points().cpu().numpy()[:, : op.d]
    assert np.array_equal(pts, op.rx)


def test_sampled_jacobian_rows(c2):
    desc, gp, op, c, F = c2
    rows = np.sort(np.random.default_rng(5).choice(op.m, 2048, replace=False))
    Jp, Js, blk = gp.rfm_get_jacobian()
    idx = torch.as_tensor(rows, device="cuda")
    Jp = Jp[idx].cpu().numpy()
    Fo, Jpo, Jso, e0, e1 = asm.assemble_rows(op, c, rows)
    lamo = asm.row_scale(Jpo, Jso)
    assert np.array_equal(blk[idx].cpu().numpy()[:, 0], e0)
    assert np.max(np.abs(Jp - lamo[:, None] * Jpo)) <= 1e-12 * 100.0
    iface = rows[(rows >= op.m_int) & (rows < op.m_int + op.m_iface)]
    if iface.size:
        sel = np.searchsorted(rows, iface)
        Js = Js[torch.as_tensor(iface - op.m_int, device="cuda")].cpu().numpy()
        assert np.max(np.abs(Js - lamo[sel, None] * Jso[sel])) <= 1e-12 * 100.0
    Fs = lamo * Fo
    assert np.max(np.abs(F[rows] - Fs)) <= 1e-12 * max(1.0, np.abs(Fs).max())


def test_sampled_sketch_entries_and_qr_properties(c2):
    desc, gp, op, c, _ = c2
    s, kJ = 65536, 0
    Bt = gp.rfm_sketch("gauss", s, kJ)  # [n][s]: column j of B contiguous
    rng = np.random.default_rng(9)
    W_ = op.W
    # B[r, j] = sum_i S[r, i] J[i, j] over the rows i touching column j's block
    for b in (0, 37, op.G - 1):
        rows = np.nonzero((op.re0 == b) | (op.re1 == b))[0]
        Fo, Jpo, Jso, e0, e1 = asm.assemble_rows(op, c, rows)
        lamo = asm.row_scale(Jpo, Jso)
        Jb = np.where((e0 == b)[:, None], Jpo, Jso) * lamo[:, None]
        srows = np.sort(rng.choice(s, 16, replace=False))
        S = philox.gaussian_sketch_rows(srows, rows, kJ, desc["seed"])
        cols = b * W_ + np.sort(rng.choice(W_, 4, replace=False))
        got = Bt[torch.as_tensor(cols, device="cuda")][:, torch.as_tensor(srows, device="cuda")].cpu().numpy().T
        ref = S @ Jb[:, cols - b * W_]
        # FP64 product bound K u |S||J|, plus the assembly tolerance (1e-12 of the
        # row maximum 100 per J entry, tested above) carried through |S|
        bound = 2 * rows.size * U * (np.abs(S) @ np.abs(Jb[:, cols - b * W_])) + 1e-10 * np.abs(S).sum(axis=1)[:, None]
        assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) / bound)
    # QR of the sketch: R^T R = B^T B and |R e_j| = |B e_j| on sampled columns
    # (Householder backward error, the same bound as the smaller QR tests)
    cols = np.sort(rng.choice(op.n, 12, replace=False))
    Bc = Bt[torch.as_tensor(cols, device="cuda")].cpu().numpy()  # [12][s]
    del Bt
    R, flag = gp.rfm_qr()  # [n][n] column-major: R[j] is column j
    Rc = R[torch.as_tensor(cols, device="cuda")].cpu().numpy()  # [12][n]
    dmax = float(torch.max(torch.diagonal(R)).item())
    del R
    keep = [k for k, j in enumerate(cols) if Rc[k, j] > 1e-12 * dmax]  # unfloored pivots
    assert len(keep) >= 8
    for a in keep:
        na = np.linalg.norm(Bc[a])
        assert abs(np.linalg.norm(Rc[a]) - na) <= 1e-14 * s * na
        for b_ in keep:
            gram = float(np.dot(Bc[a].astype(np.longdouble), Bc[b_].astype(np.longdouble)))
            rr = float(np.dot(Rc[a].astype(np.longdouble), Rc[b_].astype(np.longdouble)))
            assert abs(rr - gram) <= 1e-14 * s * na * np.linalg.norm(Bc[b_])


@pytest.mark.parametrize("precision", [0, 2])
def test_c5_instance_solve_matches_oracle(precision):
    """A whole IPN solve at the C5 size (n = 4,096) against the oracle's solve
    of the same instance, stored by tests/golden/make_c5_ipn_oracle.py: equal
    outer iterations, Jacobian evaluations and LSQR steps, and u within 1e-7
    (relative L2 on the evaluation grid)."""
    import os
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_04170_gb300 import build, rfm
    build.build()
    ref = np.load(os.path.join(os.path.dirname(__file__), "golden", "c5_ipn_oracle.npz"))
    desc = W.config_c5(*ref["params"])
    gp = rfm.Problem(desc)
    c, info = gp.rfm_ipn_solve(W.solve_opts(precision=precision))
    assert info["outer_iters"] == int(ref["outer_iters"]) and info["n_jac"] == int(ref["n_jac"])
    assert info["lsqr_iters_total"] == int(ref["lsqr_iters"].sum())
    u = gp.rfm_eval(c, torch.as_tensor(W.eval_grid(desc), device="cuda")).cpu().numpy()
    assert np.linalg.norm(u - ref["u"]) <= 1e-7 * np.linalg.norm(ref["u"])
