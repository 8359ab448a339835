"""Whole solves on the GPU against whole oracle solves of the same instances,
stored by the committed scripts in tests/golden/ (they call only the oracle):

  * the steady Gray-Scott system (two fields, 2x2x2 subdomains, M = 64 per
    field), IPN and AMIPN with inner cap 5;
  * the three further operators of Sec. 3.2 / Sec. 6.2 (nonlinear Helmholtz,
    -div((1+u^2) grad u), -div((1+|grad u|^2) grad u)) at 2x2x2 subdomains,
    M = 100, IPN and AMIPN;
  * the diffusion-reaction equation on the unit ball (Sec. 6.2: masked grids,
    Fibonacci boundary points), 2x2x2 subdomains, M = 100, AMIPN and IPN;
  * the 3D benchmark solve (4x4x4 subdomains, M = 512, n = 32,768, Gaussian
    sketch of 65,536 rows) in the configuration the benchmark times
    (tensor-core sketch and QR update), IPN.

Each must take the same outer iterations, Jacobian evaluations and LSQR steps
as the oracle, and give u within 1e-7 (relative L2 on the evaluation grid)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import rfm_workloads as W  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def rfm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_04170_gb300 import build, rfm as _rfm
    build.build()
    return _rfm


def _check(gp, c, info, u_ref, it, nj, lsqr, X):
    assert info["status"] == 0, info
    assert (info["outer_iters"], info["n_jac"]) == (int(it), int(nj))
    assert info["lsqr_iters_total"] == int(np.sum(lsqr))
    u = gp.rfm_eval(c, torch.as_tensor(X, device="cuda")).cpu().numpy()
    assert np.linalg.norm(u - u_ref) <= 1e-7 * np.linalg.norm(u_ref), np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref)


@pytest.mark.parametrize("solver", ["ipn", "amipn"])
@pytest.mark.parametrize("precision", [0, 2])
def test_grayscott_solve_matches_oracle(rfm, solver, precision):
    ref = np.load(os.path.join(GOLDEN, "grayscott_oracle.npz"))
    desc = W.grayscott_small()
    gp = rfm.Problem(desc)
    c, info = getattr(gp, f"rfm_{solver}_solve")(W.solve_opts(m_max=5, precision=precision))
    _check(gp, c, info, ref[f"{solver}_u"], ref[f"{solver}_outer_iters"], ref[f"{solver}_n_jac"],
           ref[f"{solver}_lsqr_iters"], W.eval_grid(desc))


@pytest.mark.parametrize("solver", ["ipn", "amipn"])
@pytest.mark.parametrize("kind", [4, 5, 6])
def test_operator_solve_matches_oracle(rfm, kind, solver):
    ref = np.load(os.path.join(GOLDEN, "operators_oracle.npz"))
    desc = W.operator_small(kind)
    gp = rfm.Problem(desc)
    c, info = getattr(gp, f"rfm_{solver}_solve")(W.solve_opts())
    key = f"k{kind}_{solver}"
    _check(gp, c, info, ref[key + "_u"], ref[key + "_outer_iters"], ref[key + "_n_jac"], ref[key + "_lsqr_iters"],
           W.eval_grid(desc, per_axis=4))


def test_benchmark_solve_matches_oracle(rfm):
    path = os.path.join(GOLDEN, "c2_ipn_oracle.npz")
    if not os.path.exists(path):
        pytest.skip("c2_ipn_oracle.npz not generated (tests/golden/make_c2_ipn_oracle.py)")
    ref = np.load(path)
    desc = W.config_c2()
    gp = rfm.Problem(desc)
    c, info = gp.rfm_ipn_solve(W.opts_c2(precision=2))
    _check(gp, c, info, ref["u"], ref["outer_iters"], ref["n_jac"], ref["lsqr_iters"], W.eval_grid(desc))


@pytest.mark.parametrize("solver", ["amipn", "ipn"])
def test_ball_solve_matches_oracle(rfm, solver):
    """Diffusion-reaction on the unit ball (Sec. 6.2): masked grids and
    Fibonacci boundary points."""
    ref = np.load(os.path.join(GOLDEN, "ball_oracle.npz"))
    desc = W.ball(100, 10, 2000)
    gp = rfm.Problem(desc)
    c, info = getattr(gp, f"rfm_{solver}_solve")(W.solve_opts())
    _check(gp, c, info, ref[f"{solver}_u"], ref[f"{solver}_outer_iters"], ref[f"{solver}_n_jac"],
           ref[f"{solver}_lsqr_iters"], ref["X"])
