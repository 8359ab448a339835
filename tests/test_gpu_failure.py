"""Failure paths of the solvers and of the bounded device waits, provoked
without faulting the GPU: an iteration cap, a non-finite initial guess, a
rank-deficient system, and waits that are told to give up at once (the
problem's wait limit), after which the next call must succeed."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import rfm_workloads as W  # noqa: E402
from oracle import newton  # noqa: E402
from oracle.problem import Problem as OProblem  # noqa: E402


@pytest.fixture(scope="module")
def rfm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_04170_gb300 import build, rfm as _rfm
    build.build()
    return _rfm


def test_iteration_cap_returns_enoconv_with_the_iterate(rfm):
    desc = W.small_2d()
    gp = rfm.Problem(desc)
    c, info = gp.rfm_ipn_solve(W.solve_opts(max_outer=1))
    assert info["status"] == rfm.RFM_ENOCONV and info["outer_iters"] == 1
    co, io = newton.ipn(OProblem(desc), W.solve_opts(max_outer=1))
    assert torch.count_nonzero(c).item() > 0  # the iterate after one step is written
    X = W.eval_grid(desc)
    u = gp.rfm_eval(c, torch.as_tensor(X, device="cuda")).cpu().numpy()
    uo = newton.evaluate(OProblem(desc), co, X)
    assert newton.rel_l2(u, uo) < 1e-7
    c2, info2 = gp.rfm_amipn_solve(W.solve_opts(max_outer=1, m_max=1))
    assert info2["status"] == rfm.RFM_ENOCONV and info2["outer_iters"] == 1


def test_non_finite_initial_guess_returns_enonfinite(rfm):
    desc = W.small_2d()
    gp = rfm.Problem(desc)
    c0 = torch.zeros(gp.n, dtype=torch.float64, device="cuda")
    c0[3] = float("nan")
    for solve in (gp.rfm_ipn_solve, gp.rfm_amipn_solve):
        c, info = solve(W.solve_opts(), c0)
        assert info["status"] == rfm.RFM_ENONFINITE
        assert not np.isfinite(info["final_resid"])
    # the problem stays usable: a solve from zero converges as usual
    c, info = gp.rfm_ipn_solve(W.solve_opts())
    assert info["status"] == rfm.RFM_OK


def test_rank_deficient_system_sets_the_rank_flag(rfm):
    """21 collocation rows for 40 features: the sketch has rank <= 21, so the
    QR floors pivots (Sec. 4.1 leaves rank deficiency open; both sides floor
    pivots below 1e-14 max R_jj and raise the flag)."""
    desc = W.problem(2, (1, 1), 40, (3, 3), (3, 3), (3, 3))
    gp = rfm.Problem(desc)
    c, info = gp.rfm_ipn_solve(W.solve_opts())
    co, io = newton.ipn(OProblem(desc), W.solve_opts())
    assert io.rank_flag and info["rank_flag"] == 1
    assert info["status"] == rfm.RFM_OK
    assert (info["outer_iters"], info["n_jac"]) == (io.outer_iters, io.n_jac)


def test_wait_limit_gives_up_then_recovers(rfm):
    """Every bounded flag wait of the problem is told to give up at once: the
    triangular solve (block flags) and the QR (grid barriers of the panel
    factorisation) report RFM_ETIMEOUT and return; with the default limit
    restored the same calls succeed and give the results of an undisturbed
    problem."""
    desc = W.small_3d(M=48)  # n = 384: six 64-row blocks in the triangular solve
    c = torch.as_tensor(W.random_coeffs(8 * 48, seed=3, scale=0.1), device="cuda")
    ref = rfm.Problem(desc)
    ref.rfm_assemble(c)
    ref.rfm_sketch("count", 3 * ref.n, 0, copy_out=False)
    Rref, _ = ref.rfm_qr()
    b = torch.as_tensor(np.random.default_rng(1).standard_normal(ref.n), device="cuda")
    x_ref = ref.rfm_trsv(b)
    xt_ref = ref.rfm_trsv(b, trans=1)

    gp = rfm.Problem(desc)
    gp.rfm_assemble(c)
    gp.rfm_sketch("count", 3 * gp.n, 0, copy_out=False)
    gp.rfm_set_wait_limit(-1)
    with pytest.raises(rfm.RfmError) as e:
        gp.rfm_qr()
    assert e.value.status == rfm.RFM_ETIMEOUT
    gp.rfm_set_wait_limit(0)
    gp.rfm_sketch("count", 3 * gp.n, 0, copy_out=False)
    R, _ = gp.rfm_qr()
    assert torch.equal(R, Rref)
    gp.rfm_set_wait_limit(-1)
    for trans in (0, 1):
        with pytest.raises(rfm.RfmError) as e:
            gp.rfm_trsv(b, trans=trans)
        assert e.value.status == rfm.RFM_ETIMEOUT
    gp.rfm_set_wait_limit(1 << 20)
    assert torch.equal(gp.rfm_trsv(b), x_ref)
    gp.rfm_set_wait_limit(0)
    assert torch.equal(gp.rfm_trsv(b, trans=1), xt_ref)
    # a solve on the same problem after the timeouts
    cs, info = gp.rfm_ipn_solve(W.solve_opts())
    assert info["status"] == rfm.RFM_OK
