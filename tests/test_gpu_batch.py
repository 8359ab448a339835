"""Batched solves (rfm_batch_*), the QR autotuner and the graph-replayed LSQR.

Every kernel is deterministic (fixed-order reductions, no atomics in the
arithmetic), so an instance solved inside a batch, on any stream and
concurrently with others, must reproduce the stand-alone solve bit for bit;
the stand-alone solve is itself held to the oracle by the parity tests."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import rfm_workloads as W  # noqa: E402
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


def _family(count=5):
    """Uneven instances of -div(a grad u) + kappa u^3 = f: 2D and 3D grids,
    M from 24 to 64, kappa from a seeded generator."""
    rng = np.random.default_rng(3)
    out = []
    for i in range(count):
        kappa = float(rng.uniform(0.1, 10.0))
        if i % 2 == 0:
            out.append(W.problem(2, (2 + i % 3, 2), 24 + 8 * i, (10, 10), (10, 10), (10, 10), pde_kind=2,
                                 pde_params=[kappa]))
        else:
            out.append(W.problem(3, (2, 2, 2), 32 + 8 * (i % 3), (5, 5, 5), (4, 4, 4), (4, 4, 4), pde_kind=2,
                                 pde_params=[kappa]))
    return out


def _single(desc, opts, solver="ipn"):
    gp = R().Problem(desc)
    c, info = getattr(gp, f"rfm_{solver}_solve")(opts)
    return c, info


@pytest.mark.parametrize("solver", ["ipn", "amipn"])
def test_batch_reproduces_single_solves(solver):
    descs = _family()
    opts = W.solve_opts(precision=0)
    b = R().Batch(descs, streams=3)
    cs, infos, tuned = b.solve(opts, solver=solver)
    assert tuned == [0] * len(descs)
    for d, c, info in zip(descs, cs, infos):
        c1, info1 = _single(d, opts, solver)
        assert torch.equal(c, c1)
        for k in ("outer_iters", "n_jac", "lsqr_iters_total", "lsqr_iters_max"):
            assert info[k] == info1[k], k
        assert info["final_resid"] == info1["final_resid"]


def test_batch_autotuned_precision_matches_single_solve():
    descs = _family(4)
    opts = W.solve_opts(precision=-1)
    b = R().Batch(descs, streams=2)
    cs, infos, tuned = b.solve(opts)
    assert set(tuned) <= {0, 2}
    for d, c, prec in zip(descs, cs, tuned):
        c1, _ = _single(d, W.solve_opts(precision=prec))
        assert torch.equal(c, c1)


def test_batch_instance_matches_oracle():
    desc = _family(1)[0]
    opts = W.solve_opts(precision=0)
    b = R().Batch([desc, _family(2)[1]], streams=2)
    cs, infos, _ = b.solve(opts)
    op = OProblem(desc)
    c_or, info_or = newton.ipn(op, opts)
    assert infos[0]["outer_iters"] == info_or.outer_iters and infos[0]["n_jac"] == info_or.n_jac
    X = W.eval_grid(desc)
    u = b.problems[0].rfm_eval(cs[0], torch.as_tensor(X, device="cuda")).cpu().numpy()
    assert newton.rel_l2(u, newton.evaluate(op, c_or, X)) <= 1e-7


def test_autotune_picks_the_fastest_probe():
    prec, cap, ms = R().rfm_autotune_qr(1536, 512)
    assert all(t > 0 for t in ms)
    best = int(np.argmin(ms))
    assert prec == (0 if best < 4 else 2)
    assert cap > 0
    assert R().rfm_autotune_qr(1536, 512) == (prec, cap, ms)  # cached


def test_graph_lsqr_matches_eager_lsqr():
    """Profiling switches LSQR to eager launches of the same kernels; the two
    must agree bit for bit."""
    lib = R().load()
    desc = _family(2)[1]
    opts = W.solve_opts(precision=0)
    c_graph, i_graph = _single(desc, opts)
    lib.rfm_profile_enable(0xFFFF)
    try:
        c_eager, i_eager = _single(desc, opts)
    finally:
        lib.rfm_profile_enable(0)
    assert torch.equal(c_graph, c_eager)
    assert i_graph["lsqr_iters_total"] == i_eager["lsqr_iters_total"]
