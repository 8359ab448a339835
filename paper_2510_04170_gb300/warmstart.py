"""Learned warm start for the RFM Newton solvers (an addition to the paper's
method, which starts from a fixed guess): an MLP maps PDE parameters to the
initial coefficient vector c_0, trained on converged solutions produced by the
solver itself.  The coefficient vectors cancel by orders of magnitude, so the
network regresses their coordinates in a basis of the training solutions that
is orthonormal in u-space (rfm_function_basis); c_0 = cbar + sum z_k U_k is
formed in FP64.  c_0 = 0 remains the fallback; the final Newton residual judges
the result.

Family (rfm_workloads.config_c5): -div(a grad u) + kappa u^3 = A prod sin(q pi x_d)
on [0,1]^3, a = 1 + 0.5 sin(2 pi x), zero Dirichlet data, 2x2x2 subdomains,
M = 512 (n = 4,096); parameters kappa ~ U[0.1, 10], A ~ U[0.5, 2], q ~ U{1..4}."""
import time

import numpy as np
import torch

import rfm_workloads as W

from . import rfm


def sample_params(count, seed):
    rng = np.random.default_rng(seed)
    kappa = rng.uniform(0.1, 10.0, count)
    amp = rng.uniform(0.5, 2.0, count)
    freq = rng.integers(1, 5, count).astype(np.float64)
    return np.stack([kappa, amp, freq], axis=1)


def family_desc(params, base=None):
    kappa, amp, freq = (float(v) for v in params)
    d = base(kappa, amp, freq) if base else W.config_c5(kappa, amp, freq)
    return d


def grouped_eval_points(desc, per_axis=10):
    """Cell-centred evaluation grid grouped by owning subdomain, with the
    group boundaries (G+1 entries)."""
    X = W.eval_grid(desc, per_axis)
    d = desc["dim"]
    N = desc["nsub"][:d]
    e = np.zeros(X.shape[0], dtype=np.int64)
    for b in range(d):
        lo, hi = desc["lo"][b], desc["hi"][b]
        t = np.clip(np.floor((X[:, b] - lo) / (hi - lo) * N[b]).astype(np.int64), 0, N[b] - 1)
        e = e * N[b] + t
    order = np.argsort(e, kind="stable")
    counts = np.bincount(e, minlength=int(np.prod(N)))
    starts = np.concatenate([[0], np.cumsum(counts)])
    return X[order], starts


def train_warm_start(train_params, train_c, metric_desc, hidden=256, steps=3000, lr=1e-3, seed=1, tol=1e-6):
    """Builds the warm start (rfm_warmstart_*) from training solutions (CUDA
    tensor [N][n]) and trains it for `steps` full-batch Adam steps; returns it
    with the losses."""
    gp = rfm.Problem(metric_desc)
    X = torch.as_tensor(W.eval_grid(metric_desc), device="cuda")
    P = torch.as_tensor(np.asarray(train_params, dtype=np.float64), device="cuda")
    ws = rfm.WarmStart(gp, train_c.contiguous(), P, X, tol=tol, hidden=hidden, seed=seed)
    ws.losses = []
    done = 0
    while done < steps:
        k = min(500, steps - done)
        ws.losses.append(ws.train(k, lr))
        done += k
    return ws


def _timed(fn):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def run(n_train=512, n_test=128, solver="ipn", precision=2, steps=3000, base=None, streams=4, seed_train=1,
        seed_test=10001):
    """Full experiment: batch-solve n_train instances for the targets, train,
    then batch-solve the n_test held-out instances from c_0 = 0 and from the
    network's c_0 and compare Jacobian counts, times and solutions."""
    opts = W.solve_opts(precision=precision)
    ptrain = sample_params(n_train, seed_train)
    ptest = sample_params(n_test, seed_test)
    bt = rfm.Batch([family_desc(p, base) for p in ptrain], streams=streams)
    (ctrain, _, _), t_data = _timed(lambda: bt.solve(opts, solver=solver))
    bt.close()
    ws, t_train = _timed(lambda: train_warm_start(ptrain, torch.stack(ctrain), family_desc(ptrain[0], base),
                                                  steps=steps))
    c0, t_pred = _timed(lambda: ws.predict(torch.as_tensor(ptest, device="cuda")))
    be = rfm.Batch([family_desc(p, base) for p in ptest], streams=streams)
    (cz, iz, _), t_zero = _timed(lambda: be.solve(opts, solver=solver))
    (cw, iw, _), t_warm = _timed(lambda: be.solve(opts, solver=solver, c0=[c0[i] for i in range(n_test)]))
    rows = []
    for i, prm in enumerate(ptest):
        Xe = torch.as_tensor(W.eval_grid(family_desc(prm, base)), device="cuda")
        gp = be.problems[i]
        uz = gp.rfm_eval(cz[i], Xe).cpu().numpy()
        uw = gp.rfm_eval(cw[i], Xe).cpu().numpy()
        u0 = gp.rfm_eval(c0[i].contiguous(), Xe).cpu().numpy()
        rows.append(dict(it_zero=iz[i]["outer_iters"], it_warm=iw[i]["outer_iters"], nj_zero=iz[i]["n_jac"],
                         nj_warm=iw[i]["n_jac"], lsqr_zero=iz[i]["lsqr_iters_total"],
                         lsqr_warm=iw[i]["lsqr_iters_total"], res_zero=iz[i]["final_resid"],
                         res_warm=iw[i]["final_resid"],
                         rel_warm_vs_zero=float(np.linalg.norm(uw - uz) / np.linalg.norm(uz)),
                         rel_guess=float(np.linalg.norm(u0 - uz) / np.linalg.norm(uz))))
    agg = {k: float(np.mean([r[k] for r in rows])) for k in rows[0]}
    return dict(n_train=n_train, n_test=n_test, solver=solver, precision=precision, streams=streams,
                t_data_s=t_data, t_train_s=t_train, t_predict_s=t_pred, t_zero_s=t_zero, t_warm_s=t_warm,
                solves_per_s_zero=n_test / t_zero, solves_per_s_warm=n_test / (t_warm + t_pred), rank=ws.rank,
                final_loss=ws.losses[-1], mean=agg, rows=rows)
