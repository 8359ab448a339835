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


def solve(desc, opts, c0=None, solver="ipn"):
    gp = rfm.Problem(desc)
    c0t = None if c0 is None else torch.as_tensor(np.asarray(c0, dtype=np.float64), device="cuda")
    t0 = time.perf_counter()
    c, info = getattr(gp, f"rfm_{solver}_solve")(opts, c0t)
    torch.cuda.synchronize()
    info["wall_s"] = time.perf_counter() - t0
    return gp, c, info


def train_warm_start(train_params, train_c, metric_desc, hidden=256, steps=3000, lr=1e-3, seed=1, tol=1e-6):
    """Builds the warm start (rfm_warmstart_*) from training solutions and
    trains it for `steps` full-batch Adam steps; returns it with the losses."""
    gp = rfm.Problem(metric_desc)
    X = torch.as_tensor(W.eval_grid(metric_desc), device="cuda")
    C = torch.as_tensor(np.asarray(train_c, dtype=np.float64), device="cuda")
    P = torch.as_tensor(np.asarray(train_params, dtype=np.float64), device="cuda")
    ws = rfm.WarmStart(gp, C, P, X, tol=tol, hidden=hidden, seed=seed)
    ws.losses = []
    done = 0
    while done < steps:
        k = min(500, steps - done)
        ws.losses.append(ws.train(k, lr))
        done += k
    return ws


def run(n_train=512, n_test=128, solver="ipn", precision=2, steps=3000, base=None, seed_train=1, seed_test=10001):
    """Full experiment: solve n_train instances for targets, train, then solve
    n_test held-out instances from c_0 = 0 and from the network's c_0."""
    opts = W.solve_opts(precision=precision)
    ptrain = sample_params(n_train, seed_train)
    ptest = sample_params(n_test, seed_test)
    targets = []
    t0 = time.perf_counter()
    for prm in ptrain:
        _, c, info = solve(family_desc(prm, base), opts, solver=solver)
        targets.append(c.cpu().numpy())
    t_data = time.perf_counter() - t0
    metric_desc = family_desc(ptrain[0], base)
    t0 = time.perf_counter()
    ws = train_warm_start(ptrain, np.stack(targets), metric_desc, steps=steps)
    t_train = time.perf_counter() - t0
    c0s = ws.predict(torch.as_tensor(ptest, device="cuda")).cpu().numpy()
    rows = []
    for prm, c0 in zip(ptest, c0s):
        d = family_desc(prm, base)
        gz, cz, iz = solve(d, opts, solver=solver)
        gw, cw, iw = solve(d, opts, c0=c0, solver=solver)
        Xe = torch.as_tensor(W.eval_grid(d), device="cuda")
        uz = gz.rfm_eval(cz, Xe).cpu().numpy()
        uw = gw.rfm_eval(cw, Xe).cpu().numpy()
        u0 = gw.rfm_eval(torch.as_tensor(c0, device="cuda"), Xe).cpu().numpy()
        rows.append(dict(it_zero=iz["outer_iters"], it_warm=iw["outer_iters"], nj_zero=iz["n_jac"], nj_warm=iw["n_jac"],
                         t_zero=iz["t_total"], t_warm=iw["t_total"], res_zero=iz["final_resid"],
                         res_warm=iw["final_resid"],
                         rel_warm_vs_zero=float(np.linalg.norm(uw - uz) / np.linalg.norm(uz)),
                         rel_guess=float(np.linalg.norm(u0 - uz) / np.linalg.norm(uz))))
    agg = {k: float(np.mean([r[k] for r in rows])) for k in rows[0]}
    return dict(n_train=n_train, n_test=n_test, solver=solver, t_data_s=t_data, t_train_s=t_train, rank=ws.rank,
                final_loss=ws.losses[-1], mean=agg, rows=rows)
