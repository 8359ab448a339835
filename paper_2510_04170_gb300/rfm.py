"""Thin ctypes binding of librfm (include/rfm.h).  Names mirror the C entry
points; every call only marshals arguments (torch tensors give device
pointers and streams) and raises RfmError on a non-OK status.  There is no
CPU path: loading fails loudly when the library is missing."""
import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librfm.so")

RFM_OK, RFM_EINVAL, RFM_ENOMEM, RFM_ECUDA, RFM_ENOCONV, RFM_ERANK, RFM_ENONFINITE, RFM_ETIMEOUT = range(8)
SKETCH = {"count": 0, "gauss": 1}
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ENOCONV", "ERANK", "ENONFINITE", "ETIMEOUT"]

EXPORTS = ["rfm_default_opts", "rfm_last_error", "rfm_problem_create", "rfm_problem_destroy", "rfm_problem_sizes",
           "rfm_get_features", "rfm_get_points", "rfm_assemble", "rfm_get_jacobian", "rfm_residual", "rfm_sketch",
           "rfm_qr", "rfm_set_r", "rfm_householder_r", "rfm_jmv", "rfm_trsv", "rfm_lsqr", "rfm_linesearch",
           "rfm_ipn_solve", "rfm_amipn_solve", "rfm_eval", "rfm_set_precision",
           "rfm_householder_r_tc", "rfm_emulated_dgemm", "rfm_mlp_create", "rfm_mlp_destroy",
           "rfm_mlp_num_params", "rfm_mlp_params", "rfm_mlp_forward", "rfm_mlp_gradient", "rfm_mlp_train",
           "rfm_feature_gram", "rfm_function_basis", "rfm_basis_combine", "rfm_warmstart_create",
           "rfm_warmstart_destroy", "rfm_warmstart_rank", "rfm_warmstart_network", "rfm_warmstart_train",
           "rfm_warmstart_predict", "rfm_batch_create", "rfm_batch_destroy", "rfm_batch_size", "rfm_batch_problem",
           "rfm_batch_solve", "rfm_autotune_qr", "rfm_set_wait_limit", "rfm_set_rhs"]


class RfmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class ProblemDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("nsub", ctypes.c_int * 3), ("M", ctypes.c_int), ("fields", ctypes.c_int),
                ("q_int", ctypes.c_int * 3), ("q_bdy", ctypes.c_int * 3), ("q_iface", ctypes.c_int * 3),
                ("cont_order", ctypes.c_int), ("feat_range", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("pde_kind", ctypes.c_int), ("pde_params", ctypes.c_double * 8), ("geometry", ctypes.c_int),
                ("n_sphere", ctypes.c_int64)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("sketch_kind", ctypes.c_int), ("gamma", ctypes.c_double), ("sketch_rows", ctypes.c_int64),
                ("eta", ctypes.c_double), ("eps", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("m_max", ctypes.c_int), ("tau_rel", ctypes.c_double), ("row_scale_c", ctypes.c_double),
                ("precision", ctypes.c_int), ("lsqr_max_iter", ctypes.c_int64), ("conlim", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("outer_iters", ctypes.c_int), ("n_jac", ctypes.c_int),
                ("lsqr_iters_total", ctypes.c_int), ("lsqr_iters_max", ctypes.c_int), ("rank_flag", ctypes.c_int),
                ("final_resid", ctypes.c_double), ("t_assemble", ctypes.c_double), ("t_sketch", ctypes.c_double),
                ("t_qr", ctypes.c_double), ("t_lsqr", ctypes.c_double), ("t_linesearch", ctypes.c_double),
                ("t_total", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path=LIB_PATH):
    """Loads librfm.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"librfm.so not built at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, D, I64, I, VP = ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
    sig = {
        "rfm_default_opts": (None, [ctypes.POINTER(SolveOpts)]),
        "rfm_last_error": (ctypes.c_char_p, []),
        "rfm_problem_create": (I, [ctypes.POINTER(ProblemDesc), VP, ctypes.POINTER(P)]),
        "rfm_problem_destroy": (I, [P]),
        "rfm_problem_sizes": (I, [P] + [ctypes.POINTER(I64)] * 7),
        "rfm_set_wait_limit": (I, [P, I64]),
        "rfm_set_rhs": (I, [P, VP]),
        "rfm_get_features": (I, [P, VP]),
        "rfm_get_points": (I, [P, VP]),
        "rfm_assemble": (I, [P, VP, D, VP, VP]),
        "rfm_get_jacobian": (I, [P, VP, VP, VP]),
        "rfm_residual": (I, [P, VP, VP, ctypes.POINTER(D)]),
        "rfm_sketch": (I, [P, I, I64, I, VP]),
        "rfm_qr": (I, [P, VP]),
        "rfm_set_r": (I, [P, VP]),
        "rfm_householder_r": (I, [VP, I64, I64, VP, VP, ctypes.POINTER(I)]),
        "rfm_jmv": (I, [P, I, VP, VP]),
        "rfm_trsv": (I, [P, I, VP, VP]),
        "rfm_lsqr": (I, [P, VP, D, D, I64, VP, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "rfm_linesearch": (I, [P, VP, VP, D, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "rfm_ipn_solve": (I, [P, ctypes.POINTER(SolveOpts), VP, ctypes.POINTER(SolveInfo)]),
        "rfm_amipn_solve": (I, [P, ctypes.POINTER(SolveOpts), VP, ctypes.POINTER(SolveInfo)]),
        "rfm_eval": (I, [P, VP, VP, I64, VP]),
        "rfm_set_precision": (I, [P, I]),
        "rfm_householder_r_tc": (I, [VP, I64, I64, VP, VP, ctypes.POINTER(I)]),
        "rfm_emulated_dgemm": (I, [VP, I64, VP, I64, VP, I64, I64, I64, I64, I, VP]),
        "rfm_mlp_create": (I, [I, I, I, ctypes.c_uint64, VP, ctypes.POINTER(P)]),
        "rfm_mlp_destroy": (I, [P]),
        "rfm_mlp_num_params": (I64, [P]),
        "rfm_mlp_params": (I, [P, VP, VP, ctypes.POINTER(I64)]),
        "rfm_mlp_forward": (I, [P, VP, I, VP]),
        "rfm_mlp_gradient": (I, [P, VP, VP, I, VP, I, VP, ctypes.POINTER(D)]),
        "rfm_mlp_train": (I, [P, VP, VP, I, VP, I, I, ctypes.c_float, ctypes.POINTER(D)]),
        "rfm_feature_gram": (I, [P, VP, I64, ctypes.POINTER(I64), VP]),
        "rfm_function_basis": (I, [P, VP, I, VP, I64, D, VP, VP, VP, ctypes.POINTER(I)]),
        "rfm_basis_combine": (I, [VP, VP, I64, I, VP, I, D, VP, VP]),
        "rfm_warmstart_create": (I, [P, VP, VP, I, I, VP, I64, D, I, ctypes.c_uint64, ctypes.POINTER(P)]),
        "rfm_warmstart_destroy": (I, [P]),
        "rfm_warmstart_rank": (I, [P]),
        "rfm_warmstart_network": (P, [P]),
        "rfm_warmstart_train": (I, [P, I, ctypes.c_float, ctypes.POINTER(D)]),
        "rfm_warmstart_predict": (I, [P, VP, I, VP]),
        "rfm_batch_create": (I, [VP, I, I, ctypes.POINTER(P)]),
        "rfm_batch_destroy": (I, [P]),
        "rfm_batch_size": (I, [P]),
        "rfm_batch_problem": (P, [P, I]),
        "rfm_batch_solve": (I, [P, VP, I, VP, VP, VP]),
        "rfm_autotune_qr": (I, [I64, I64, VP, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(st, ok=(RFM_OK,)):
    if st not in ok:
        raise RfmError(st, load().rfm_last_error().decode())
    return st


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or t.dtype not in (torch.float64, torch.int32, torch.float32) or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA float64/float32/int32 tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def make_desc(d):
    D = ProblemDesc()
    D.dim = d["dim"]
    for b in range(3):
        D.lo[b] = d["lo"][b] if b < d["dim"] else 0.0
        D.hi[b] = d["hi"][b] if b < d["dim"] else 1.0
        D.nsub[b] = d["nsub"][b] if b < d["dim"] else 1
        D.q_int[b] = d["q_int"][b] if b < d["dim"] else 1
        D.q_bdy[b] = d["q_bdy"][b] if b < d["dim"] else 1
        D.q_iface[b] = d["q_iface"][b] if b < d["dim"] else 1
    D.M, D.fields, D.cont_order = d["M"], d["fields"], d["cont_order"]
    D.feat_range, D.seed, D.pde_kind = d["feat_range"], d["seed"], d["pde_kind"]
    for i in range(8):
        D.pde_params[i] = d["pde_params"][i]
    D.geometry = {"box": 0, "ball": 1}[d.get("geometry", "box")]
    D.n_sphere = int(d.get("n_sphere", 0))
    return D


def make_opts(o):
    O = SolveOpts()
    load().rfm_default_opts(ctypes.byref(O))
    O.sketch_kind = SKETCH[o.get("sketch_kind", "count")]
    O.gamma = o.get("gamma", 3.0)
    O.sketch_rows = o.get("sketch_rows", 0)
    O.eta, O.eps = o.get("eta", 1e-6), o.get("eps", 1e-10)
    O.max_outer, O.m_max = o.get("max_outer", 50), o.get("m_max", 3)
    O.tau_rel, O.row_scale_c = o.get("tau_rel", 1e-3), o.get("row_scale_c", 100.0)
    O.precision = o.get("precision", 0)
    O.lsqr_max_iter, O.conlim = o.get("lsqr_max_iter", 0), o.get("conlim", 1e8)
    return O


class Problem:
    """Owns an rfm_problem.  `desc` is a problem dict (rfm_workloads)."""

    def __init__(self, desc, stream=None):
        lib = load()
        self.desc = desc
        self.stream = stream
        self._h = ctypes.c_void_p()
        _check(lib.rfm_problem_create(ctypes.byref(make_desc(desc)), _stream(stream), ctypes.byref(self._h)))
        v = [ctypes.c_int64() for _ in range(7)]
        _check(lib.rfm_problem_sizes(self._h, *[ctypes.byref(x) for x in v]))
        self.m, self.n, self.W, self.G, self.m_int, self.m_iface, self.nnz = (x.value for x in v)

    def close(self):
        if self._h:
            load().rfm_problem_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, *shape, dtype=torch.float64):
        return torch.empty(*shape, dtype=dtype, device="cuda")

    # -- A1: features and points
    def rfm_get_features(self):
        out = self._dev(self.G * self.desc["fields"] * self.desc["M"], 4)
        _check(load().rfm_get_features(self._h, _ptr(out)))
        return out

    def rfm_get_points(self):
        out = self._dev(self.m, 4)
        _check(load().rfm_get_points(self._h, _ptr(out)))
        return out

    # -- A2/A3: assembly with row scaling
    def rfm_assemble(self, c, c_scale=100.0):
        F, lam = self._dev(self.m), self._dev(self.m)
        _check(load().rfm_assemble(self._h, _ptr(c), c_scale, _ptr(F), _ptr(lam)))
        return F, lam

    def rfm_get_jacobian(self):
        Jp = self._dev(self.m, self.W)
        Js = self._dev(max(1, self.m_iface), self.W)
        blk = self._dev(self.m, 2, dtype=torch.int32)
        _check(load().rfm_get_jacobian(self._h, _ptr(Jp), _ptr(Js), _ptr(blk)))
        return Jp, Js[: self.m_iface], blk

    def rfm_residual(self, c):
        F = self._dev(self.m)
        nv = ctypes.c_double()
        _check(load().rfm_residual(self._h, _ptr(c), _ptr(F), ctypes.byref(nv)))
        return F, nv.value

    # -- A4/A5: sketch and QR
    def rfm_set_precision(self, precision):
        _check(load().rfm_set_precision(self._h, precision))

    def rfm_set_wait_limit(self, polls):
        _check(load().rfm_set_wait_limit(self._h, polls))

    def rfm_set_rhs(self, rhs):
        _check(load().rfm_set_rhs(self._h, _ptr(rhs)))

    def rfm_sketch(self, kind, s, kJ, copy_out=True):
        B = self._dev(self.n, s) if copy_out else None
        _check(load().rfm_sketch(self._h, SKETCH[kind], s, kJ, _ptr(B)))
        return B

    def rfm_qr(self, copy_out=True):
        R = self._dev(self.n, self.n) if copy_out else None
        st = _check(load().rfm_qr(self._h, _ptr(R)), ok=(RFM_OK, RFM_ERANK))
        return R, st == RFM_ERANK

    def rfm_set_r(self, R_colmajor):
        _check(load().rfm_set_r(self._h, _ptr(R_colmajor)))

    # -- A6/A7: matvecs, triangular solves, LSQR
    def rfm_jmv(self, x, trans=0):
        y = self._dev(self.n if trans else self.m)
        _check(load().rfm_jmv(self._h, trans, _ptr(x), _ptr(y)))
        return y

    def rfm_trsv(self, b, trans=0):
        x = self._dev(self.n)
        _check(load().rfm_trsv(self._h, trans, _ptr(b), _ptr(x)))
        return x

    def rfm_lsqr(self, b, eta=1e-6, conlim=1e8, max_iter=0):
        d = self._dev(self.n)
        it, istop = ctypes.c_int(), ctypes.c_int()
        _check(load().rfm_lsqr(self._h, _ptr(b), eta, conlim, max_iter, _ptr(d), ctypes.byref(it), ctypes.byref(istop)))
        return d, it.value, istop.value

    # -- A8: line search
    def rfm_linesearch(self, c, d, f0):
        a, fb = ctypes.c_double(), ctypes.c_double()
        _check(load().rfm_linesearch(self._h, _ptr(c), _ptr(d), f0, ctypes.byref(a), ctypes.byref(fb)))
        return a.value, fb.value

    # -- A9/A10: solvers
    def _solve(self, fn, opts, c0):
        c = torch.zeros(self.n, dtype=torch.float64, device="cuda") if c0 is None else c0.clone()
        info = SolveInfo()
        st = fn(self._h, ctypes.byref(make_opts(opts)), _ptr(c), ctypes.byref(info))
        # a solver failure (iteration cap, non-finite residual) still returns
        # the last iterate; info["status"] carries it
        _check(st, ok=(RFM_OK, RFM_ENOCONV, RFM_ENONFINITE))
        return c, info.as_dict()

    def rfm_ipn_solve(self, opts, c0=None):
        return self._solve(load().rfm_ipn_solve, opts, c0)

    def rfm_amipn_solve(self, opts, c0=None):
        return self._solve(load().rfm_amipn_solve, opts, c0)

    # -- A11: evaluation
    def rfm_eval(self, c, pts):
        pts = pts.contiguous()
        u = self._dev(pts.shape[0], self.desc["fields"])
        _check(load().rfm_eval(self._h, _ptr(c), _ptr(pts), pts.shape[0], _ptr(u)))
        return u


def rfm_householder_r(A_colmajor, s, n, stream=None):
    """R of an s x n column-major matrix given as a CUDA tensor of shape
    (n, s) (A is overwritten)."""
    R = torch.empty(n, n, dtype=torch.float64, device="cuda")
    flag = ctypes.c_int()
    _check(load().rfm_householder_r(_ptr(A_colmajor), s, n, _stream(stream), _ptr(R), ctypes.byref(flag)))
    return R, bool(flag.value)


def rfm_householder_r_tc(A_colmajor, s, n, stream=None):
    """Tensor-core (emulated FP64 trailing update) Householder R; A is (n, s)
    row-major == s x n column-major and is overwritten."""
    R = torch.empty(n, n, dtype=torch.float64, device="cuda")
    flag = ctypes.c_int()
    _check(load().rfm_householder_r_tc(_ptr(A_colmajor), s, n, _stream(stream), _ptr(R), ctypes.byref(flag)))
    return R, bool(flag.value)


def rfm_emulated_dgemm(A, B, digits=8, stream=None):
    """C = A B for CUDA float64 matrices given column-major as tensors of
    shape (K, M) and (N, K) (row-major transposes); returns C as (N, M)."""
    K, M = A.shape
    N = B.shape[0]
    C = torch.empty(N, M, dtype=torch.float64, device="cuda")
    _check(load().rfm_emulated_dgemm(_ptr(A), M, _ptr(B), K, _ptr(C), M, M, N, K, digits, _stream(stream)))
    return C


class MLP:
    """Warm-start network (rfm_mlp_*): d_in -> H -> H -> d_out, bf16 weights and
    activations with FP32 accumulation and FP32 Adam master weights."""

    def __init__(self, d_in, hidden, d_out, seed=1, stream=None):
        self._h = ctypes.c_void_p()
        self.d_in, self.hidden, self.d_out = d_in, hidden, d_out
        _check(load().rfm_mlp_create(d_in, hidden, d_out, seed, _stream(stream), ctypes.byref(self._h)))
        self.num_params = load().rfm_mlp_num_params(self._h)

    def close(self):
        if self._h:
            load().rfm_mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        out = torch.empty(self.num_params, dtype=torch.float32, device="cuda")
        offs = (ctypes.c_int64 * 6)()
        _check(load().rfm_mlp_params(self._h, _ptr(out), None, offs))
        return out, list(offs)

    def set_params(self, flat):
        _check(load().rfm_mlp_params(self._h, None, _ptr(flat.contiguous()), None))

    def forward(self, x):
        y = torch.empty(x.shape[0], self.d_out, dtype=torch.float32, device="cuda")
        _check(load().rfm_mlp_forward(self._h, _ptr(x.contiguous()), x.shape[0], _ptr(y)))
        return y

    def gradient(self, x, t, G=None, gblk=0):
        g = torch.empty(self.num_params, dtype=torch.float32, device="cuda")
        loss = ctypes.c_double()
        _check(load().rfm_mlp_gradient(self._h, _ptr(x.contiguous()), _ptr(t.contiguous()), x.shape[0],
                                       _ptr(G), gblk, _ptr(g), ctypes.byref(loss)))
        return g, loss.value

    def train(self, x, t, steps, lr, G=None, gblk=0):
        loss = ctypes.c_double()
        _check(load().rfm_mlp_train(self._h, _ptr(x.contiguous()), _ptr(t.contiguous()), x.shape[0], _ptr(G), gblk,
                                    steps, lr, ctypes.byref(loss)))
        return loss.value


def rfm_feature_gram(problem, pts, owner_start):
    """Per-subdomain feature Gram at points grouped by owner (see rfm.h)."""
    G = torch.empty(problem.G * problem.desc["fields"], problem.desc["M"], problem.desc["M"],
                    dtype=torch.float32, device="cuda")
    starts = (ctypes.c_int64 * len(owner_start))(*[int(v) for v in owner_start])
    _check(load().rfm_feature_gram(problem._h, _ptr(pts.contiguous()), pts.shape[0], starts, _ptr(G)))
    return G


def rfm_function_basis(problem, C, pts, tol=1e-8):
    """Centred snapshot basis orthonormal in u-space (see rfm.h).  C is a CUDA
    float64 tensor [N][n]; returns (mean [n], U [rank][n], Z [N][rank])."""
    N, n = C.shape
    mean = torch.empty(n, dtype=torch.float64, device="cuda")
    U = torch.empty(N, n, dtype=torch.float64, device="cuda")
    Z = torch.empty(N, N, dtype=torch.float64, device="cuda")
    rank = ctypes.c_int()
    _check(load().rfm_function_basis(problem._h, _ptr(C.contiguous()), N, _ptr(pts.contiguous()), pts.shape[0], tol,
                                     _ptr(mean), _ptr(U), _ptr(Z), ctypes.byref(rank)))
    r = rank.value
    return mean, U[:r].contiguous(), Z[:, :r].contiguous()


def rfm_basis_combine(mean, U, y, scale=1.0, stream=None):
    """c = mean + scale * y U for a batch y [batch][rank] (float32)."""
    batch = y.shape[0]
    c = torch.empty(batch, mean.shape[0], dtype=torch.float64, device="cuda")
    _check(load().rfm_basis_combine(_ptr(mean), _ptr(U), mean.shape[0], U.shape[0], _ptr(y.contiguous()), batch,
                                    scale, _ptr(c), _stream(stream)))
    return c


class WarmStart:
    """rfm_warmstart_*: basis of training solutions plus the coordinate network."""

    def __init__(self, problem, C, params, pts, tol=1e-6, hidden=256, seed=1):
        self._h = ctypes.c_void_p()
        self.n = problem.n
        _check(load().rfm_warmstart_create(problem._h, _ptr(C.contiguous()), _ptr(params.contiguous()), C.shape[0],
                                           params.shape[1], _ptr(pts.contiguous()), pts.shape[0], tol, hidden, seed,
                                           ctypes.byref(self._h)))
        self.rank = load().rfm_warmstart_rank(self._h)

    def close(self):
        if self._h:
            load().rfm_warmstart_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def train(self, steps, lr=1e-3):
        loss = ctypes.c_double()
        _check(load().rfm_warmstart_train(self._h, steps, lr, ctypes.byref(loss)))
        return loss.value

    def predict(self, params):
        c = torch.empty(params.shape[0], self.n, dtype=torch.float64, device="cuda")
        _check(load().rfm_warmstart_predict(self._h, _ptr(params.contiguous()), params.shape[0], _ptr(c)))
        return c


class _BorrowedProblem(Problem):
    """A problem owned by a batch (not destroyed by this handle)."""

    def __init__(self, handle, desc):
        lib = load()
        self.desc = desc
        self.stream = None
        self._h = ctypes.c_void_p(handle)
        v = [ctypes.c_int64() for _ in range(7)]
        _check(lib.rfm_problem_sizes(self._h, *[ctypes.byref(x) for x in v]))
        self.m, self.n, self.W, self.G, self.m_int, self.m_iface, self.nnz = (x.value for x in v)

    def close(self):
        self._h = ctypes.c_void_p()


class Batch:
    """rfm_batch_*: independent instances solved concurrently on one GPU."""

    def __init__(self, descs, streams=4):
        self.descs = list(descs)
        arr = (ProblemDesc * len(self.descs))(*[make_desc(d) for d in self.descs])
        self._h = ctypes.c_void_p()
        _check(load().rfm_batch_create(arr, len(self.descs), streams, ctypes.byref(self._h)))
        self.problems = [_BorrowedProblem(load().rfm_batch_problem(self._h, i), d) for i, d in enumerate(self.descs)]

    def close(self):
        if self._h:
            load().rfm_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, opts, solver="ipn", c0=None):
        """Returns (list of solutions, list of info dicts, tuned precisions)."""
        k = len(self.problems)
        cs = [torch.zeros(p.n, dtype=torch.float64, device="cuda") if c0 is None else c0[i].clone()
              for i, p in enumerate(self.problems)]
        ptrs = (ctypes.c_void_p * k)(*[c.data_ptr() for c in cs])
        infos = (SolveInfo * k)()
        tuned = (ctypes.c_int * k)()
        st = load().rfm_batch_solve(self._h, ctypes.byref(make_opts(opts)), 0 if solver == "ipn" else 1, ptrs, infos,
                                    tuned)
        _check(st, ok=(RFM_OK, RFM_ENOCONV))
        return cs, [i.as_dict() for i in infos], list(tuned)


def rfm_autotune_qr(s, n, stream=None):
    prec, cap = ctypes.c_int(), ctypes.c_int()
    ms = (ctypes.c_double * 8)()
    _check(load().rfm_autotune_qr(s, n, _stream(stream), ctypes.byref(prec), ctypes.byref(cap), ms))
    return prec.value, cap.value, list(ms)
