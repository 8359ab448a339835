"""GPU check of rfm_householder_r_noalloc, the Householder-R entry point for
callers that cannot allocate device memory while they run (services that
reserve all GPU memory up front in their own pool, fixed-latency loops).

Three calls in a row, on different inputs, through the C ABI (the third
smaller than the second, so it starts on the scratch the larger call left
behind): each R must equal, bit for bit, the R of the allocating entry point
rfm_householder_r, which runs the same deterministic kernels (fixed-order
reductions).  Sizes beyond the fixed scratch limit must be rejected.
This file sorts last so that a run stopping at the first failure has already
run every other test."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _matrix(s, n, cond, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((s, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return U @ np.diag(np.logspace(0, -np.log10(cond), n)) @ V.T


def test_noalloc_householder_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_04170_gb300 import build, rfm
    build.build()
    lib = rfm.load()
    fn = lib.rfm_householder_r_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.POINTER(ctypes.c_int)]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (s, n, cond) in enumerate([(700, 300, 1e8), (2100, 512, 1e6), (600, 200, 1e10)]):
        B = _matrix(s, n, cond, seed=100 + call)
        ref, ref_flag = rfm.rfm_householder_r(torch.as_tensor(B.T.copy(), device="cuda"), s, n)
        A = torch.as_tensor(B.T.copy(), device="cuda")
        R = torch.empty(n, n, dtype=torch.float64, device="cuda")
        flag = ctypes.c_int(-1)
        st = fn(ctypes.c_void_p(A.data_ptr()), s, n, stream, ctypes.c_void_p(R.data_ptr()), ctypes.byref(flag))
        assert st == rfm.RFM_OK, lib.rfm_last_error().decode()
        assert flag.value == int(ref_flag)
        assert torch.equal(R, ref)
        assert bool(torch.all(torch.diagonal(R) > 0))
    # more columns than the fixed scratch holds: rejected with a clear message
    A = torch.zeros(513, 600, dtype=torch.float64, device="cuda")
    R = torch.empty(513, 513, dtype=torch.float64, device="cuda")
    st = fn(ctypes.c_void_p(A.data_ptr()), 600, 513, stream, ctypes.c_void_p(R.data_ptr()), None)
    assert st == rfm.RFM_EINVAL
    assert "512" in lib.rfm_last_error().decode()
