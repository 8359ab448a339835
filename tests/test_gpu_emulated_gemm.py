"""Emulated FP64 products on the bf16 tensor cores (digit splitting with exact
FP32 level accumulation): accuracy against an extended-precision product,
relative to the componentwise bound |A||B|, must match an FP64 GEMM's class."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_04170_gb300 import build, rfm
    build.build()
    L = rfm.load()
    L.rfm_emulated_dgemm.restype = ctypes.c_int
    L.rfm_emulated_dgemm.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]
    return L


def _run(lib, A, B, digits):
    M, K = A.shape
    N = B.shape[1]
    Ad = torch.as_tensor(A.reshape(-1, order="F").copy(), device="cuda")
    Bd = torch.as_tensor(B.reshape(-1, order="F").copy(), device="cuda")
    Cd = torch.zeros(M * N, dtype=torch.float64, device="cuda")
    st = lib.rfm_emulated_dgemm(ctypes.c_void_p(Ad.data_ptr()), M, ctypes.c_void_p(Bd.data_ptr()), K,
                                ctypes.c_void_p(Cd.data_ptr()), M, M, N, K, digits,
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.rfm_last_error().decode()
    return Cd.cpu().numpy().reshape(N, M).T


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (300, 200, 1500), (130, 70, 4100), (1, 1, 1), (257, 65, 513)])
def test_emulated_dgemm_fp64_class(lib, M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K)) * np.logspace(0, -6, K)[None, :]
    B = rng.standard_normal((K, N)) * np.logspace(0, -3, N)[None, :]
    ref = (A.astype(np.longdouble) @ B.astype(np.longdouble)).astype(np.float64)
    bound = np.abs(A) @ np.abs(B)
    C = _run(lib, A, B, 8)
    rel = np.max(np.abs(C - ref) / bound)
    assert rel <= 4e-15, rel
    # plain bf16-sized inputs (one exact digit) are reproduced exactly
    Ai = rng.integers(-100, 100, (M, K)).astype(np.float64)
    Bi = rng.integers(-100, 100, (K, N)).astype(np.float64)
    C1 = _run(lib, Ai, Bi, 2)
    assert np.array_equal(C1, Ai @ Bi)
