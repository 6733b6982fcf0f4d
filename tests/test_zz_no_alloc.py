"""tsqr_r_noalloc: the R factor for callers that cannot allocate device memory when they call
(for example a serving loop that must not allocate after start-up, or a process whose
framework already holds the device's memory in its own caching allocator).  It works in one
static device array instead of the library's per-stream workspace.

The test calls it through the C ABI, twice in a row on the same inputs (the array keeps the
previous call's contents, so the second call checks that everything that must start at zero
is cleared), and compares each result with tsqr_r's within the parity tolerance of the GPU
tests: every entry within c(m) kappa u ||R||_F, c(m) = max(50, 2 sqrt(m)).  The file is named
to be collected last."""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module")
def T():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1002_4250_gb300 import _build
    _build.build()
    import paper_1002_4250_gb300 as T
    return T


def _call_noalloc(T, A, R):
    import torch
    m, n = A.shape
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return T.capi.tsqr_r_noalloc(A.data_ptr(), m, n, A.stride(1), R.data_ptr(), R.stride(1),
                                 stream)


@pytest.mark.parametrize("m,n", [(1_000_003, 32), (123_457, 16), (300_001, 64), (5_000, 3)])
def test_noalloc_matches_tsqr_r_on_two_calls(T, m, n):
    import torch
    At = workloads.gaussian(m, n, seed=m % 97)
    A = At.cuda().T
    R_ref = T.tsqr_r(A).cpu().numpy()
    s = np.linalg.svd(R_ref, compute_uv=False)
    tol = max(50.0, 2.0 * np.sqrt(m)) * (s[0] / s[-1]) * U * np.linalg.norm(R_ref)
    for _ in range(2):
        R = T.empty_r(n, "cuda")
        R.fill_(float("nan"))
        assert _call_noalloc(T, A, R) == T.SUCCESS
        assert T.tsqr_last_launch_count() == 1
        used = T.last_plan()
        assert used.tree == T.TREE_HYBRID and used.ctas > 0  # one reduction, never the panels
        torch.cuda.synchronize()
        np.testing.assert_allclose(R.cpu().numpy(), R_ref, rtol=0, atol=tol)


def test_noalloc_rejects_what_does_not_fit(T):
    import torch
    m, n = 100_000, 128
    A = torch.zeros(n, m, dtype=torch.float64, device="cuda").T
    R = T.empty_r(n, "cuda")
    assert _call_noalloc(T, A, R) == T.ERR_UNSUPPORTED
    assert T.tsqr_last_launch_count() == 0 and T.last_plan().tree == 0
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert T.capi.tsqr_r_noalloc(A.data_ptr(), m, 129, m, R.data_ptr(), 129, stream) == T.ERR_UNSUPPORTED
    assert T.capi.tsqr_r_noalloc(A.data_ptr(), m, 8, m - 1, R.data_ptr(), 8, stream) == T.ERR_INVALID_ARG
