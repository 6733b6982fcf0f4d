"""GPU parity of libtsqr's mixed-precision path (FP32 or BF16 A; FP32 leaf arithmetic, FP64
reflector norms, scalars and tree) against the FP64 CPU oracle, through the C ABI.

"A" is the stored FP32/BF16 matrix, widened exactly to FP64 for the oracle.  Acceptance:
||R^T R - A^T A||_F / ||A||_F^2 <= 2e-6.  Every entry of R must also lie within
c(m) kappa(A) u32 ||R_oracle||_F of the oracle's R, u32 = 2^-24 and c(m) = max(50, 2 sqrt(m))
as in the FP64 tests (forward error <= kappa x backward error, the leaf's rounding being FP32).
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def T():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1002_4250_gb300 as T
    return T


def _check(oracle, T, At_lowp, plan=None, nthreads=16):
    """At_lowp: (n, m) FP32/BF16 CPU tensor holding the column-major input."""
    import torch
    A = oracle.from_torch_colmajor(At_lowp.to(torch.float64))
    R = T.tsqr_r_ex(At_lowp.cuda().T, plan=plan).cpu().numpy()
    Ro = oracle.householder_r(A, nthreads=nthreads)
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) >= 0)
    res = oracle.gram_residual(A, R, nthreads=nthreads)
    assert res <= 2e-6, f"gram residual {res:.3e}"
    m = A.shape[0]
    kap = oracle.kappa_from_r(Ro)
    tol = max(50.0, 2.0 * np.sqrt(m)) * kap * U32 * np.linalg.norm(Ro)
    np.testing.assert_allclose(R, Ro, rtol=0, atol=tol)
    return res, oracle.rel_err(R, Ro), kap


@pytest.mark.parametrize("dtype", ["float32", "bfloat16"])
@pytest.mark.parametrize("m,n", [(20000, 8), (33333, 16), (100001, 32), (65537, 64), (5000, 1),
                                 (3000, 3), (4097, 128)])
def test_mixed_gaussian(oracle, T, dtype, m, n):
    import torch
    At = workloads.gaussian(m, n, seed=n, dtype=getattr(torch, dtype))
    _check(oracle, T, At)


@pytest.mark.parametrize("dtype", ["float32", "bfloat16"])
@pytest.mark.parametrize("kappa", [1e2, 1e4, 1e6])
def test_mixed_conditioned(oracle, T, dtype, kappa):
    """The mixed-precision workload's conditioning, at 2^20 x 64."""
    import torch
    At = workloads.conditioned(1 << 20, 64, kappa, seed=0, dtype=getattr(torch, dtype))
    _check(oracle, T, At)


@pytest.mark.parametrize("tree,b", [("binary", 256), ("flat", 0), ("hybrid", 512)])
def test_mixed_trees(oracle, T, tree, b):
    import torch
    At = workloads.gaussian(40000, 24, seed=3, dtype=torch.float32)
    _check(oracle, T, At, plan=T.make_plan(tree, tile_rows=b))


def test_mixed_bit_reproducible(T):
    import torch
    At = workloads.gaussian(300000, 32, seed=4, dtype=torch.float32).cuda().T
    a = T.tsqr_r_ex(At).clone()
    b = T.tsqr_r_ex(At).clone()
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_mixed_leading_dimension_and_tail(oracle, T):
    import torch
    m, n = 7777, 20
    At = workloads.gaussian(m, n, seed=5, dtype=torch.float32)
    big = torch.zeros(n, m + 3, dtype=torch.float32)
    big[:, :m] = At
    R = T.tsqr_r_ex(big.cuda().T[:m, :]).cpu().numpy()
    A = oracle.from_torch_colmajor(At.to(torch.float64))
    assert oracle.gram_residual(A, R) <= 2e-6


def test_mixed_full_size_kappa_1e6(oracle, T):
    """The mixed-precision workload at full size: 2^24 x 64 FP32, kappa = 1e6."""
    import torch
    At = workloads.conditioned(1 << 24, 64, 1e6, seed=0, dtype=torch.float32)
    _check(oracle, T, At)
