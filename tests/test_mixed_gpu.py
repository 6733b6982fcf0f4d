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


# ---- the blocked leaf (TSQR_LEAF_PANELS: 16-column panels, compact WY updates on the tensor
#      cores) explicitly, against the oracle; and the fold (TSQR_LEAF_FOLD) beside it

@pytest.mark.parametrize("dtype", ["float32", "bfloat16"])
@pytest.mark.parametrize("n", [1, 3, 8, 15, 16, 17, 31, 32, 33, 47, 48, 63, 64])
@pytest.mark.parametrize("h", [256, 512, 640, 768, 1024])
def test_panels_leaf_widths(oracle, T, dtype, n, h):
    if (h == 768 and n > 48) or (h == 1024 and n > 32):
        pytest.skip("chunk taller than the width's shared and tensor memory allow")
    if h == 640 and n < 15:
        pytest.skip("640-row chunks are the AUTO height of 49 to 64 columns; a few widths suffice")
    import torch
    m = 70001 if n > 16 else 30011  # several chunks per leaf and a ragged last chunk
    At = workloads.gaussian(m, n, seed=100 + n, dtype=getattr(torch, dtype))
    plan = T.make_plan("hybrid", tile_rows=h, leaf="panels")
    _check(oracle, T, At, plan=plan)
    used = T.last_plan()
    assert used.leaf == T.LEAF_PANELS and used.tile_rows == h


@pytest.mark.parametrize("tree,b,ctas", [("binary", 256, 0), ("binary", 768, 0), ("flat", 0, 0),
                                         ("hybrid", 256, 7), ("hybrid", 512, 3)])
def test_panels_leaf_trees(oracle, T, tree, b, ctas):
    import torch
    At = workloads.gaussian(50000, 40, seed=7, dtype=torch.float32)
    _check(oracle, T, At, plan=T.make_plan(tree, tile_rows=b, ctas=ctas, leaf="panels"))


def test_panels_leaf_odd_leading_dimension(oracle, T):
    """lda not a multiple of 4 floats: the chunk loads fall back from 16-byte copies."""
    import torch
    m, n = 33333, 48
    At = workloads.gaussian(m, n, seed=9, dtype=torch.float32)
    big = torch.zeros(n, m + 1, dtype=torch.float32)
    big[:, :m] = At
    R = T.tsqr_r_ex(big.cuda().T[:m, :], plan=T.make_plan(leaf="panels")).cpu().numpy()
    A = oracle.from_torch_colmajor(At.to(torch.float64))
    assert oracle.gram_residual(A, R) <= 2e-6
    Ro = oracle.householder_r(A, nthreads=16)
    np.testing.assert_allclose(R, Ro, rtol=0, atol=max(50.0, 2.0 * np.sqrt(m)) *
                               oracle.kappa_from_r(Ro) * U32 * np.linalg.norm(Ro))


@pytest.mark.parametrize("dtype", ["float32", "bfloat16"])
@pytest.mark.parametrize("n", [8, 24, 40, 64])
def test_panels_leaf_tma_and_thread_loads_agree(oracle, T, dtype, n):
    """A 16-byte aligned leading dimension takes the TMA box loads (FP32 boxes land swizzled;
    BF16 boxes are staged and widened); an odd one takes the thread copies.  Both put the same
    chunk in shared memory, so R is the same to the bit.  m = 50,001 leaves a ragged last chunk
    (the TMA's zero fill past A's last row)."""
    import torch
    m = 50001
    dt = getattr(torch, dtype)
    At = workloads.gaussian(m, n, seed=200 + n, dtype=dt)

    def run(ld):
        big = torch.zeros(n, ld, dtype=dt)
        big[:, :m] = At
        return T.tsqr_r_ex(big.cuda().T[:m, :], plan=T.make_plan(leaf="panels")).cpu()

    Ra = run(m + 15)  # 50,016: a multiple of 8 elements (16 bytes of BF16, 32 of FP32)
    Rb = run(m + 2)   # 50,003: odd
    assert torch.equal(Ra, Rb)
    A = oracle.from_torch_colmajor(At.to(torch.float64))
    assert oracle.gram_residual(A, Ra.numpy()) <= 2e-6


def test_panels_leaf_rank_deficient(oracle, T):
    """Zero and repeated columns (identity reflectors, zero pivots): R^T R = A^T A still."""
    import torch
    m, n = 40000, 40
    At = workloads.gaussian(m, n, seed=11, dtype=torch.float32)
    At[5] = 0.0
    At[20] = At[3]
    At[39] = 0.0
    R = T.tsqr_r_ex(At.cuda().T, plan=T.make_plan(leaf="panels")).cpu().numpy()
    A = oracle.from_torch_colmajor(At.to(torch.float64))
    assert np.all(np.isfinite(R)) and np.all(np.diag(R) >= 0)
    assert oracle.gram_residual(A, R) <= 2e-6


def test_panels_leaf_bit_reproducible(T):
    import torch
    At = workloads.gaussian(400000, 64, seed=12, dtype=torch.float32).cuda().T
    p = T.make_plan(leaf="panels")
    a = T.tsqr_r_ex(At, plan=p).clone()
    b = T.tsqr_r_ex(At, plan=p).clone()
    torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("leaf", ["fold", "panels"])
def test_mixed_leaves_conditioned_report(oracle, T, leaf):
    """Both mixed leaves at 2^20 x 64, kappa = 1e6, FP32: the Gram residual and the forward
    error against the oracle, printed beside 50 kappa u32 (run with -s to see them)."""
    import torch
    At = workloads.conditioned(1 << 20, 64, 1e6, seed=0, dtype=torch.float32)
    res, err, kap = _check(oracle, T, At, plan=T.make_plan(leaf=leaf))
    print(f"\n{leaf}: gram residual {res:.3e}, |R - R_oracle|/|R_oracle| {err:.3e}, "
          f"50 kappa u32 {50 * kap * U32:.3e}")


@pytest.mark.parametrize("dtype", ["float32", "bfloat16"])
@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_panels_leaf_nonfinite_input_is_reported(T, dtype, bad):
    """A NaN or Inf in A propagates into R and sets the non-finite status (no wait gives up);
    the next clean call is clean again."""
    import torch
    dt = getattr(torch, dtype)
    At = workloads.gaussian(70001, 48, seed=31, dtype=dt)
    At[17, 40000] = bad
    T.tsqr_get_device_status()  # clear
    R = T.tsqr_r_ex(At.cuda().T, plan=T.make_plan(leaf="panels"))
    assert T.tsqr_get_device_status() == T.STATUS_NONFINITE
    assert not torch.isfinite(R).all()
    R = T.tsqr_r_ex(workloads.gaussian(70001, 48, seed=31, dtype=dt).cuda().T,
                    plan=T.make_plan(leaf="panels"))
    assert T.tsqr_get_device_status() == T.SUCCESS
    assert torch.isfinite(R).all()


@pytest.mark.parametrize("dtype", ["float32", "bfloat16"])
@pytest.mark.parametrize("n", [65, 72, 80, 81, 96, 97, 112])
def test_panels_leaf_wide(oracle, T, dtype, n):
    """The blocked leaf past 64 columns, at the chunk height the width's memory allows (512 rows
    to 80 columns, 384 to 96, 256 to 112), with a ragged last chunk; against the oracle.  AUTO
    takes it too, and its plan passed back gives the same bytes."""
    import torch
    m = 30011
    At = workloads.gaussian(m, n, seed=500 + n, dtype=getattr(torch, dtype))
    _check(oracle, T, At, plan=T.make_plan(leaf="panels"))
    used = T.last_plan()
    assert used.leaf == T.LEAF_PANELS
    assert used.tile_rows == (512 if n <= 80 else 384 if n <= 96 else 256)
    Ad = At.cuda().T
    Ra = T.tsqr_r_ex(Ad)
    auto = T.last_plan()
    assert auto.leaf == T.LEAF_PANELS
    assert torch.equal(T.tsqr_r_ex(Ad, plan=auto), Ra)
