"""GPU parity of tsqr_qr (thin Q and R) against the CPU oracle's Householder QR, through the C
ABI.  Q is unique for A of full rank under diag(R) >= 0, so the GPU's Q is compared entry by
entry with the oracle's: every entry within c(m) kappa u ||Q_oracle||_F, c(m) = max(50, 2 sqrt(m))
as for R.  R must be bit-identical to tsqr_r's under the same plan (same kernels, same order).
Orthogonality ||Q^T Q - I||_max and the backward error ||A - Q R||_F / ||A||_F are bounded by
c(m) n u."""
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
    import paper_1002_4250_gb300 as T
    return T


def _c(m):
    return max(50.0, 2.0 * np.sqrt(max(m, 1)))


def _check(oracle, T, At, plan=None, nthreads=16):
    """At: (n, m) CPU FP64 tensor holding the column-major input."""
    A = oracle.from_torch_colmajor(At)
    m, n = A.shape
    Ad = At.cuda().T
    Q, R = T.tsqr_qr(Ad, plan=plan)
    # the plan used: the given or AUTO plan, or its four-warp form where that plan runs another
    # warp count or chunks too tall for the Q passes
    used = T.last_plan()
    if plan is not None and plan.warps:
        assert used.warps == plan.warps
    Rr = T.tsqr_r_ex(Ad, plan=used)
    Qh, Rh = Q.cpu().numpy(), R.cpu().numpy()
    assert np.array_equal(Rh, Rr.cpu().numpy()), "R differs from tsqr_r's under the same plan"
    Qo, Ro = oracle.householder_qr(A, nthreads=nthreads)
    kap = oracle.kappa_from_r(Ro)
    tol = _c(m) * kap * U * np.linalg.norm(Qo)
    np.testing.assert_allclose(Qh, Qo, rtol=0, atol=tol)
    assert np.abs(Qh.T @ Qh - np.eye(n)).max() <= _c(m) * n * U
    assert np.linalg.norm(A - Qh @ Rh) / np.linalg.norm(A) <= _c(m) * n * U
    return Qh, Rh


@pytest.mark.parametrize("m,n", [(10000, 16), (100003, 32), (65537, 8), (50001, 64), (3000, 1),
                                 (777, 3), (200003, 48), (4097, 5)])
def test_qr_gaussian(oracle, T, m, n):
    _check(oracle, T, workloads.gaussian(m, n, seed=m % 101))


@pytest.mark.parametrize("m,n", [(100003, 128), (65537, 96), (30011, 80)])
def test_qr_wide_column_groups(oracle, T, m, n):
    """Widths whose chunk, Q rows and carried block do not fit shared memory together: the
    passes take the columns in groups (and the tails live outside Q)."""
    _check(oracle, T, workloads.gaussian(m, n, seed=n))


@pytest.mark.parametrize("tree,b,ctas,arity", [("binary", 256, 0, 0), ("flat", 0, 0, 0),
                                               ("hybrid", 0, 37, 2), ("hybrid", 0, 61, 5),
                                               ("hybrid", 0, 100, 8)])
def test_qr_trees(oracle, T, tree, b, ctas, arity):
    At = workloads.gaussian(120001, 24, seed=11)
    _check(oracle, T, At, plan=T.make_plan(tree, tile_rows=b, ctas=ctas, arity=arity))


def test_qr_conditioned(oracle, T):
    _check(oracle, T, workloads.conditioned(200000, 32, 1e8, seed=0))


@pytest.mark.parametrize("m,n", [(32, 32), (300, 32), (129, 64), (1, 1), (5, 5), (130, 64),
                                 (133, 64), (386, 32)])
def test_qr_single_leaf_and_square(oracle, T, m, n):
    """Also shapes whose last leaf holds one to five rows: a chunk that runs out of rank, with
    tiny tails and huge scales c in its later reflectors."""
    _check(oracle, T, workloads.gaussian(m, n, seed=3))


def test_qr_leading_dimensions(oracle, T):
    import torch
    m, n = 33333, 20
    At = workloads.gaussian(m, n, seed=5)
    big = torch.zeros(n, m + 7, dtype=torch.float64)
    big[:, :m] = At
    Ad = big.cuda().T[:m, :]
    Qbig = torch.full((n, m + 3), float("nan"), dtype=torch.float64, device="cuda")
    Q, R = T.tsqr_qr(Ad, Q=Qbig.T[:m, :])
    A = oracle.from_torch_colmajor(At)
    Qo, Ro = oracle.householder_qr(A, nthreads=16)
    tol = _c(m) * oracle.kappa_from_r(Ro) * U * np.linalg.norm(Qo)
    np.testing.assert_allclose(Q.cpu().numpy(), Qo, rtol=0, atol=tol)
    assert torch.isnan(Qbig[:, m:]).all()  # the padding rows of Q are not written


def test_qr_bit_reproducible_and_launches(T):
    import torch
    Ad = workloads.gaussian(300000, 32, seed=4).cuda().T
    Q1, R1 = T.tsqr_qr(Ad)
    Q1 = Q1.clone()
    n_launch = T.capi.tsqr_last_launch_count()
    Q2, R2 = T.tsqr_qr(Ad)
    torch.cuda.synchronize()
    assert torch.equal(Q1, Q2) and torch.equal(R1, R2)
    levels = 1
    p = T.tsqr_resolve_plan(300000, 32)
    c = p.ctas
    while c > 1:
        c = (c + p.arity - 1) // p.arity
        levels += 1
    # the factorization, one tree pass per level below the root and the leaf pass (which forms
    # the chunks' compact WY factors itself when Q's columns form one group)
    assert n_launch == 1 + (levels - 1) + 1


def test_qr_full_size_4m_x_32(oracle, T):
    """The benchmark's workload at full size."""
    _check(oracle, T, workloads.gaussian(4194304, 32, seed=0))


def test_qr_argument_errors(T):
    import torch
    with pytest.raises(T.TsqrError) as e:
        T.tsqr_qr(torch.zeros(8, 4, dtype=torch.float64, device="cuda").T)  # m = 4 < n = 8
    assert e.value.status == T.ERR_INVALID_ARG
    # a binary tile of 20,001 rows is taller than any chunk (a multiple of 32 W rows), so it is
    # folded in chunks that do not divide it
    with pytest.raises(T.TsqrError) as e:
        T.tsqr_qr(workloads.gaussian(50000, 32, seed=1).cuda().T,
                  plan=T.make_plan("binary", tile_rows=20001))
    assert e.value.status == T.ERR_UNSUPPORTED


def test_qr_rank_deficient(oracle, T):
    """Rank-deficient A has no unique Q; what holds is A = Q R with R the (valid) R factor.
    The zero matrix gives R = 0; two equal columns give a zero (to rounding) R(1,1)."""
    import torch
    Z = torch.zeros(8, 100, dtype=torch.float64, device="cuda").T
    Q, R = T.tsqr_qr(Z)
    torch.cuda.synchronize()
    assert np.all(R.cpu().numpy() == 0) and np.all(np.isfinite(Q.cpu().numpy()))
    At = workloads.gaussian(50000, 6, seed=9)
    At[3] = At[1]
    A = oracle.from_torch_colmajor(At)
    Q, R = T.tsqr_qr(At.cuda().T)
    Qh, Rh = Q.cpu().numpy(), R.cpu().numpy()
    assert oracle.gram_residual(A, Rh) <= 1e-13
    assert np.linalg.norm(A - Qh @ Rh) / np.linalg.norm(A) <= _c(50000) * 6 * U


def test_last_plan(T):
    """tsqr_last_plan: tsqr_r's is the resolved AUTO plan (panels at n = 64) and, passed back,
    gives the same bytes; tsqr_qr factorizes with one reduction, and where that plan's
    twelve-warp chunks are too tall for the Q passes (n = 64) with four warps, and reports it; a
    call that fails reports a zero plan."""
    import torch
    m = 200003
    Ad = workloads.gaussian(m, 64, seed=12).cuda().T
    R1 = T.tsqr_r(Ad).clone()
    p = T.last_plan()
    auto = T.tsqr_resolve_plan(m, 64)
    assert (p.tree, p.tile_rows, p.ctas, p.warps, p.arity) == \
        (auto.tree, auto.tile_rows, auto.ctas, auto.warps, auto.arity)
    assert torch.equal(T.tsqr_r_ex(Ad, plan=p), R1)
    Q, R = T.tsqr_qr(Ad)
    q = T.last_plan()
    assert auto.tree == T.TREE_PANELS and auto.tile_rows == 16
    assert q.tree == T.TREE_HYBRID and q.warps == 4
    assert T.tsqr_resolve_plan(m, 64, plan=T.make_plan("hybrid")).warps == 12
    assert torch.equal(T.tsqr_r_ex(Ad, plan=q), R)
    with pytest.raises(T.TsqrError):
        T.tsqr_qr(torch.zeros(8, 4, dtype=torch.float64, device="cuda").T)
    z = T.last_plan()
    assert (z.tree, z.tile_rows, z.ctas, z.warps, z.arity) == (0, 0, 0, 0, 0)



@pytest.mark.parametrize("n", [9, 13, 20, 36, 41, 52])
def test_qr_widths_whose_auto_plan_has_other_warp_counts(oracle, T, n):
    """Where tsqr_r's AUTO plan runs 3, 5, 6, 7 or 9 bulk warps, tsqr_qr takes four (its passes
    run 4, 8 or 12) and still equals tsqr_r under that plan; explicit plans with other counts
    are refused."""
    m = 60013
    At = workloads.gaussian(m, n, seed=400 + n)
    _check(oracle, T, At)
    assert T.last_plan().warps % 4 == 0
    with pytest.raises(T.TsqrError) as e:
        T.tsqr_qr(At.cuda().T, plan=T.make_plan("hybrid", warps=6))
    assert e.value.status == T.ERR_INVALID_ARG
