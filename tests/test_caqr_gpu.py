"""GPU parity of tsqr_caqr_r (R of a general m x n matrix by TSQR panels and trailing updates,
Section 5) against the CPU oracle's unblocked Householder R, through the C ABI.

The panels change only the order of the arithmetic, so R is the oracle's up to rounding.  The
bound on R's error grows with the rows and the columns the reflectors run over: every entry is
held to c(m, n) kappa u ||R_oracle||_F with c(m, n) = max(50, 2 sqrt(m n / 32)), which is the
TSQR tests' c(m) = max(50, 2 sqrt(m)) at n = 32.  The Gram residual ||R^T R - A^T A||_F /
||A||_F^2 must stay below 1e-13 as for tsqr_r.  At a size the oracle cannot factor in seconds
the tests use what holds at any size: R's leading panel block is the R of A's first panel,
sampled column norms are kept (||R(:, j)|| = ||A(:, j)||), and sampled Gram entries
(R^T R)(i, j) = A(:, i) . A(:, j) are checked against compensated dot products."""
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


def _c(m, n):
    return max(50.0, 2.0 * np.sqrt(max(m, 1) * max(n, 1) / 32.0))


def _check(oracle, T, At, panel=0, plan=None):
    """At: (n, m) CPU FP64 tensor holding the column-major input."""
    A = oracle.from_torch_colmajor(At)
    m, n = A.shape
    R = T.tsqr_caqr_r(At.cuda().T, panel=panel, plan=plan).cpu().numpy()
    Ro = oracle.householder_r(A, nthreads=16)
    kap = oracle.kappa_from_r(Ro)
    assert np.all(np.tril(R, -1) == 0.0) and np.all(np.diag(R) >= 0.0)
    np.testing.assert_allclose(R, Ro, rtol=0, atol=_c(m, n) * kap * U * np.linalg.norm(Ro))
    assert oracle.gram_residual(A, R, nthreads=16) <= 1e-13
    return R


@pytest.mark.parametrize("m,n,panel", [(20000, 200, 32), (30011, 150, 0), (5000, 300, 64),
                                       (12345, 100, 48), (40000, 97, 16), (9000, 129, 128),
                                       (65537, 256, 32), (385, 200, 32), (257, 130, 64)])
def test_caqr_gaussian(oracle, T, m, n, panel):
    _check(oracle, T, workloads.gaussian(m, n, seed=n), panel=panel)


def test_caqr_square_and_small(oracle, T):
    _check(oracle, T, workloads.gaussian(300, 300, seed=1), panel=32)   # m = n
    _check(oracle, T, workloads.gaussian(1000, 10, seed=2), panel=1)    # one column per panel
    _check(oracle, T, workloads.gaussian(257, 3, seed=3), panel=2)
    _check(oracle, T, workloads.gaussian(1, 1, seed=4))


@pytest.mark.parametrize("n", [24, 32])
def test_caqr_one_panel_is_tsqr_r(T, n):
    """One panel (panel >= n) is the TSQR factorization itself: R is tsqr_r's bit for bit under
    the plan the call reports (tsqr_r's AUTO plan where it runs 4, 8 or 12 bulk warps: n = 32;
    else the four-warp plan the reflector-keeping passes take: n = 24)."""
    At = workloads.gaussian(100003, n, seed=5)
    R = T.tsqr_caqr_r(At.cuda().T, panel=32)
    assert T.capi.tsqr_last_launch_count() == 1
    used = T.last_plan()
    assert used.warps % 4 == 0
    assert np.array_equal(R.cpu().numpy(), T.tsqr_r_ex(At.cuda().T, plan=used).cpu().numpy())
    if T.tsqr_resolve_plan(100003, n).warps % 4 == 0:
        assert np.array_equal(R.cpu().numpy(), T.tsqr_r(At.cuda().T).cpu().numpy())


def test_caqr_conditioned(oracle, T):
    _check(oracle, T, workloads.conditioned(60000, 160, 1e8, seed=0), panel=32)


@pytest.mark.parametrize("tree,b,ctas,arity", [("flat", 0, 0, 0), ("binary", 256, 0, 0),
                                               ("hybrid", 0, 37, 3), ("hybrid", 0, 100, 8)])
def test_caqr_plans(oracle, T, tree, b, ctas, arity):
    """Every panel on the given tree: the leaves, and so the rows each update leaves behind
    ((leaves - 1) panel rows per panel), differ from plan to plan; R does not."""
    At = workloads.gaussian(50001, 100, seed=6)
    _check(oracle, T, At, panel=32, plan=T.make_plan(tree, tile_rows=b, ctas=ctas, arity=arity))


def test_caqr_leading_dimensions(oracle, T):
    import torch
    m, n = 23456, 70
    At = workloads.gaussian(m, n, seed=7)
    big = torch.zeros(n, m + 9, dtype=torch.float64)
    big[:, :m] = At
    Rbig = torch.full((n, n + 5), float("nan"), dtype=torch.float64, device="cuda")
    R = T.tsqr_caqr_r(big.cuda().T[:m, :], panel=32, R=Rbig.T[:n, :])
    A = oracle.from_torch_colmajor(At)
    Ro = oracle.householder_r(A, nthreads=16)
    tol = _c(m, n) * oracle.kappa_from_r(Ro) * U * np.linalg.norm(Ro)
    np.testing.assert_allclose(R.cpu().numpy(), Ro, rtol=0, atol=tol)
    assert torch.isnan(Rbig[:, n:]).all()  # the padding rows of R are not written


def test_caqr_bit_reproducible_and_launches(T):
    import torch
    Ad = workloads.gaussian(200000, 100, seed=8).cuda().T
    R1 = T.tsqr_caqr_r(Ad, panel=32).clone()
    # panels of 32, 32, 32, 4: the factorization, the chunks' compact WY factors and the update
    # for each but the last, the last one's factorization alone
    assert T.capi.tsqr_last_launch_count() == 3 * 3 + 1
    R2 = T.tsqr_caqr_r(Ad, panel=32)
    torch.cuda.synchronize()
    assert torch.equal(R1, R2)


def test_caqr_large_properties(oracle, T):
    """262,144 x 512 (1 GiB): the leading panel block against the oracle's R of the first
    panel, and sampled column norms and Gram entries against compensated dot products."""
    m, n, nb = 262144, 512, 32
    At = workloads.gaussian(m, n, seed=9)
    R = T.tsqr_caqr_r(At.cuda().T, panel=nb).cpu().numpy()
    A = oracle.from_torch_colmajor(At)
    R0 = oracle.householder_r(np.asfortranarray(A[:, :nb]), nthreads=16)
    np.testing.assert_allclose(R[:nb, :nb], R0, rtol=0,
                               atol=_c(m, nb) * oracle.kappa_from_r(R0) * U * np.linalg.norm(R0))
    # columns 0 and n - 1 and ten more: their norms and every Gram entry among them, each
    # within c(m, n) u ||a_i|| ||a_j|| (the columnwise backward error of Householder QR)
    rng = np.random.default_rng(0)
    pick = np.unique(np.concatenate([[0, n - 1], rng.choice(n, 10, replace=False)]))
    G = oracle.gram_dot2(np.asfortranarray(A[:, pick]), nthreads=16)
    cn = np.sqrt(np.diag(G))
    tol = _c(m, n) * U
    np.testing.assert_allclose(np.linalg.norm(R[:, pick], axis=0), cn, rtol=tol, atol=0)
    Gr = R[:, pick].T @ R[:, pick]
    assert np.all(np.abs(Gr - G) <= tol * np.outer(cn, cn))


def test_caqr_rank_deficient_and_nonfinite(oracle, T):
    """Rank-deficient A (a zero column, two equal columns) has no unique R beyond the rank, but
    R^T R = A^T A still holds; a NaN in A is reported as TSQR_STATUS_NONFINITE."""
    import torch
    At = workloads.gaussian(30000, 70, seed=13)
    At[5] = 0.0
    At[40] = At[7]
    A = oracle.from_torch_colmajor(At)
    R = T.tsqr_caqr_r(At.cuda().T, panel=16).cpu().numpy()
    assert np.all(np.isfinite(R)) and np.all(np.diag(R) >= 0.0)
    assert oracle.gram_residual(A, R, nthreads=16) <= 1e-13
    T.tsqr_get_device_status()  # clears the status word
    At[3, 1234] = float("nan")
    T.tsqr_caqr_r(At.cuda().T, panel=16)
    torch.cuda.synchronize()
    assert T.tsqr_get_device_status() == T.STATUS_NONFINITE


def test_tsqr_r_beyond_128_columns_is_panels(oracle, T):
    """tsqr_r and tsqr_r_ex take any tall n by panels: above 128 columns the AUTO plan is
    PANELS, and R equals tsqr_caqr_r's with the default panel byte for byte."""
    import torch
    At = workloads.gaussian(25000, 200, seed=14)
    Ad = At.cuda().T
    R = T.tsqr_r(Ad)
    assert torch.equal(R, T.tsqr_caqr_r(Ad))
    assert torch.equal(T.tsqr_r_ex(Ad), R)
    p = T.tsqr_resolve_plan(25000, 200)
    assert (p.tree, p.tile_rows) == (T.TREE_PANELS, 16)
    _check(oracle, T, At)
    with pytest.raises(T.TsqrError) as e:  # wide (m < n) above 128 columns
        T.tsqr_r(torch.zeros(200, 150, dtype=torch.float64, device="cuda").T)
    assert e.value.status == T.ERR_UNSUPPORTED


def test_caqr_argument_errors(T):
    import torch
    A = torch.zeros(8, 100, dtype=torch.float64, device="cuda").T
    for kw in ({"panel": -1}, {"panel": 129}):
        with pytest.raises(T.TsqrError) as e:
            T.tsqr_caqr_r(A, **kw)
        assert e.value.status in (T.ERR_INVALID_ARG, T.ERR_UNSUPPORTED)
    with pytest.raises(T.TsqrError) as e:
        T.tsqr_caqr_r(torch.zeros(8, 4, dtype=torch.float64, device="cuda").T)  # m < n
    assert e.value.status == T.ERR_INVALID_ARG
