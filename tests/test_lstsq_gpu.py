"""GPU parity of tsqr_lstsq against the CPU oracle's least squares (X = R^-1 Q^T B through its
Householder QR), through the C ABI, on both of its paths: few right-hand sides
(k <= max(1, n // 4), n + k <= 128) factorize [A | B] (its R holds (Q^T B)(0:n,:) beside R),
more apply Q^T to B with the stored reflectors.
Consistent systems B = A X0 must return X0 to c(m) kappa u; general B the oracle's X to
c(m) (kappa + kappa^2 ||r|| / (||A|| ||X||)) u, the perturbation bound of least squares.  R is
bit-identical to tsqr_r's on the stored-reflector path and within c(m) kappa u ||R|| of it on
the augmented one.  c(m) = max(50, 2 sqrt(m)) as elsewhere."""
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


def _bmat(m, k, seed):
    import torch
    g = torch.Generator().manual_seed(seed)
    return torch.randn(k, m, generator=g, dtype=torch.float64)  # (k, m): column-major (m, k)


def _check(oracle, T, At, Bt, plan=None):
    A = oracle.from_torch_colmajor(At)
    Bn = oracle.from_torch_colmajor(Bt)
    m, n = A.shape
    k = Bn.shape[1]
    X, R = T.tsqr_lstsq(At.cuda().T, Bt.cuda().T, plan=plan)
    augmented = k <= max(1, n // 4) and n + k <= 128
    # the stored-reflector path's factorization plan (the plan the call reports) gives a
    # bit-identical R
    used = plan if augmented else T.last_plan()
    Rr = T.tsqr_r_ex(At.cuda().T, plan=used).cpu().numpy()
    Xh = X.cpu().numpy()
    Xo = oracle.lstsq(A, Bn, nthreads=16)
    kap = oracle.kappa_from_r(oracle.householder_r(A, nthreads=16))
    if not augmented:
        assert np.array_equal(R.cpu().numpy(), Rr)
    else:
        np.testing.assert_allclose(R.cpu().numpy(), Rr, rtol=0,
                                   atol=_c(m) * kap * U * np.linalg.norm(Rr))
    res = np.linalg.norm(Bn - A @ Xo)
    tol = _c(m) * (kap + kap ** 2 * res / (np.linalg.norm(A, 2) * np.linalg.norm(Xo))) * U
    assert np.linalg.norm(Xh - Xo) <= tol * np.linalg.norm(Xo)
    return Xh


@pytest.mark.parametrize("m,n,k", [(100003, 32, 1), (50001, 16, 3), (20000, 8, 13), (65537, 64, 2),
                                   (3000, 1, 1), (777, 5, 5), (4194304, 32, 1),
                                   (50001, 16, 120), (20000, 8, 125), (65537, 64, 70),
                                   (300000, 32, 100), (129, 64, 40), (386, 32, 20)])
def test_lstsq_general_rhs(oracle, T, m, n, k):
    """(129, 64) and (386, 32) end in a leaf of one or two rows: its chunk runs out of rank, the
    later reflectors' tails are tiny and their scale c huge (only c x is well scaled)."""
    _check(oracle, T, workloads.gaussian(m, n, seed=m % 97), _bmat(m, k, seed=n))


@pytest.mark.parametrize("kappa", [1.0, 1e6])
def test_lstsq_consistent_system(oracle, T, kappa):
    import torch
    m, n, k = 200000, 24, 4
    At = workloads.conditioned(m, n, kappa, seed=2)
    X0 = torch.randn(n, k, generator=torch.Generator().manual_seed(3), dtype=torch.float64)
    Bt = (At.T @ X0).T.contiguous()  # (k, m): B = A X0
    X, _ = T.tsqr_lstsq(At.cuda().T, Bt.cuda().T)
    kap = oracle.kappa_from_r(oracle.householder_r(oracle.from_torch_colmajor(At), nthreads=16))
    err = np.linalg.norm(X.cpu().numpy() - X0.numpy()) / np.linalg.norm(X0.numpy())
    assert err <= _c(m) * kap * U


@pytest.mark.parametrize("tree,b,ctas,arity", [("binary", 256, 0, 0), ("flat", 0, 0, 0),
                                               ("hybrid", 0, 61, 5), ("hybrid", 0, 100, 8)])
def test_lstsq_trees(oracle, T, tree, b, ctas, arity):
    _check(oracle, T, workloads.gaussian(120001, 24, seed=11), _bmat(120001, 2, seed=5),
           plan=T.make_plan(tree, tile_rows=b, ctas=ctas, arity=arity))


def test_lstsq_vector_and_more_columns_than_n(oracle, T):
    import torch
    At = workloads.gaussian(30000, 6, seed=8)
    b = torch.randn(30000, generator=torch.Generator().manual_seed(9), dtype=torch.float64)
    x, _ = T.tsqr_lstsq(At.cuda().T, b.cuda())
    xo = oracle.lstsq(oracle.from_torch_colmajor(At), b.numpy())
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-12 * np.linalg.norm(xo)
    _check(oracle, T, At, _bmat(30000, 17, seed=4))    # stored reflectors: groups of 6 columns
    _check(oracle, T, At, _bmat(30000, 130, seed=4))


@pytest.mark.parametrize("m,n,k", [(20000, 200, 3), (30011, 150, 40), (5000, 129, 1)])
def test_lstsq_wide_by_panels(oracle, T, m, n, k):
    """Above 128 columns [A | B] is factorized by panels (as tsqr_caqr_r) and R X = C solved:
    X within the least-squares bound of the oracle's, with c(m, n) = max(50, 2 sqrt(m n / 32))
    as for the panels' R."""
    At = workloads.gaussian(m, n, seed=n)
    Bt = _bmat(m, k, seed=k)
    A = oracle.from_torch_colmajor(At)
    Bn = oracle.from_torch_colmajor(Bt)
    X, R = T.tsqr_lstsq(At.cuda().T, Bt.cuda().T)
    Xh = X.cpu().numpy()
    Xo = oracle.lstsq(A, Bn, nthreads=16)
    Ro = oracle.householder_r(A, nthreads=16)
    kap = oracle.kappa_from_r(Ro)
    c = max(50.0, 2.0 * np.sqrt(m * n / 32.0))
    np.testing.assert_allclose(R.cpu().numpy(), Ro, rtol=0, atol=c * kap * U * np.linalg.norm(Ro))
    res = np.linalg.norm(Bn - A @ Xo)
    tol = c * (kap + kap ** 2 * res / (np.linalg.norm(A, 2) * np.linalg.norm(Xo))) * U
    assert np.linalg.norm(Xh - Xo) <= tol * np.linalg.norm(Xo)


def test_lstsq_rank_deficient_and_errors(T):
    import torch
    At = workloads.gaussian(5000, 4, seed=1)
    At[2] = 0.0  # a zero column: R(2,2) = 0
    T.tsqr_get_device_status()
    X, _ = T.tsqr_lstsq(At.cuda().T, _bmat(5000, 1, seed=2).cuda().T)
    assert T.tsqr_get_device_status() == T.STATUS_NONFINITE
    with pytest.raises(T.TsqrError) as e:
        T.tsqr_lstsq(torch.zeros(8, 4, dtype=torch.float64, device="cuda").T,
                     torch.zeros(1, 4, dtype=torch.float64, device="cuda").T)
    assert e.value.status == T.ERR_INVALID_ARG
