"""Pins of the CPU oracle against things other than itself (CPU only).

The paper prints no worked example and no error values, so the oracle is pinned by:
hand-derived closed forms (tests/golden), a planted R0 = R(Q0 R0) with Q0 built from
known reflectors, a multiprecision Cholesky of the exact Gram matrix, LAPACK's QR, exact
invariances (power-of-two scaling, positive column scaling, the identity-reflector path),
the algebraic properties of Section 2 (associativity and commutativity of qr(R1, R2) up to
row signs, tree independence) and the operator's cost claim in Table 3 (2/3 n^3).
"""
import fractions
import glob
import math
import os

import numpy as np
import pytest

U = np.finfo(np.float64).eps / 2  # unit roundoff 2^-53
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(path):
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([float(x) for x in line.split()])
    m, n = int(rows[0][0]), int(rows[0][1])
    A = np.array(rows[1:1 + m], dtype=np.float64).reshape(m, n)
    R = np.array(rows[1 + m:1 + m + n], dtype=np.float64).reshape(n, n)
    return A, R


GOLDEN_FILES = sorted(glob.glob(os.path.join(GOLDEN, "g*.txt")))


def _rand_upper(rng, n, kappa=10.0):
    """Upper triangle with positive diagonal and modest condition number."""
    R = np.triu(rng.standard_normal((n, n))) / np.sqrt(n)
    d = np.geomspace(1.0, 1.0 / kappa, n)
    R[np.diag_indices(n)] = d * (1.0 + 0.1 * rng.random(n))
    return R


def _planted_q0(rng, m, n):
    """Q0 = H_1 H_2 ... H_n [I_n; 0] with H_k = I - 2 u_k u_k^T, u_k known unit vectors."""
    Q = np.zeros((m, n))
    Q[:n, :n] = np.eye(n)
    for _ in range(n):
        u = rng.standard_normal(m)
        u /= np.linalg.norm(u)
        Q = Q - 2.0 * np.outer(u, u @ Q)
    return Q


def _mp_cholesky_r(A, dps=50):
    """Upper Cholesky factor of the EXACT Gram matrix, in mpmath with `dps` digits."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = dps
    m, n = A.shape
    F = [[fractions.Fraction(float(A[i, k])) for k in range(n)] for i in range(m)]
    G = [[sum(F[i][k] * F[i][l] for i in range(m)) for l in range(n)] for k in range(n)]
    Gm = [[mpmath.mpf(g.numerator) / g.denominator for g in row] for row in G]
    Rm = [[mpmath.mpf(0)] * n for _ in range(n)]
    for k in range(n):
        d = Gm[k][k] - sum(Rm[i][k] ** 2 for i in range(k))
        Rm[k][k] = mpmath.sqrt(d)
        for l in range(k + 1, n):
            Rm[k][l] = (Gm[k][l] - sum(Rm[i][k] * Rm[i][l] for i in range(k))) / Rm[k][k]
    return np.array([[float(x) for x in row] for row in Rm])


# ----------------------------------------------------------------------------------------
# hand-derived closed forms
# ----------------------------------------------------------------------------------------
@pytest.mark.parametrize("path", GOLDEN_FILES, ids=[os.path.basename(p) for p in GOLDEN_FILES])
def test_golden_householder(oracle, path):
    A, Rg = _read_golden(path)
    R = oracle.householder_r(A)
    tol = 8 * U * max(1.0, np.abs(A).max()) * A.shape[0]
    np.testing.assert_allclose(R, Rg, rtol=0, atol=tol)
    assert np.all(np.diag(R) >= 0)
    assert np.all(np.tril(R, -1) == 0)


@pytest.mark.parametrize("path", GOLDEN_FILES, ids=[os.path.basename(p) for p in GOLDEN_FILES])
@pytest.mark.parametrize("tree,b", [("binary", 1), ("flat", 1), ("binary", 2), ("hybrid", 2)])
def test_golden_tsqr(oracle, path, tree, b):
    A, Rg = _read_golden(path)
    R = oracle.tsqr_r(A, b=b, tree=tree, group=2)
    tol = 16 * U * max(1.0, np.abs(A).max()) * A.shape[0]
    np.testing.assert_allclose(R, Rg, rtol=0, atol=tol)


def test_golden_files_present():
    assert len(GOLDEN_FILES) >= 10


# ----------------------------------------------------------------------------------------
# special cases with exact answers
# ----------------------------------------------------------------------------------------
def test_single_column_is_the_norm(oracle):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(1)
    for m in (1, 2, 7, 1000):
        a = rng.standard_normal(m) * 10.0 ** rng.integers(-5, 5)
        exact = mpmath.sqrt(sum(mpmath.mpf(float(x)) ** 2 for x in a))
        R = oracle.householder_r(a.reshape(m, 1))
        assert R.shape == (1, 1)
        # a-priori bound of a recursive sum of m scaled squares, halved by the square root
        assert abs(R[0, 0] - float(exact)) <= (m / 2 + 3) * U * float(exact)


def test_single_column_extreme_scale_does_not_overflow(oracle):
    a = np.array([3e200, 4e200, 0.0])
    assert oracle.householder_r(a.reshape(3, 1))[0, 0] == pytest.approx(5e200, rel=4 * U)
    b = np.array([3e-200, 4e-200])
    assert oracle.householder_r(b.reshape(2, 1))[0, 0] == pytest.approx(5e-200, rel=4 * U)


def test_r0_over_zero_block_is_exact(oracle):
    """[R0; 0]: every reflector is the identity (tau = 0), so R is R0 bit for bit."""
    rng = np.random.default_rng(2)
    for n in (1, 3, 16):
        R0 = _rand_upper(rng, n)
        A = np.vstack([R0, np.zeros((5, n))])
        assert np.array_equal(oracle.householder_r(A), R0)
        assert np.array_equal(oracle.tsqr_r(A, b=n, tree="binary"), R0)


def test_stacked_copies_give_sqrt2(oracle):
    rng = np.random.default_rng(3)
    for n in (2, 8, 32):
        R0 = _rand_upper(rng, n)
        R = oracle.householder_r(np.vstack([R0, R0]))
        kap = np.linalg.cond(R0)
        assert oracle.rel_err(R, math.sqrt(2.0) * R0) <= 50 * kap * U


def test_orthogonal_columns_give_diagonal(oracle):
    # Sylvester Hadamard matrix: orthogonal +-1 columns of norm sqrt(m)
    H = np.array([[1.0]])
    while H.shape[0] < 64:
        H = np.block([[H, H], [H, -H]])
    d = np.array([1.0, 2.0, 0.5, 8.0, 3.0, 0.25, 1.5, 6.0])
    A = H[:, :8] * d
    R = oracle.householder_r(A)
    np.testing.assert_allclose(R, np.diag(d * 8.0), rtol=0, atol=64 * U * 8.0 * 8.0)


def test_empty_and_degenerate(oracle):
    R = oracle.householder_r(np.zeros((0, 4)))
    assert R.shape == (4, 4) and np.all(R == 0)
    R = oracle.householder_r(np.zeros((10, 3)))
    assert np.all(R == 0)
    R = oracle.tsqr_r(np.zeros((0, 3)), b=4)
    assert np.all(R == 0)


# ----------------------------------------------------------------------------------------
# planted R0 and independent solvers
# ----------------------------------------------------------------------------------------
@pytest.mark.parametrize("m,n,kappa", [(40, 5, 10.0), (300, 16, 1e3), (2000, 32, 1e6)])
def test_planted_r0(oracle, m, n, kappa):
    rng = np.random.default_rng(m + n)
    R0 = _rand_upper(rng, n, kappa)
    Q0 = _planted_q0(rng, m, n)
    A = Q0 @ R0
    kap = np.linalg.cond(R0)
    R = oracle.householder_r(A)
    assert oracle.rel_err(R, R0) <= 50 * kap * U
    Rt = oracle.tsqr_r(A, b=max(n, m // 7), tree="binary")
    assert oracle.rel_err(Rt, R0) <= 50 * kap * U


@pytest.mark.parametrize("m,n", [(3, 2), (8, 3), (12, 5), (30, 6)])
def test_multiprecision_cholesky(oracle, m, n):
    rng = np.random.default_rng(10 * m + n)
    A = rng.standard_normal((m, n))
    Rmp = _mp_cholesky_r(A)
    kap = np.linalg.cond(A)
    assert oracle.rel_err(oracle.householder_r(A), Rmp) <= 50 * kap * U
    # long double Cholesky squares the condition number but carries >= 64-bit mantissas
    assert oracle.rel_err(oracle.cholesky_r_ld(A), Rmp) <= 50 * kap * kap * U


def test_long_double_cholesky_brute_force(oracle):
    rng = np.random.default_rng(5)
    for m, n in [(8, 2), (40, 6), (64, 8)]:
        A = rng.standard_normal((m, n))
        kap = np.linalg.cond(A)
        assert kap < 1e3
        Rc = oracle.cholesky_r_ld(A)
        assert oracle.rel_err(oracle.householder_r(A), Rc) <= 50 * kap * kap * U


@pytest.mark.parametrize("m,n,kappa", [(500, 8, 1.0), (3000, 32, 1e4), (1000, 64, 1e8)])
def test_lapack_cross_check(oracle, m, n, kappa):
    rng = np.random.default_rng(7)
    G = rng.standard_normal((m, n))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = G @ np.diag(np.geomspace(1, 1 / kappa, n)) @ V.T
    R_lapack = np.linalg.qr(A, mode="r")
    R_lapack = R_lapack * np.sign(np.diag(R_lapack))[:, None]
    R = oracle.householder_r(A)
    kap = np.linalg.cond(R)
    assert oracle.rel_err(R, R_lapack) <= 50 * kap * U


# ----------------------------------------------------------------------------------------
# exact invariances
# ----------------------------------------------------------------------------------------
def test_power_of_two_scaling_is_exact(oracle):
    rng = np.random.default_rng(11)
    A = rng.standard_normal((200, 12))
    R = oracle.householder_r(A)
    for alpha in (2.0, 0.125, -4.0, -1.0):
        assert np.array_equal(oracle.householder_r(alpha * A), abs(alpha) * R)


def test_positive_column_scaling(oracle):
    rng = np.random.default_rng(12)
    A = rng.standard_normal((300, 10))
    d = 2.0 ** rng.integers(-3, 4, size=10)
    R = oracle.householder_r(A)
    Rd = oracle.householder_r(A * d)
    np.testing.assert_allclose(Rd, R * d, rtol=0, atol=64 * U * np.abs(R * d).max())


def test_row_permutation_invariance(oracle):
    rng = np.random.default_rng(13)
    A = rng.standard_normal((500, 16))
    P = rng.permutation(500)
    R = oracle.householder_r(A)
    kap = np.linalg.cond(R)
    assert oracle.rel_err(oracle.householder_r(A[P]), R) <= 50 * kap * U


def test_thread_count_is_bitwise_invisible(oracle):
    rng = np.random.default_rng(14)
    A = rng.standard_normal((5000, 24))
    R1 = oracle.householder_r(A, nthreads=1)
    for t in (2, 3, 8):
        assert np.array_equal(oracle.householder_r(A, nthreads=t), R1)


def test_gram_residual_of_householder(oracle):
    rng = np.random.default_rng(15)
    A = rng.standard_normal((20000, 16))
    R = oracle.householder_r(A)
    res = oracle.gram_residual(A, R)
    assert res <= 1e-14  # well inside the 1e-13 FP64 acceptance bound
    # a perturbation of one entry by 1e-12 relative is seen by the compensated checker
    R2 = R.copy()
    R2[3, 7] += 1e-12 * np.abs(R).max()
    assert oracle.gram_residual(A, R2) > 10 * res


# ----------------------------------------------------------------------------------------
# the reduction operator qr(R1, R2) (Section 2, Table 3)
# ----------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 5, 16, 33, 64])
def test_operator_equals_dense_qr_of_stack(oracle, n):
    rng = np.random.default_rng(100 + n)
    R1, R2 = _rand_upper(rng, n), _rand_upper(rng, n)
    Rop, V, tau = oracle.qr_uppers(R1, R2)
    Rop = oracle.sign_fix(Rop)
    stack = np.vstack([R1, R2])
    kap = np.linalg.cond(stack)
    assert oracle.rel_err(Rop, oracle.householder_r(stack)) <= 50 * kap * U
    Rl = np.linalg.qr(stack, mode="r")
    Rl = Rl * np.sign(np.diag(Rl))[:, None]
    assert oracle.rel_err(Rop, Rl) <= 50 * kap * U
    # V keeps the triangle: reflector j has support R1(j,j) and R2(0:j, j) only
    assert np.all(np.tril(V, -1) == 0)


def test_operator_reflectors_reproduce_the_stack(oracle):
    """Applying the stored reflectors H_0 ... H_{n-1} to [R; 0] gives back [R1; R2]."""
    rng = np.random.default_rng(21)
    n = 7
    R1, R2 = _rand_upper(rng, n), _rand_upper(rng, n)
    Rraw, V, tau = oracle.qr_uppers(R1, R2)
    Y = np.vstack([np.triu(Rraw), np.zeros((n, n))])
    for j in reversed(range(n)):
        u = np.zeros(2 * n)
        u[j] = 1.0
        u[n:n + j + 1] = V[:j + 1, j]
        Y = Y - tau[j] * np.outer(u, u @ Y)
    np.testing.assert_allclose(Y, np.vstack([R1, R2]), rtol=0, atol=1e-14 * 8)


def test_operator_associative_and_commutative(oracle):
    rng = np.random.default_rng(22)
    n = 12
    R1, R2, R3 = (_rand_upper(rng, n) for _ in range(3))

    def op(a, b):
        return np.triu(oracle.qr_uppers(a, b)[0])

    left = oracle.sign_fix(op(op(R1, R2), R3))
    right = oracle.sign_fix(op(R1, op(R2, R3)))
    kap = np.linalg.cond(np.vstack([R1, R2, R3]))
    assert oracle.rel_err(left, right) <= 50 * kap * U
    assert oracle.rel_err(oracle.sign_fix(op(R1, R2)), oracle.sign_fix(op(R2, R1))) <= 50 * kap * U


def test_operator_tau_zero_skip(oracle):
    """qr(R1, 0): all reflectors are identities, R1 comes back unchanged."""
    rng = np.random.default_rng(23)
    R1 = _rand_upper(rng, 9)
    R, V, tau = oracle.qr_uppers(R1, np.zeros((9, 9)))
    assert np.all(tau == 0) and np.array_equal(R, R1)


def test_operator_cost_is_two_thirds_n_cubed(oracle):
    """Table 3's claim: the operator costs 2/3 n^3 (vs 10/3 n^3 for a dense 2n x n QR)."""
    rng = np.random.default_rng(24)
    for n in (64, 256):
        R1, R2 = _rand_upper(rng, n), _rand_upper(rng, n)
        _, _, _, flops = oracle.qr_uppers(R1, R2, count_flops=True)
        ratio = flops / (2.0 * n ** 3 / 3.0)
        assert 1.0 <= ratio <= 1.0 + 8.0 / n
        dense = 2.0 * (2 * n) * n ** 2 - 2.0 * n ** 3 / 3.0
        assert dense / flops == pytest.approx(5.0, rel=8.0 / n)


# ----------------------------------------------------------------------------------------
# TSQR: the tree does not change R (Section 2)
# ----------------------------------------------------------------------------------------
@pytest.mark.parametrize("m,n,b", [(1000, 16, 256), (777, 8, 50), (130, 32, 32), (20, 5, 3)])
def test_tree_independence(oracle, m, n, b):
    rng = np.random.default_rng(m * n)
    A = rng.standard_normal((m, n))
    R = oracle.householder_r(A)
    kap = np.linalg.cond(R)
    for tree in ("binary", "flat", "hybrid"):
        Rt = oracle.tsqr_r(A, b=b, tree=tree, group=3)
        assert oracle.rel_err(Rt, R) <= 50 * kap * U, tree
        assert np.all(np.diag(Rt) >= 0)


def test_tsqr_tile_shorter_than_n(oracle):
    rng = np.random.default_rng(31)
    A = rng.standard_normal((37, 10))
    R = oracle.householder_r(A)
    for b in (1, 3, 7, 10, 11):
        assert oracle.rel_err(oracle.tsqr_r(A, b=b, tree="binary"), R) <= 1e-13


# ----------------------------------------------------------------------------------------
# the Gram-residual check (compensated dot products)
# ----------------------------------------------------------------------------------------
def test_dot2_gram_is_compensated(oracle):
    # catastrophic cancellation: exact answer 1, naive summation gives 0
    A = np.array([[1e16, 1.0], [1.0, 1.0], [-1e16, 1.0]])
    G = oracle.gram_dot2(A)
    assert G[0, 1] == 1.0 and G[1, 0] == 1.0
    # the product's own rounding error matters: x.y = 2^-60 exactly, naive gives 0
    t = 2.0 ** -30
    D = np.array([[1 + t, 1 + t], [1.0, -(1 + 2 * t)]])
    assert oracle.gram_dot2(D)[0, 1] == 2.0 ** -60
    # integer matrix with an exactly representable Gram: compare with exact integers
    rng = np.random.default_rng(40)
    B = rng.integers(-2 ** 20, 2 ** 20, size=(5000, 4)).astype(np.float64)
    exact = [[sum(int(x) * int(y) for x, y in zip(B[:, k], B[:, l])) for l in range(4)]
             for k in range(4)]
    Gb = oracle.gram_dot2(B, nthreads=3)
    for k in range(4):
        for l in range(4):
            assert Gb[k, l] == float(exact[k][l])


def test_rel_err_and_kappa_helpers(oracle):
    R = np.diag([4.0, 2.0, 1.0])
    assert oracle.kappa_from_r(R) == pytest.approx(4.0)
    assert oracle.rel_err(R, R) == 0.0


def test_nearly_aligned_column_is_stable(oracle):
    """Column 0 almost parallel to e_1: with beta = +sign(alpha)||.|| the divisor alpha - beta
    would cancel to zero; the reflector's stable sign keeps full accuracy."""
    A = np.array([[1.0, 2.0], [1e-9, 3.0], [0.0, 4.0], [1e-12, -1.0]])
    Rmp = _mp_cholesky_r(A)
    kap = np.linalg.cond(A)
    R = oracle.householder_r(A)
    assert np.all(np.isfinite(R))
    assert oracle.rel_err(R, Rmp) <= 50 * kap * U
    assert oracle.rel_err(oracle.tsqr_r(A, b=2, tree="binary"), Rmp) <= 50 * kap * U
