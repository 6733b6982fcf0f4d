"""Pins of the oracle's thin Q factor (``householder_qr``), each against something other than
the oracle itself:

* planted factors: A = Q0 R0 with Q0 = H_1 ... H_n [I; 0] built from known reflectors and R0
  upper with a positive diagonal, so Q = Q0 (the QR factorization with diag(R) > 0 is unique,
  Section 2);
* closed forms: n = 1 gives Q = a / ||a||; mutually orthogonal columns give
  Q = A diag(1 / ||a_k||) and R = diag(||a_k||);
* the triangular-solve route Q = A R^-1 and LAPACK's QR (numpy.linalg.qr) after the same sign
  convention;
* invariants: Q^T Q = I and A = Q R to working accuracy, R identical to ``householder_r``'s,
  and a result independent of the thread count.

Tolerances: forward errors scale with kappa(A) u (u = 2^-53), as for R; the orthogonality and
backward errors are bounded by m n u (the a-priori bound of Householder QR is a small multiple
of that)."""
import numpy as np
import pytest

from test_oracle_pins import U, _planted_q0, _rand_upper


def _rel(X, Y):
    return np.linalg.norm(X - Y) / np.linalg.norm(Y)


@pytest.mark.parametrize("m,n,kappa", [(40, 5, 10.0), (300, 16, 1e3), (2000, 32, 1e6), (64, 64, 1e2)])
def test_q_planted(oracle, m, n, kappa):
    rng = np.random.default_rng(7 * m + n)
    R0 = _rand_upper(rng, n, kappa)
    Q0 = _planted_q0(rng, m, n)
    A = Q0 @ R0
    kap = np.linalg.cond(R0)
    Q, R = oracle.householder_qr(A)
    assert _rel(R, R0) <= 50 * kap * U
    assert _rel(Q, Q0) <= 50 * kap * U


def test_q_single_column(oracle):
    rng = np.random.default_rng(3)
    a = rng.standard_normal((777, 1)) * 3.0
    Q, R = oracle.householder_qr(a)
    nrm = np.linalg.norm(a)
    assert abs(R[0, 0] - nrm) <= 4 * U * nrm
    np.testing.assert_allclose(Q, a / nrm, rtol=0, atol=8 * U)


def test_q_orthogonal_columns(oracle):
    # columns of a Hadamard matrix of order 16, scaled: mutually orthogonal
    H = np.array([[1.0]])
    while H.shape[0] < 16:
        H = np.block([[H, H], [H, -H]])
    d = np.geomspace(1.0, 1e3, 6)
    A = H[:, :6] * d
    Q, R = oracle.householder_qr(A)
    np.testing.assert_allclose(Q, H[:, :6] / 4.0, rtol=0, atol=16 * U)
    np.testing.assert_allclose(R, np.diag(4.0 * d), rtol=0, atol=16 * U * 4e3)


@pytest.mark.parametrize("m,n", [(1000, 7), (513, 32), (50, 50), (4097, 3)])
def test_q_invariants(oracle, m, n):
    rng = np.random.default_rng(m * n)
    A = rng.standard_normal((m, n))
    Q, R = oracle.householder_qr(A, nthreads=3)
    assert np.abs(Q.T @ Q - np.eye(n)).max() <= m * n * U
    assert np.linalg.norm(A - Q @ R) / np.linalg.norm(A) <= m * n * U
    assert np.array_equal(R, oracle.householder_r(A))
    assert np.all(np.diag(R) >= 0) and np.all(np.tril(R, -1) == 0)
    Q1, R1 = oracle.householder_qr(A, nthreads=1)
    assert np.array_equal(Q1, Q) and np.array_equal(R1, R)


@pytest.mark.parametrize("m,n,kappa", [(800, 12, 1.0), (3000, 20, 1e4)])
def test_q_matches_triangular_solve_and_lapack(oracle, m, n, kappa):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(n)
    A = rng.standard_normal((m, n)) @ np.diag(np.geomspace(1.0, 1.0 / kappa, n))
    Q, R = oracle.householder_qr(A)
    kap = np.linalg.cond(A)
    Qs = scipy_linalg.solve_triangular(R, A.T, trans="T", lower=False).T  # A R^-1
    assert _rel(Q, Qs) <= 50 * kap * U
    Ql, Rl = np.linalg.qr(A, mode="reduced")
    D = np.sign(np.diag(Rl))
    assert _rel(Q, Ql * D) <= 50 * kap * U
    assert _rel(R, D[:, None] * Rl) <= 50 * kap * U


def test_q_rejects_wide(oracle):
    with pytest.raises(RuntimeError):
        oracle.householder_qr(np.ones((3, 5)))
