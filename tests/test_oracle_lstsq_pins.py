"""Pins of the oracle's least-squares solve (``lstsq``: the thin Householder QR, then
X = R^-1 Q^T B by back substitution), each against something other than the oracle:

* consistent systems: B = A X0 with a planted X0 is solved exactly, X = X0 to c kappa u;
* closed forms: n = 1 gives x = a.b / a.a; a square nonsingular A gives A^-1 B (LAPACK's solve);
* LAPACK's least squares (numpy.linalg.lstsq) within the perturbation bound of the problem,
  c (kappa + kappa^2 ||r|| / (||A|| ||X||)) u;
* the normal equations: A^T (A X - B) = 0 to working accuracy."""
import numpy as np
import pytest

from test_oracle_pins import U


def _rel(X, Y):
    return np.linalg.norm(X - Y) / np.linalg.norm(Y)


@pytest.mark.parametrize("m,n,k,kappa", [(200, 5, 1, 1.0), (1000, 12, 3, 1e3), (3000, 24, 2, 1e6)])
def test_lstsq_consistent_system(oracle, m, n, k, kappa):
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n)) @ np.diag(np.geomspace(1.0, 1.0 / kappa, n))
    X0 = rng.standard_normal((n, k))
    X = oracle.lstsq(A, A @ X0)
    assert _rel(X, X0) <= 50 * np.linalg.cond(A) * U


def test_lstsq_single_column(oracle):
    rng = np.random.default_rng(1)
    a, b = rng.standard_normal(500), rng.standard_normal(500)
    x = oracle.lstsq(a[:, None], b)
    assert abs(x[0] - (a @ b) / (a @ a)) <= 20 * U * abs(x[0]) + 20 * U


def test_lstsq_square_is_solve(oracle):
    rng = np.random.default_rng(2)
    A = rng.standard_normal((40, 40)) + 10 * np.eye(40)
    B = rng.standard_normal((40, 3))
    np.testing.assert_allclose(oracle.lstsq(A, B), np.linalg.solve(A, B), rtol=0,
                               atol=50 * np.linalg.cond(A) * U * np.abs(np.linalg.solve(A, B)).max())


@pytest.mark.parametrize("m,n,kappa", [(800, 10, 1.0), (5000, 20, 1e4)])
def test_lstsq_matches_lapack_and_normal_equations(oracle, m, n, kappa):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((m, n)) @ np.diag(np.geomspace(1.0, 1.0 / kappa, n))
    B = rng.standard_normal((m, 2))
    X = oracle.lstsq(A, B)
    Xl = np.linalg.lstsq(A, B, rcond=None)[0]
    kap = np.linalg.cond(A)
    r = B - A @ X
    bound = 50 * (kap + kap ** 2 * np.linalg.norm(r) / (np.linalg.norm(A, 2) * np.linalg.norm(X))) * U
    assert _rel(X, Xl) <= bound
    assert np.linalg.norm(A.T @ r) <= 50 * m * U * np.linalg.norm(A) * (np.linalg.norm(A) * np.linalg.norm(X) + np.linalg.norm(B))


def test_back_substitution_closed_form(oracle):
    R = np.triu(np.arange(1.0, 10.0).reshape(3, 3)) + np.eye(3)
    C = R @ np.array([[1.0], [-2.0], [0.5]])
    np.testing.assert_allclose(oracle.back_substitute(R, C), [[1.0], [-2.0], [0.5]], rtol=0, atol=1e-14)
