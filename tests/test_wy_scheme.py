"""The compact WY form the blocked passes use, checked on the CPU with numpy: a chunk's
reflectors v_J = [e_J; c_J x_J] (row J of the carried triangle, then the chunk's rows) with
tau_J, and S built column by column from G(i, J) = (c_i x_i) . (c_J x_J) for i < J by
S(J, J) = tau_J, S(0:J, J) = -tau_J S(0:J, 0:J) G(0:J, J), must satisfy
H_0 H_1 ... H_{n-1} = I - V S V^T with V = [I; X diag(c)].  Both directions of its use are
checked against applying the reflectors one by one: Q^T (first to last) on [T; Z] and Q (last
to first) on [T; 0].  A chunk that runs out of rank has tiny tails and huge c: the product c x
stays well scaled while c_i c_J overflows, which is why the kernels scale the tails first."""
import numpy as np
import pytest


def _reflectors(n, h, rng, tau_zero=()):
    X = rng.standard_normal((h, n))
    c = rng.standard_normal(n) * 0.3
    tau = 2.0 / (1.0 + c ** 2 * (X ** 2).sum(axis=0))  # tau = 2 / ||v||^2
    for j in tau_zero:
        tau[j] = 0.0
    return X, c, tau


def _s_factor(Xs, tau):
    n = Xs.shape[1]
    G = Xs.T @ Xs
    S = np.zeros((n, n))
    for J in range(n):
        S[J, J] = tau[J]
        for i in range(J):
            S[i, J] = -tau[J] * sum(S[i, k] * G[k, J] for k in range(i, J))
    return S


def _apply_one_by_one(X, c, tau, T, Z, order):
    T, Z = T.copy(), Z.copy()
    for J in order:
        w = T[J] + c[J] * (X[:, J] @ Z)
        T[J] -= tau[J] * w
        Z -= np.outer(tau[J] * c[J] * X[:, J], w)
    return T, Z


@pytest.mark.parametrize("n,h,k,tz", [(7, 23, 5, (3,)), (16, 40, 9, ()), (1, 5, 3, ()),
                                      (12, 12, 12, (0, 11))])
def test_compact_wy_matches_reflectors(n, h, k, tz):
    rng = np.random.default_rng(n * 100 + h)
    X, c, tau = _reflectors(n, h, rng, tz)
    Xs = X * c
    S = _s_factor(Xs, tau)
    assert np.allclose(np.tril(S, -1), 0.0)
    # the product of the reflectors
    V = np.vstack([np.eye(n), Xs])
    H = np.eye(n + h)
    for J in range(n):
        v = V[:, J]
        H = H @ (np.eye(n + h) - tau[J] * np.outer(v, v))
    np.testing.assert_allclose(np.eye(n + h) - V @ S @ V.T, H, rtol=0, atol=1e-13)
    # Q^T on [T; Z], first to last: W = T + Xs^T Z, Y = S^T W, T -= Y, Z -= Xs Y
    T0, Z0 = rng.standard_normal((n, k)), rng.standard_normal((h, k))
    Tr, Zr = _apply_one_by_one(X, c, tau, T0, Z0, range(n))
    Y = S.T @ (T0 + Xs.T @ Z0)
    np.testing.assert_allclose(T0 - Y, Tr, rtol=0, atol=1e-13)
    np.testing.assert_allclose(Z0 - Xs @ Y, Zr, rtol=0, atol=1e-13)
    # Q on [T; 0], last to first: Y = S T, T -= Y, Z = -Xs Y
    Tq, Zq = _apply_one_by_one(X, c, tau, T0, np.zeros((h, k)), reversed(range(n)))
    Y = S @ T0
    np.testing.assert_allclose(T0 - Y, Tq, rtol=0, atol=1e-13)
    np.testing.assert_allclose(-Xs @ Y, Zq, rtol=0, atol=1e-13)


def test_scaled_tails_stay_finite_where_c_overflows():
    """Tiny tails with huge c (a chunk out of rank): c_i c_J overflows, c x does not."""
    x = np.array([1e-170, -2e-170, 3e-171])
    s = np.abs(x).max()
    c = 1.0 / (s * np.linalg.norm(x / s))  # about 4e169 (a scaled norm): c * c overflows
    with np.errstate(over="ignore", invalid="ignore"):
        assert not np.isfinite((c * c) * (x @ x))
    xs = c * x
    assert np.isfinite(xs @ xs) and abs(xs @ xs - 1.0) < 1e-15
