"""CPU checks (numpy) of the arithmetic the blocked mixed-precision leaf rests on.

1. The compact WY form of a panel of reflectors H_J = I - tau_J v_J v_J^T, v_J = [e_J; c_J x_J]
   (x_J the unscaled tail, tau_J = 2 / v_J^T v_J): H_0 H_1 ... H_{p-1} = I - V S V^T with
   S^-1 = diag(1 / tau) + strict_upper(G), G(i, J) = c_i c_J x_i . x_J (Joffrain, Low,
   Quintana-Orti, van de Geijn, "Accumulating Householder transformations, revisited"), S
   computed column by column as the kernel does (S(J, J) = tau_J, S(i, J) = -tau_i
   sum_{l = i+1..J} G(i, l) S(l, J)), identity reflectors (tau = 0) included; and the update of
   the columns right of the panel, W = R(P, T) + diag(c) X^T C, Y = S^T W, R(P, T) -= Y,
   C -= X diag(c) Y, against the reflectors applied one by one.
2. The TF32 parts (11 significant bits, round to nearest with ties away, as cvt.rna.tf32.f32):
   a value rounded to 22 bits is exactly two parts, an FP32 value exactly three; and the
   kernels' split of an FP32 value by truncation (its top 11 significant bits, the next 11, the
   last 2, each difference taken in FP32) is exact too.
"""
import numpy as np


def _reflectors(rng, h, p, identity=()):
    X = rng.standard_normal((h, p))
    c = rng.uniform(0.2, 1.5, p) * np.where(rng.random(p) < 0.5, -1.0, 1.0)
    tau = 2.0 / (1.0 + c ** 2 * np.sum(X ** 2, axis=0))
    for j in identity:
        tau[j] = 0.0
        c[j] = 0.0
    return X, c, tau


def _S_by_columns(tau, G):
    p = len(tau)
    S = np.zeros((p, p))
    for J in range(p):
        S[J, J] = tau[J]
        for i in range(J - 1, -1, -1):
            S[i, J] = -tau[i] * sum(G[i, l] * S[l, J] for l in range(i + 1, J + 1))
    return S


def test_compact_wy_product():
    rng = np.random.default_rng(1)
    for identity in ((), (0,), (3, 7), (15,)):
        h, p = 40, 16
        X, c, tau = _reflectors(rng, h, p, identity)
        V = np.vstack([np.eye(p), X * c])
        H = np.eye(p + h)
        for J in range(p):
            H = H @ (np.eye(p + h) - tau[J] * np.outer(V[:, J], V[:, J]))
        G = np.triu((X * c).T @ (X * c), 1)
        S = _S_by_columns(tau, G)
        np.testing.assert_allclose(np.eye(p + h) - V @ S @ V.T, H, atol=1e-13)
        if not identity:
            Sinv = np.diag(1.0 / tau) + G
            np.testing.assert_allclose(S, np.linalg.inv(Sinv), atol=1e-13)


def test_trailing_update_matches_one_by_one():
    rng = np.random.default_rng(2)
    h, p, nt = 64, 16, 24
    X, c, tau = _reflectors(rng, h, p, identity=(5,))
    RP = rng.standard_normal((p, nt))
    C = rng.standard_normal((h, nt))
    # one by one: [R(J, :); C] <- H_J [R(J, :); C], reflector J touching row J of the panel
    R1, C1 = RP.copy(), C.copy()
    for J in range(p):
        w = R1[J] + c[J] * (X[:, J] @ C1)
        R1[J] -= tau[J] * w
        C1 -= np.outer(tau[J] * c[J] * X[:, J], w)
    G = np.triu((X * c).T @ (X * c), 1)
    S = _S_by_columns(tau, G)
    W = RP + c[:, None] * (X.T @ C)
    Y = S.T @ W
    np.testing.assert_allclose(RP - Y, R1, atol=1e-12)
    np.testing.assert_allclose(C - X @ (c[:, None] * Y), C1, atol=1e-12)


def _tf32(x):
    """cvt.rna.tf32.f32: 10 explicit fraction bits, round to nearest, ties away from zero."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    mag = (b & 0x7FFFFFFF) + 0x1000
    out = (b & 0x80000000) | (mag & 0x7FFFE000)
    return out.astype(np.uint32).view(np.float32)


def test_tf32_parts_are_exact():
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(200000) * np.exp(rng.uniform(-30, 30, 200000))).astype(np.float32)
    h = _tf32(x)
    r22 = (h + _tf32(x - h)).astype(np.float32)
    # round22 keeps 22 bits: two parts hold it exactly, and the parts are TF32 values
    h2 = _tf32(r22)
    l2 = _tf32(r22 - h2)
    assert np.all(h2.astype(np.float64) + l2.astype(np.float64) == r22.astype(np.float64))
    assert np.all(_tf32(l2) == l2)
    assert np.all(np.abs(r22.astype(np.float64) - x) <= 2.0 ** -22 * np.abs(x.astype(np.float64)))
    # any FP32 value is exactly three TF32 parts
    m = _tf32(x - h)
    l3 = _tf32((x - h) - m)
    assert np.all(h.astype(np.float64) + m.astype(np.float64) + l3.astype(np.float64)
                  == x.astype(np.float64))
    # products of TF32 values are exact in FP32
    a, b = _tf32(x[:1000]), _tf32(x[1000:2000])
    prod32 = (a * b).astype(np.float64)
    exact = a.astype(np.float64) * b.astype(np.float64)
    ok = np.isfinite(prod32) & (np.abs(exact) > 1e-30) & (np.abs(exact) < 1e30)
    assert np.all(prod32[ok] == exact[ok])


def _tf32_trunc(x):
    """The top 11 significant bits: the low 13 fraction bits cleared."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32)
    return (b & np.uint32(0xFFFFE000)).view(np.float32)


def test_truncated_tf32_parts_are_exact():
    """x = h + m + l with h = trunc(x), m = trunc(x - h), l = (x - h) - m in FP32: both
    differences are exact, every part is a TF32 value and l has at most 2 significant bits;
    the parts' magnitudes fall by 2^-11 and 2^-22 (at most) as with rounding."""
    rng = np.random.default_rng(5)
    x = (rng.standard_normal(200000) * np.exp(rng.uniform(-30, 30, 200000))).astype(np.float32)
    x[:4] = np.array([0.0, -0.0, 1.0, -3.0], dtype=np.float32)
    h = _tf32_trunc(x)
    r = (x - h).astype(np.float32)
    m = _tf32_trunc(r)
    l = (r - m).astype(np.float32)
    x64 = x.astype(np.float64)
    assert np.all(r.astype(np.float64) == x64 - h.astype(np.float64))
    assert np.all(h.astype(np.float64) + m.astype(np.float64) + l.astype(np.float64) == x64)
    for part in (h, m, l):
        assert np.all(_tf32_trunc(part) == part)
    assert np.all((l.view(np.uint32) & np.uint32(0x003FFFFF)) == 0)  # <= 2 significant bits
    assert np.all(np.abs(m.astype(np.float64)) <= 2.0 ** -10 * np.abs(x64))
    assert np.all(np.abs(l.astype(np.float64)) <= 2.0 ** -21 * np.abs(x64))


def test_forward_recurrence_equals_inverse_form():
    """dlarft's forward recurrence, as the kernel forms S column by column (S(J, J) = tau_J,
    S(i, J) = -tau_J sum_{l = i..J-1} S(i, l) G(l, J)), gives the same S as the back substitution
    and as the inverse of diag(1/tau) + strict_upper(G); identity reflectors included."""
    rng = np.random.default_rng(4)
    for identity in ((), (2,), (0, 9)):
        X, c, tau = _reflectors(rng, 50, 16, identity)
        G = np.triu((X * c).T @ (X * c), 1)
        S = np.zeros((16, 16))
        for J in range(16):
            S[J, J] = tau[J]
            for i in range(J):
                S[i, J] = -tau[J] * sum(S[i, l] * G[l, J] for l in range(i, J))
        np.testing.assert_allclose(S, _S_by_columns(tau, G), atol=1e-13)
        if not identity:
            np.testing.assert_allclose(S, np.linalg.inv(np.diag(1.0 / tau) + G), atol=1e-13)
