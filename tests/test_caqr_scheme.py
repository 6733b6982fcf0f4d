"""The panel-and-update scheme of tsqr_caqr_r (Section 5), modelled on the CPU with numpy's
Householder QR as the local step: it must give the R of the whole matrix, and each panel on L
leaves must add exactly (L - 1) panel rows to the next panel's matrix.

The model follows the GPU's data flow, not its arithmetic: every leaf folds its rows under a
zero triangle of `w` rows (so its orthogonal transformation runs over its rows plus w virtual
ones), the leaves' top blocks are combined along a k-ary tree (the first child on top), and every
row a transformation leaves below its top block stays in the next panel's matrix."""
import numpy as np
import pytest


def _q_full(M):
    """Full orthogonal Q of M (rows x cols, rows >= cols) with M = Q [R; 0]."""
    Q, _ = np.linalg.qr(M, mode="complete")
    return Q


def _panel_step(C, w, leaves, arity):
    """One panel: R's block row (w x ncols) and the next matrix (rows left behind)."""
    m, ncols = C.shape
    bounds = np.linspace(0, m, leaves + 1).astype(int)
    tops, left = [], []
    for l in range(leaves):
        rows = C[bounds[l]:bounds[l + 1]]
        aug = np.vstack([np.zeros((w, ncols)), rows])  # the zero triangle, then the leaf's rows
        T = _q_full(aug[:, :w]).T @ aug
        tops.append(T[:w])
        left.append(T[w:])  # as many rows as the leaf had
    level = tops
    while len(level) > 1:
        nxt = []
        for p in range(0, len(level), arity):
            kids = level[p:p + arity]
            if len(kids) == 1:
                nxt.append(kids[0])
                continue
            S = np.vstack(kids)
            T = _q_full(S[:, :w]).T @ S
            nxt.append(T[:w])
            left.append(T[w:])  # every child's block but the first's
        level = nxt
    return level[0], np.vstack(left)


def _caqr_r(A, w, leaves, arity):
    m, n = A.shape
    R = np.zeros((n, n))
    C = A.copy()
    growth = []
    for j0 in range(0, n, w):
        wj = min(w, n - j0)
        L = min(leaves, C.shape[0])
        top, rest = _panel_step(C, wj, L, arity)
        R[j0:j0 + wj, j0:] = top
        growth.append(rest.shape[0] - C.shape[0])
        assert growth[-1] == (L - 1) * wj
        C = rest[:, wj:]
    # the sign convention: diag(R) >= 0 by row signs
    return np.sign(np.where(np.diag(R) == 0, 1.0, np.diag(R)))[:, None] * R, growth


@pytest.mark.parametrize("m,n,w,leaves,arity", [(400, 40, 8, 5, 2), (300, 37, 16, 7, 3),
                                                (129, 20, 4, 9, 8), (64, 64, 16, 3, 2)])
def test_panels_give_the_r_of_the_whole_matrix(m, n, w, leaves, arity):
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n))
    R, growth = _caqr_r(A, w, leaves, arity)
    Rl = np.linalg.qr(A, mode="r")
    Rl = np.sign(np.diag(Rl))[:, None] * Rl
    assert np.allclose(np.tril(R, -1), 0.0)
    np.testing.assert_allclose(R, Rl, rtol=0, atol=1e-11 * np.linalg.norm(Rl))
    assert all(g >= 0 for g in growth)
