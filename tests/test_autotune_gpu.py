"""tsqr_autotune: it returns a plan that AUTO calls of the same (n, leaf precision,
floor(log2 m)) bucket then use, the tuned AUTO result keeps parity with the oracle (FP64:
every entry within c(m) kappa u ||R||_F, Gram residual <= 1e-13; mixed: Gram residual <= 2e-6),
other buckets are untouched, and tsqr_autotune_reset restores the built-in rules."""
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
    T.tsqr_autotune_reset()
    yield T
    T.tsqr_autotune_reset()  # later test files see the built-in AUTO plans


def _fields(p):
    return (p.tile_rows, p.ctas, p.warps)


def test_autotune_fp64(oracle, T):
    import torch
    m, n = 1 << 20, 32
    At = workloads.gaussian(m, n, seed=21)
    Ad = At.cuda().T
    default = T.tsqr_resolve_plan(m, n)
    other = T.tsqr_resolve_plan(m, 16)
    best = T.tsqr_autotune(Ad)
    assert best.tree == T.TREE_HYBRID and best.warps in (4, 8, 12) and best.tile_rows >= n
    assert _fields(T.tsqr_resolve_plan(m, n)) == _fields(best)
    assert _fields(T.tsqr_resolve_plan(m + 12345, n)) == _fields(best)  # same log2 bucket
    assert _fields(T.tsqr_resolve_plan(m, 16)) == _fields(other)        # other n untouched
    if best.arity:  # the arity stage picked a tree arity: AUTO resolves to it
        assert T.tsqr_resolve_plan(m, n).arity == best.arity
    Rt = T.tsqr_r(Ad)
    assert torch.equal(Rt, T.tsqr_r_ex(Ad, plan=best))  # AUTO returns the tuned plan's bytes
    R = Rt.cpu().numpy()
    A = oracle.from_torch_colmajor(At)
    Ro = oracle.householder_r(A, nthreads=16)
    kap = oracle.kappa_from_r(Ro)
    np.testing.assert_allclose(R, Ro, rtol=0,
                               atol=max(50.0, 2.0 * np.sqrt(m)) * kap * U * np.linalg.norm(Ro))
    assert oracle.gram_residual(A, R, nthreads=16) <= 1e-13
    T.tsqr_autotune_reset()
    assert _fields(T.tsqr_resolve_plan(m, n)) == _fields(default)


def test_autotune_mixed(oracle, T):
    import torch
    m, n = 300000, 64
    At = workloads.gaussian(m, n, seed=22, dtype=torch.float32)
    best = T.tsqr_autotune(At.cuda().T)
    assert best.warps in (4, 8)
    p = T.tsqr_resolve_plan(m, n, dtype=T.F32, prec=T.PREC_MIXED)
    assert _fields(p) == _fields(best)
    R = T.tsqr_r_ex(At.cuda().T).cpu().numpy()
    A = oracle.from_torch_colmajor(At.to(torch.float64))
    assert oracle.gram_residual(A, R, nthreads=16) <= 2e-6
    T.tsqr_autotune_reset()


def test_autotune_wide_considers_panels(oracle, T):
    """From n = 48 on the FP64 candidates include panels of 16 and 32 columns; whatever wins,
    later AUTO calls of the bucket return its bytes, with parity; tsqr_qr keeps one reduction."""
    import torch
    m, n = 1 << 19, 96
    At = workloads.gaussian(m, n, seed=23)
    Ad = At.cuda().T
    best = T.tsqr_autotune(Ad)
    R = T.tsqr_r(Ad)
    assert torch.equal(R, T.tsqr_r_ex(Ad, plan=best))
    A = oracle.from_torch_colmajor(At)
    assert oracle.gram_residual(A, R.cpu().numpy(), nthreads=16) <= 1e-13
    T.tsqr_qr(Ad)
    assert T.last_plan().tree == T.TREE_HYBRID
    T.tsqr_autotune_reset()

