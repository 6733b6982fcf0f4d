"""GPU parity of tsqr_r_batched (varlen batch, one persistent launch) against the CPU oracle,
problem by problem, through the C ABI.  FP64: every R_i within c(m_i) kappa u ||R_i||_F of the
oracle's and a Gram residual <= 1e-13; mixed FP32: Gram residual <= 2e-6 (tolerances of the
single-matrix tests)."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu
U = 2.0 ** -53
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def T():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1002_4250_gb300 as T
    return T


def _c(m):
    return max(50.0, 2.0 * np.sqrt(max(m, 1)))


def _run(T, buf_dev, ms, ns, offs, dtype, prec):
    import torch
    es = buf_dev.element_size()
    base = buf_dev.data_ptr()
    ptrs = [base + es * offs[i] for i in range(len(ms))]
    roff = [0]
    for n in ns:
        roff.append(roff[-1] + n * n)
    Rp = torch.full((roff[-1],), float("nan"), dtype=torch.float64, device="cuda")
    T.tsqr_r_batched(ptrs, ms, ns, roff, Rp, dtype=dtype, prec=prec)
    torch.cuda.synchronize()
    return Rp.cpu().numpy(), roff


def _problem(buf_cpu, offs, ms, ns, i):
    m, n = ms[i], ns[i]
    return np.asarray(buf_cpu[offs[i]:offs[i] + m * n], dtype=np.float64).reshape(n, m).T


def _edge_batch():
    import torch
    g = torch.Generator().manual_seed(7)
    ms = [0, 1, 2, 5, 7, 63, 64, 65, 300, 1000, 4097, 12345, 3, 129, 50000, 256]
    ns = [4, 1, 3, 8, 7, 16, 64, 64, 32, 128, 5, 24, 12, 128, 64, 16]
    offs = [0]
    for m, n in zip(ms, ns):
        offs.append(offs[-1] + m * n)
    buf = torch.randn(offs[-1], generator=g, dtype=torch.float64)
    return buf, ms, ns, offs


def test_batched_fp64_edge_cases(oracle, T):
    buf, ms, ns, offs = _edge_batch()
    R, roff = _run(T, buf.cuda(), ms, ns, offs, T.F64, T.PREC_F64)
    for i, (m, n) in enumerate(zip(ms, ns)):
        Ri = R[roff[i]:roff[i + 1]].reshape(n, n).T
        A = _problem(buf.numpy(), offs, ms, ns, i)
        Ro = oracle.householder_r(A)
        assert np.all(np.isfinite(Ri)) and np.all(np.tril(Ri, -1) == 0), i
        if m == 0:
            assert np.all(Ri == 0)
            continue
        assert oracle.gram_residual(A, Ri) <= 1e-13, i
        if m >= n:
            kap = oracle.kappa_from_r(Ro)
            np.testing.assert_allclose(Ri, Ro, rtol=0, atol=_c(m) * kap * U * np.linalg.norm(Ro))


def test_batched_matches_single_calls(T):
    import torch
    buf, ms, ns, offs = _edge_batch()
    bd = buf.cuda()
    R, roff = _run(T, bd, ms, ns, offs, T.F64, T.PREC_F64)
    for i, (m, n) in enumerate(zip(ms, ns)):
        if m == 0:
            continue
        A = bd[offs[i]:offs[i] + m * n].view(n, m).T
        Rs = T.tsqr_r(A).cpu().numpy()
        Ri = R[roff[i]:roff[i + 1]].reshape(n, n).T
        s = np.linalg.svd(Rs, compute_uv=False)
        kap = s[0] / s[-1] if s[-1] > 0 else 1e16
        if m >= n and kap < 1e12:
            np.testing.assert_allclose(Ri, Rs, rtol=0, atol=_c(m) * kap * U * np.linalg.norm(Rs))


@pytest.mark.parametrize("dtype", ["float32", "bfloat16"])
def test_batched_mixed(oracle, T, dtype):
    import torch
    buf, ms, ns, offs = workloads.varlen_batch(48, 512, 40000, seed=1)
    low = buf.to(getattr(torch, dtype))
    code = T.F32 if dtype == "float32" else T.BF16
    R, roff = _run(T, low.cuda(), ms, ns, offs, code, T.PREC_MIXED)
    wide = low.to(torch.float64).numpy()
    for i, (m, n) in enumerate(zip(ms, ns)):
        Ri = R[roff[i]:roff[i + 1]].reshape(n, n).T
        A = _problem(wide, offs, ms, ns, i)
        assert oracle.gram_residual(A, Ri) <= 2e-6, i


def test_batched_varlen_distribution(oracle, T):
    """The varlen workload's distribution (m log-uniform in [512, 262144], n in {8,16,32,64})
    with 256 problems; every problem's Gram residual, and the oracle's R on a sample."""
    buf, ms, ns, offs = workloads.varlen_batch(256, 512, 262144, seed=0)
    R, roff = _run(T, buf.cuda(), ms, ns, offs, T.F64, T.PREC_F64)
    rng = np.random.default_rng(0)
    sample = set(rng.choice(len(ms), size=12, replace=False).tolist())
    bn = buf.numpy()
    for i, (m, n) in enumerate(zip(ms, ns)):
        Ri = R[roff[i]:roff[i + 1]].reshape(n, n).T
        A = _problem(bn, offs, ms, ns, i)
        assert oracle.gram_residual(A, Ri, nthreads=16) <= 1e-13, i
        if i in sample:
            Ro = oracle.householder_r(A, nthreads=16)
            kap = oracle.kappa_from_r(Ro)
            np.testing.assert_allclose(Ri, Ro, rtol=0, atol=_c(m) * kap * U * np.linalg.norm(Ro))


def test_batched_bit_reproducible_and_graph_capture(T):
    import torch
    buf, ms, ns, offs = workloads.varlen_batch(64, 512, 20000, seed=2)
    bd = buf.cuda()
    R1, roff = _run(T, bd, ms, ns, offs, T.F64, T.PREC_F64)
    R2, _ = _run(T, bd, ms, ns, offs, T.F64, T.PREC_F64)
    assert np.array_equal(R1, R2)
    # capture the same call (descriptors already resident) in a CUDA graph and replay it
    es = bd.element_size()
    ptrs = [bd.data_ptr() + es * o for o in offs[:-1]]
    Rg = torch.full((roff[-1],), float("nan"), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        T.tsqr_r_batched(ptrs, ms, ns, roff, Rg)   # warm-up on the capture stream
    torch.cuda.synchronize()
    Rg.fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        T.tsqr_r_batched(ptrs, ms, ns, roff, Rg)
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(Rg.cpu().numpy(), R1)


def test_batched_argument_errors(T):
    import ctypes
    import torch
    Rp = torch.zeros(100, dtype=torch.float64, device="cuda")
    A = torch.zeros(1000, dtype=torch.float64, device="cuda")
    with pytest.raises(T.TsqrError) as e:
        T.tsqr_r_batched([A.data_ptr()], [100], [8], [0, 10], Rp)   # room for 10 < 64 entries
    assert e.value.status == T.ERR_INVALID_ARG
    with pytest.raises(T.TsqrError) as e:
        T.tsqr_r_batched([A.data_ptr()], [5], [129], [0, 129 * 129], Rp)
    assert e.value.status == T.ERR_UNSUPPORTED
    with pytest.raises(T.TsqrError) as e:
        T.tsqr_r_batched([A.data_ptr()], [5], [4], [0, 16], Rp, dtype=T.F32, prec=T.PREC_F64)
    assert e.value.status == T.ERR_INVALID_ARG


# ---- batch knobs (tsqr_r_batched_ex) and batch autotuning (tsqr_autotune_batched)

def _ptrs_roff(bd, ms, ns, offs):
    es = bd.element_size()
    ptrs = [bd.data_ptr() + es * o for o in offs[:-1]]
    roff = [0]
    for n in ns:
        roff.append(roff[-1] + n * n)
    return ptrs, roff


def _check_all(oracle, bn, ms, ns, offs, R, roff, tol):
    for i, (m, n) in enumerate(zip(ms, ns)):
        Ri = R[roff[i]:roff[i + 1]].reshape(n, n).T
        assert np.all(np.tril(Ri, -1) == 0) and np.all(np.diag(Ri) >= 0), i
        assert oracle.gram_residual(_problem(bn, offs, ms, ns, i), Ri, nthreads=16) <= tol, i


@pytest.mark.parametrize("knobs", [dict(warps=4, ctas_per_sm=1), dict(warps=8, ctas_per_sm=1),
                                   dict(warps=12, ctas_per_sm=1, leaves_per_cta=2),
                                   dict(leaves_per_cta=16, arity=(2, 2, 2, 2)),
                                   dict(warps=4, ctas_per_sm=2, arity=(8, 4, 3, 2))])
@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_batched_knobs(oracle, T, knobs, prec):
    """Every knob setting gives a correct R for every problem of a varlen batch, and the knobs
    the call reports are the ones asked for."""
    import torch
    buf, ms, ns, offs = workloads.varlen_batch(96, 512, 60000, seed=5)
    if prec == "f64":
        bd, code, p, tol = buf.cuda(), T.F64, T.PREC_F64, 1e-13
    else:
        bd, code, p, tol = buf.to(torch.float32).cuda(), T.F32, T.PREC_MIXED, 2e-6
        knobs = dict(knobs, leaf="fold")  # warps and chunk height are the fold leaf's knobs
    ptrs, roff = _ptrs_roff(bd, ms, ns, offs)
    Rp = torch.full((roff[-1],), float("nan"), dtype=torch.float64, device="cuda")
    plan = T.make_batch_plan(**knobs)
    T.tsqr_r_batched(ptrs, ms, ns, roff, Rp, dtype=code, prec=p, plan=plan)
    used = T.last_batch_plan()
    for k in ("warps", "ctas_per_sm", "leaves_per_cta"):
        if knobs.get(k):
            assert getattr(used, k) == knobs[k], k
    assert tuple(used.arity) == tuple(knobs.get("arity", (0, 0, 0, 0)))
    torch.cuda.synchronize()
    _check_all(oracle, bd.to(torch.float64).cpu().numpy(), ms, ns, offs, Rp.cpu().numpy(), roff,
               tol)


def test_batched_knob_errors(T):
    import torch
    buf, ms, ns, offs = workloads.varlen_batch(4, 512, 2000, seed=6)
    bd = buf.cuda()
    ptrs, roff = _ptrs_roff(bd, ms, ns, offs)
    Rp = torch.zeros(roff[-1], dtype=torch.float64, device="cuda")
    for bad in (dict(warps=13), dict(ctas_per_sm=3), dict(leaves_per_cta=65),
                dict(arity=(1, 0, 0, 0)), dict(arity=(0, 0, 9, 0))):
        with pytest.raises(T.TsqrError) as e:
            T.tsqr_r_batched(ptrs, ms, ns, roff, Rp, plan=T.make_batch_plan(**bad))
        assert e.value.status == T.ERR_INVALID_ARG, bad


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_batched_autotune_bucket(oracle, T, prec):
    """The tuned knobs are cached for the batch's shape bucket: an AUTO call on the same batch,
    and on another batch of the same bucket, runs with them, is bit-reproducible, and equals
    the explicit call with the tuned knobs; after a reset AUTO goes back to the built-in
    rules."""
    import torch
    buf, ms, ns, offs = workloads.varlen_batch(128, 512, 60000, seed=8)
    if prec == "f64":
        bd, code, p, tol = buf.cuda(), T.F64, T.PREC_F64, 1e-13
    else:
        bd, code, p, tol = buf.to(torch.float32).cuda(), T.F32, T.PREC_MIXED, 2e-6
    ptrs, roff = _ptrs_roff(bd, ms, ns, offs)
    Rp = torch.zeros(roff[-1], dtype=torch.float64, device="cuda")
    T.tsqr_autotune_reset()
    try:
        T.tsqr_r_batched(ptrs, ms, ns, roff, Rp, dtype=code, prec=p)
        builtin = T.last_batch_plan().as_tuple()
        best = T.tsqr_autotune_batched(ptrs, ms, ns, roff, Rp, dtype=code, prec=p)
        R1 = Rp.clone()
        T.tsqr_r_batched(ptrs, ms, ns, roff, R1, dtype=code, prec=p)
        used = T.last_batch_plan()
        if best.warps:
            assert used.warps == best.warps
        if best.ctas_per_sm:
            assert used.ctas_per_sm == best.ctas_per_sm
        if best.leaves_per_cta:
            assert used.leaves_per_cta == best.leaves_per_cta
        assert tuple(used.arity) == tuple(best.arity)
        R2 = torch.zeros_like(R1)
        T.tsqr_r_batched(ptrs, ms, ns, roff, R2, dtype=code, prec=p)
        R3 = torch.zeros_like(R1)
        T.tsqr_r_batched(ptrs, ms, ns, roff, R3, dtype=code, prec=p, plan=best)
        torch.cuda.synchronize()
        assert torch.equal(R1, R2) and torch.equal(R1, R3)
        _check_all(oracle, bd.to(torch.float64).cpu().numpy(), ms, ns, offs, R1.cpu().numpy(),
                   roff, tol)
        # the same shapes at another address are in the same bucket
        bd2 = bd.clone()
        ptrs2, _ = _ptrs_roff(bd2, ms, ns, offs)
        T.tsqr_r_batched(ptrs2, ms, ns, roff, R2, dtype=code, prec=p)
        assert T.last_batch_plan().as_tuple() == used.as_tuple()
        torch.cuda.synchronize()
        assert torch.equal(R1, R2)
    finally:
        T.tsqr_autotune_reset()
    T.tsqr_r_batched(ptrs, ms, ns, roff, Rp, dtype=code, prec=p)
    assert T.last_batch_plan().as_tuple() == builtin


# ---- the blocked tensor-core leaf in the mixed batch

def _odd_mixed_batch(dtype, widths=(1, 3, 8, 16, 17, 33, 48, 64)):
    import torch
    g = torch.Generator().manual_seed(9)
    ms = [0, 1, 5, 100, 511, 512, 513, 3000, 40000, 257, 1024, 70001]
    ns = [widths[i % len(widths)] for i in range(len(ms))]
    offs = [0]
    for m, n in zip(ms, ns):
        offs.append(offs[-1] + m * n)
    buf = torch.randn(offs[-1], generator=g, dtype=torch.float64).to(dtype)
    return buf, ms, ns, offs


@pytest.mark.parametrize("dtype", ["float32", "bfloat16"])
@pytest.mark.parametrize("leaf", ["auto", "fold", "panels"])
def test_batched_mixed_leaves(oracle, T, dtype, leaf):
    """The mixed batch on either leaf (the blocked one is AUTO up to 112 columns): every
    problem's R upper triangular with diag >= 0 and R^T R = A^T A within 2e-6, including
    m = 0, m < n, one row, one column and ragged chunks."""
    import torch
    buf, ms, ns, offs = _odd_mixed_batch(getattr(torch, dtype))
    code = T.F32 if dtype == "float32" else T.BF16
    bd = buf.cuda()
    ptrs, roff = _ptrs_roff(bd, ms, ns, offs)
    Rp = torch.full((roff[-1],), float("nan"), dtype=torch.float64, device="cuda")
    T.tsqr_r_batched(ptrs, ms, ns, roff, Rp, dtype=code, prec=T.PREC_MIXED,
                     plan=T.make_batch_plan(leaf=leaf))
    assert T.last_batch_plan().leaf == (T.LEAF_FOLD if leaf == "fold" else T.LEAF_PANELS)
    torch.cuda.synchronize()
    assert T.tsqr_get_device_status() == T.SUCCESS
    _check_all(oracle, buf.to(torch.float64).numpy(), ms, ns, offs, Rp.cpu().numpy(), roff, 2e-6)


def test_batched_panels_reproducible_and_graph(T):
    """The blocked-leaf batch is bit-reproducible, and a captured call replays it bit for bit."""
    import torch
    buf, ms, ns, offs = workloads.varlen_batch(64, 512, 30000, seed=3, dtype=torch.float32)
    bd = buf.cuda()
    ptrs, roff = _ptrs_roff(bd, ms, ns, offs)
    plan = T.make_batch_plan(leaf="panels")
    R1 = torch.zeros(roff[-1], dtype=torch.float64, device="cuda")
    R2 = torch.zeros_like(R1)
    T.tsqr_r_batched(ptrs, ms, ns, roff, R1, dtype=T.F32, prec=T.PREC_MIXED, plan=plan)
    T.tsqr_r_batched(ptrs, ms, ns, roff, R2, dtype=T.F32, prec=T.PREC_MIXED, plan=plan)
    torch.cuda.synchronize()
    assert torch.equal(R1, R2)
    s = torch.cuda.Stream()
    Rg = torch.full_like(R1, float("nan"))
    with torch.cuda.stream(s):
        T.tsqr_r_batched(ptrs, ms, ns, roff, Rg, dtype=T.F32, prec=T.PREC_MIXED, plan=plan,
                         stream=s)
    torch.cuda.synchronize()
    Rg.fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        T.tsqr_r_batched(ptrs, ms, ns, roff, Rg, dtype=T.F32, prec=T.PREC_MIXED, plan=plan,
                         stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(Rg, R1)


def test_batched_panels_refused(T):
    """The blocked leaf is mixed precision up to 112 columns: an FP64 batch or a wider problem
    asks for it in vain."""
    import torch
    A = torch.zeros(100 * 80, dtype=torch.float64, device="cuda")
    Rp = torch.zeros(80 * 80, dtype=torch.float64, device="cuda")
    with pytest.raises(T.TsqrError) as e:
        T.tsqr_r_batched([A.data_ptr()], [100], [8], [0, 64], Rp,
                         plan=T.make_batch_plan(leaf="panels"))
    assert e.value.status == T.ERR_UNSUPPORTED
    A32 = torch.zeros(200 * 120, dtype=torch.float32, device="cuda")
    Rw = torch.zeros(120 * 120, dtype=torch.float64, device="cuda")
    with pytest.raises(T.TsqrError) as e:
        T.tsqr_r_batched([A32.data_ptr()], [200], [120], [0, 14400], Rw, dtype=T.F32,
                         prec=T.PREC_MIXED, plan=T.make_batch_plan(leaf="panels"))
    assert e.value.status == T.ERR_UNSUPPORTED


def test_batched_mixed_wide_problem_takes_the_fold(oracle, T):
    """A mixed batch with a problem wider than 112 columns runs on the fold leaf as a whole
    (AUTO), and every problem's R is right."""
    import torch
    buf, ms, ns, offs = _odd_mixed_batch(torch.float32, widths=(8, 16, 120, 33, 64))
    bd = buf.cuda()
    ptrs, roff = _ptrs_roff(bd, ms, ns, offs)
    Rp = torch.full((roff[-1],), float("nan"), dtype=torch.float64, device="cuda")
    T.tsqr_r_batched(ptrs, ms, ns, roff, Rp, dtype=T.F32, prec=T.PREC_MIXED)
    assert T.last_batch_plan().leaf == T.LEAF_FOLD
    torch.cuda.synchronize()
    _check_all(oracle, buf.to(torch.float64).numpy(), ms, ns, offs, Rp.cpu().numpy(), roff, 2e-6)


@pytest.mark.parametrize("leaf", ["auto", "panels"])
def test_batched_panels_wide(oracle, T, leaf):
    """A mixed batch up to 112 columns on the blocked leaf, AUTO or asked for."""
    import torch
    buf, ms, ns, offs = _odd_mixed_batch(torch.float32, widths=(8, 100, 65, 112, 33))
    bd = buf.cuda()
    ptrs, roff = _ptrs_roff(bd, ms, ns, offs)
    Rp = torch.full((roff[-1],), float("nan"), dtype=torch.float64, device="cuda")
    T.tsqr_r_batched(ptrs, ms, ns, roff, Rp, dtype=T.F32, prec=T.PREC_MIXED,
                     plan=T.make_batch_plan(leaf=leaf))
    assert T.last_batch_plan().leaf == T.LEAF_PANELS
    torch.cuda.synchronize()
    _check_all(oracle, buf.to(torch.float64).numpy(), ms, ns, offs, Rp.cpu().numpy(), roff, 2e-6)
