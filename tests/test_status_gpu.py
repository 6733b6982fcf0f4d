"""Fault-free failure detection on the GPU.  The leaf kernels wait for their tensor-core
commits and TMA loads on mbarriers, each wait bounded by a poll count; a wait that gives up
sets the timeout bit of the stream's device status word, which tsqr_get_device_status reports
as TSQR_ERR_TIMEOUT (and clears).  The test hook tsqr_internal_wait_selftest runs that wait in
one CTA on an mbarrier nothing arrives at, so that it runs out (a few dozen polls: no fault,
trap or hang), and as a control on one its own arrival completes."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1002_4250_gb300 as T
    fn = T.capi.tsqr_internal_wait_selftest
    fn.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return T


def _wait(T, limit, arrive):
    import torch
    res = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = T.capi.tsqr_internal_wait_selftest(limit, arrive, ctypes.c_void_p(res.data_ptr()), stream)
    torch.cuda.synchronize()
    return st, int(res.item())


def test_completed_wait_reports_nothing(T):
    T.tsqr_get_device_status()  # clear
    st, ok = _wait(T, 1000, 1)
    assert st == T.SUCCESS and ok == 1
    assert T.tsqr_get_device_status() == T.SUCCESS


def test_wait_that_runs_out_reports_timeout_and_the_context_stays_usable(T):
    import torch
    import workloads
    T.tsqr_get_device_status()
    st, ok = _wait(T, 64, 0)
    assert st == T.SUCCESS and ok == 0
    assert T.tsqr_get_device_status() == T.ERR_TIMEOUT
    assert T.tsqr_get_device_status() == T.SUCCESS  # read once, then cleared
    # the context is intact: a factorization right after is right
    At = workloads.gaussian(20000, 8, seed=2)
    R = T.tsqr_r(At.cuda().T)
    torch.cuda.synchronize()
    assert T.tsqr_get_device_status() == T.SUCCESS
    Rt = torch.linalg.qr(At.T, mode="r")[1]
    Rt = Rt * torch.sign(torch.diagonal(Rt))[:, None]
    assert torch.allclose(R.cpu(), Rt, rtol=0, atol=1e-10 * float(Rt.abs().max()))


def test_wait_hook_argument_checks(T):
    st, _ = _wait(T, 0, 0)
    assert st == T.ERR_INVALID_ARG
    st, _ = _wait(T, 1 << 21, 0)
    assert st == T.ERR_INVALID_ARG
