"""The reflector's scalar routines (third-order steps for 1/sqrt(t) and 1/x seeded by FP32
hardware estimates) against CUDA's own FP64 rsqrt and reciprocal, over the whole exponent
range: within 2 ulp."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_newton_scalars_match_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1002_4250_gb300 as T
    lib = T.capi
    fn = lib.tsqr_internal_scalar_selftest
    fn.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    g = torch.Generator().manual_seed(0)
    n = 1 << 20
    mant = 1.0 + torch.rand(n, generator=g, dtype=torch.float64)
    expo = torch.randint(-1000, 1000, (n,), generator=g).to(torch.float64)
    sign = torch.where(torch.rand(n, generator=g) < 0.5, -1.0, 1.0).to(torch.float64)
    x = (sign * mant * torch.pow(2.0, expo)).cuda()
    x[:4] = torch.tensor([1.0, 4.0, 2.0 ** -1022, 2.0 ** 1023], dtype=torch.float64)
    rs = torch.empty_like(x)
    rc = torch.empty_like(x)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert fn(n, x.data_ptr(), rs.data_ptr(), rc.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    ref_rs = torch.rsqrt(x.abs())
    ref_rc = torch.reciprocal(x)
    ulp = lambda v: torch.abs(torch.nextafter(v, torch.full_like(v, float("inf"))) - v)
    assert torch.all(torch.abs(rs - ref_rs) <= 2 * ulp(ref_rs))
    assert torch.all(torch.abs(rc - ref_rc) <= 2 * ulp(ref_rc))
    assert rs[1].item() == 0.5 and rc[1].item() == 0.25
