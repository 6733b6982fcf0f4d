"""The tensor-core building blocks on the GPU: tcgen05 operand layouts (K-major A unswizzled or
with the 128-byte swizzle, or A in tensor memory as the mixed-precision leaf's update uses it,
times a K-major unswizzled B; D read back from tensor memory), checked exactly against numpy on
integer inputs, and the peak microbenchmarks' sanity."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1002_4250_gb300 as T
    return T


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("N", [16, 48, 112, 256])
def test_tcgen05_layouts(T, N, variant):
    import torch
    D = torch.full((128, N), float("nan"), dtype=torch.float32, device="cuda")
    assert T.capi.tsqr_internal_tc_layout_selftest(D.data_ptr(), N, variant) == T.SUCCESS
    i = np.arange(128)[:, None]
    k = np.arange(16)[None, :]
    A = ((7 * i + 3 * k) % 11 - 5).astype(np.float64)
    kk = np.arange(16)[:, None]
    c = np.arange(N)[None, :]
    B = ((5 * kk + 2 * c) % 7 - 3).astype(np.float64)
    np.testing.assert_array_equal(D.cpu().numpy().astype(np.float64), A @ B)


def test_peaks_are_plausible(T):
    p = T.measure_peaks()
    assert 0.3 < p["fp64_dfma"] < 5.0
    assert 20.0 < p["fp32_ffma"] < 200.0
    assert 50.0 < p["tf32_mma_sync"] < 3000.0
    assert 100.0 < p["tf32_tcgen05"] < 4000.0
    assert 300.0 < p["bf16_tcgen05"] < 6000.0
