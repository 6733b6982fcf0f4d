"""tsqr_r_host (A and R in host memory; page-locked A is read in place by tsqr_r's kernel
through its device mapping, other memory is copied first): parity with the oracle (every entry
within c(m) kappa u ||R||_F, c(m) = max(50, 2 sqrt(m)), Gram residual <= 1e-13), R equal to
tsqr_r's bytes (same plan and kernel), page-locked and pageable A, a padded lda and ldr, m = 0,
a clean device status afterwards, and the same R with every launch serialized
(CUDA_LAUNCH_BLOCKING=1), which a design that needs copies and kernels to run concurrently
would fail."""
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
    return T


def _check(oracle, A, R):
    m = A.shape[0]
    Ro = oracle.householder_r(A, nthreads=16)
    kap = oracle.kappa_from_r(Ro)
    np.testing.assert_allclose(R, Ro, rtol=0,
                               atol=max(50.0, 2.0 * np.sqrt(m)) * kap * U * np.linalg.norm(Ro))
    assert oracle.gram_residual(A, R, nthreads=16) <= 1e-13


@pytest.mark.parametrize("m,n,pinned", [(5000, 16, True), (300000, 32, True), (1000003, 32, False),
                                        (2500000, 24, True), (4194304, 32, True), (777, 3, False)])
def test_host_input_parity(oracle, T, m, n, pinned):
    import torch
    At = workloads.gaussian(m, n, seed=m % 89)
    Ah = At.pin_memory() if pinned else At
    R = T.tsqr_r_host(Ah.T)
    assert T.capi.tsqr_last_launch_count() == 1
    assert T.tsqr_get_device_status() == T.SUCCESS
    assert torch.equal(R, T.tsqr_r(At.cuda().T).cpu())
    _check(oracle, oracle.from_torch_colmajor(At), R.numpy())


@pytest.mark.parametrize("m,n,pinned", [(200003, 96, True), (50000, 200, False)])
def test_host_input_by_panels(oracle, T, m, n, pinned):
    """Where the AUTO plan runs by panels (n >= 56, tall; and every n above 128), host A is
    copied whole and the panels run on it: R equals tsqr_r's bytes on the device copy."""
    import torch
    At = workloads.gaussian(m, n, seed=n)
    Ah = At.pin_memory() if pinned else At
    R = T.tsqr_r_host(Ah.T)
    torch.cuda.synchronize()
    p = T.last_plan()
    assert (p.tree, p.tile_rows) == (T.TREE_PANELS, 16)
    assert torch.equal(R, T.tsqr_r(At.cuda().T).cpu())
    Ro = oracle.householder_r(oracle.from_torch_colmajor(At), nthreads=16)
    c = max(50.0, 2.0 * np.sqrt(m * n / 32.0))
    np.testing.assert_allclose(R.numpy(), Ro, rtol=0,
                               atol=c * oracle.kappa_from_r(Ro) * U * np.linalg.norm(Ro))


def test_host_input_leading_dimensions_and_empty(oracle, T):
    import torch
    m, n = 123457, 20
    At = workloads.gaussian(m, n, seed=3)
    big = torch.zeros(n, m + 5, dtype=torch.float64)
    big[:, :m] = At
    Rbig = torch.full((n, n + 2), float("nan"), dtype=torch.float64)
    R = T.tsqr_r_host(big.pin_memory().T[:m, :], R=Rbig.T[:n, :])
    torch.cuda.synchronize()
    _check(oracle, oracle.from_torch_colmajor(At), R.numpy())
    assert torch.isnan(Rbig[:, n:]).all()
    Z = torch.zeros(0, 4, dtype=torch.float64)
    assert np.all(T.tsqr_r_host(Z).numpy() == 0)


_SERIAL = r"""
import sys, torch
sys.path.insert(0, {root!r})
import workloads, paper_1002_4250_gb300 as T
At = workloads.gaussian({m}, {n}, seed=7)
Rh = T.tsqr_r_host(At.pin_memory().T)
Rd = T.tsqr_r(At.cuda().T).cpu()
torch.cuda.synchronize()
assert T.tsqr_get_device_status() == T.SUCCESS
torch.save(Rh.T.contiguous(), {out!r})
print("same" if torch.equal(Rh, Rd) else "differ")
"""


def test_host_input_serialized_launches(oracle, T, tmp_path):
    """With CUDA_LAUNCH_BLOCKING=1 every launch and copy runs alone: R must still be tsqr_r's
    R (no part of the call may depend on a copy and a kernel running at the same time)."""
    import os
    import subprocess
    import sys
    import torch
    m, n = 1500000, 32
    out = str(tmp_path / "R.pt")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CUDA_LAUNCH_BLOCKING="1")
    r = subprocess.run([sys.executable, "-c", _SERIAL.format(root=root, m=m, n=n, out=out)],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip().endswith("same")
    R = torch.load(out).T.numpy()
    _check(oracle, oracle.from_torch_colmajor(workloads.gaussian(m, n, seed=7)), R)
