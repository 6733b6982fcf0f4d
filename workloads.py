"""Seeded synthetic inputs shaped like the tall-and-skinny workloads of the R-factor TSQR.

This module only draws random matrices; it holds none of the method's arithmetic and is the
one module that both the GPU path's callers and the CPU oracle's callers share.

Storage convention: a column-major m x n matrix A with leading dimension lda = m is held by a
row-major torch tensor of shape (n, m) (row k of the tensor is column k of A).

Recipes (all in float64 on the CPU unless ``device`` says otherwise):

* ``gaussian``      -- iid N(0, 1) entries from ``torch.Generator().manual_seed(seed)``,
  drawn as ``randn(n, m)`` so that column k of A is drawn before column k+1.
* ``conditioned``   -- A = G diag(sigma) V^T with G iid N(0,1) (m x n, drawn first),
  V Haar-orthogonal n x n (QR of an n x n Gaussian from the same generator with the column
  signs fixed so that the triangular factor has a positive diagonal, Mezzadri 2007), and
  sigma_k = kappa^(-k/(n-1)), k = 0..n-1 (geometric from 1 to 1/kappa).
* ``varlen_batch``  -- a batch of independent Gaussian problems with m log-uniform in
  [m_lo, m_hi] and n uniform over a set, drawn in the order: all m, then all n, then the
  matrices one after another; packed back to back into one column-major buffer.
"""
from __future__ import annotations

import hashlib
import math

import torch


def gaussian(m: int, n: int, seed: int = 0, dtype=torch.float64, device="cpu") -> torch.Tensor:
    """(n, m) tensor holding a column-major m x n matrix with iid N(0,1) entries."""
    if device == "cpu":
        g = torch.Generator().manual_seed(seed)
        a = torch.randn(n, m, generator=g, dtype=torch.float64)
    else:
        g = torch.Generator(device=device).manual_seed(seed)
        a = torch.randn(n, m, generator=g, dtype=torch.float64, device=device)
    return a if dtype == torch.float64 else a.to(dtype)


def haar_orthogonal(n: int, g: torch.Generator) -> torch.Tensor:
    """n x n Haar-distributed orthogonal matrix (Mezzadri's sign-fixed QR of a Gaussian)."""
    z = torch.randn(n, n, generator=g, dtype=torch.float64)
    q, r = torch.linalg.qr(z)
    d = torch.sign(torch.diagonal(r))
    d[d == 0] = 1.0
    return q * d


def conditioned(m: int, n: int, kappa: float, seed: int = 0, dtype=torch.float64,
                device="cpu", device_draw: bool = False) -> torch.Tensor:
    """(n, m) tensor holding A = G diag(sigma) V^T, sigma geometric from 1 to 1/kappa.

    With ``device_draw`` and a CUDA ``device``, G is drawn on the device by a device generator
    seeded with ``seed`` (same distribution, other values; for large sizes), V still from the
    CPU generator."""
    g = torch.Generator().manual_seed(seed)
    if device_draw and device != "cpu":
        gd = torch.Generator(device=device).manual_seed(seed)
        G = torch.randn(n, m, generator=gd, dtype=torch.float64, device=device)
        torch.randn(n, 1, generator=g, dtype=torch.float64)  # keep V's draw independent of m
    else:
        G = torch.randn(n, m, generator=g, dtype=torch.float64)       # column-major G
    V = haar_orthogonal(n, g)
    if n > 1:
        k = torch.arange(n, dtype=torch.float64)
        sigma = torch.pow(torch.tensor(float(kappa), dtype=torch.float64), -k / (n - 1))
    else:
        sigma = torch.ones(1, dtype=torch.float64)
    M = sigma[:, None] * V.T                                            # diag(sigma) V^T
    # A = G M  =>  A^T = M^T G^T, and the (n, m) storage of A is A^T.
    dev = device if device != "cpu" else "cpu"
    At = M.T.to(dev) @ G.to(dev)
    return At if dtype == torch.float64 else At.to(dtype)


def varlen_batch(count: int, m_lo: int, m_hi: int, n_choices=(8, 16, 32, 64), seed: int = 0,
                 dtype=torch.float64, device="cpu"):
    """Packed varlen batch.

    Returns (buf, ms, ns, offs): ``buf`` a flat tensor holding every A_i column-major with
    lda_i = m_i back to back, ``offs[i]`` the element offset of A_i in ``buf``.  With a CUDA
    ``device`` the sizes are drawn as on the CPU but the entries come from one device-side
    N(0,1) draw (for large batches)."""
    g = torch.Generator().manual_seed(seed)
    u = torch.rand(count, generator=g, dtype=torch.float64)
    ms = torch.round(torch.exp(math.log(m_lo) + u * (math.log(m_hi) - math.log(m_lo))))
    ms = ms.to(torch.int64).clamp(m_lo, m_hi)
    idx = torch.randint(0, len(n_choices), (count,), generator=g)
    ns = torch.tensor(n_choices, dtype=torch.int64)[idx]
    sizes = ms * ns
    offs = torch.zeros(count + 1, dtype=torch.int64)
    offs[1:] = torch.cumsum(sizes, 0)
    if device != "cpu":
        gd = torch.Generator(device=device).manual_seed(seed)
        buf = torch.randn(int(offs[-1]), generator=gd, dtype=torch.float64, device=device)
        return (buf if dtype == torch.float64 else buf.to(dtype)), ms.tolist(), ns.tolist(), \
            offs.tolist()
    buf = torch.empty(int(offs[-1]), dtype=torch.float64)
    for i in range(count):
        buf[int(offs[i]):int(offs[i + 1])] = torch.randn(int(sizes[i]), generator=g,
                                                         dtype=torch.float64)
    if dtype != torch.float64:
        buf = buf.to(dtype)
    return buf, ms.tolist(), ns.tolist(), offs.tolist()


def sha256(t: torch.Tensor) -> str:
    """SHA-256 of a tensor's bytes (recorded beside each workload)."""
    return hashlib.sha256(t.detach().cpu().contiguous().numpy().tobytes()).hexdigest()
