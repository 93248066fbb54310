"""Seeded synthetic inputs shared by the tests, the bench and the oracle runs.

This module only builds inputs: Hermitian test matrices with a prescribed
spectrum, the correlated perturbations of a problem sequence and random start
blocks.  It contains none of the eigensolver's arithmetic.  Every generator
takes an integer seed and a torch device; the same seed on the same device
type gives the same tensor.

Workload shapes follow the paper's DFT workloads (Sec. 4.1.4, Sec. 6.1):
a dense low band of eigenvalues below a sparse tail, and sequences whose
consecutive problems differ by a small Hermitian perturbation.
"""

from __future__ import annotations

import math
import threading

import torch

# torch.fft executes cached cuFFT plans whose stream and work area are set
# on the shared plan just before each execution; generators running in
# several threads at once (the serving loop builds each request's matrices
# in its own thread) take this lock around every FFT call so that a plan is
# never re-pointed by one thread while another enqueues it.
_FFT_LOCK = threading.Lock()


def _fft(x, dim, inverse=False):
    with _FFT_LOCK:
        return (torch.fft.ifft if inverse else torch.fft.fft)(x, dim=dim, norm="ortho")

__all__ = [
    "generator",
    "gaussian_block",
    "unitary_qr",
    "unitary_dft",
    "spectrum_clustered",
    "spectrum_dft",
    "spectrum_uniform",
    "hermitian_from",
    "hermitian_dft",
    "hermitian_noise",
    "batched_shapes",
    "orthogonal_qr",
    "symmetric_from",
    "gaussian_block_real",
]


def generator(seed: int, device="cpu") -> torch.Generator:
    g = torch.Generator(device=torch.device(device))
    g.manual_seed(int(seed))
    return g


def gaussian_block(n: int, b: int, seed: int, device="cpu") -> torch.Tensor:
    """i.i.d. complex Gaussian block (n x b, complex128, column-major storage)."""
    g = generator(seed, device)
    re = torch.randn(b, n, dtype=torch.float64, device=device, generator=g)
    im = torch.randn(b, n, dtype=torch.float64, device=device, generator=g)
    # store as the transpose of a contiguous (b, n) tensor: columns are contiguous
    return torch.complex(re, im).mul_(1.0 / math.sqrt(2.0)).t()


def unitary_qr(n: int, seed: int, device="cpu") -> torch.Tensor:
    """Random unitary: QR of an i.i.d. complex Gaussian, phases fixed so that
    R has a positive real diagonal (Haar distributed)."""
    g = generator(seed, device)
    re = torch.randn(n, n, dtype=torch.float64, device=device, generator=g)
    im = torch.randn(n, n, dtype=torch.float64, device=device, generator=g)
    z = torch.complex(re, im)
    q, r = torch.linalg.qr(z)
    d = torch.diagonal(r)
    ph = d / d.abs()
    return q * ph[None, :]


def unitary_dft(n: int, seed: int, device="cpu") -> torch.Tensor:
    """Dense structured unitary ``D1 F D2 F D3`` (F the unitary DFT, D_i
    random phase diagonals).  O(n^2 log n) to form, unitary to rounding."""
    g = generator(seed, device)
    ph = torch.rand(3, n, dtype=torch.float64, device=device, generator=g) * (2.0 * math.pi)
    d = torch.polar(torch.ones_like(ph), ph)
    x = torch.diag(d[2])
    x = _fft(x, 0)
    x = x * d[1][:, None]
    x = _fft(x, 0)
    return x * d[0][:, None]


def spectrum_clustered(n: int, seed: int, n_cluster: int = 60, device="cpu") -> torch.Tensor:
    """``n_cluster`` values U[-1, -0.9] and the rest U(-0.9, 1]; ascending."""
    g = generator(seed, device)
    lo = -1.0 + 0.1 * torch.rand(n_cluster, dtype=torch.float64, device=device, generator=g)
    hi = -0.9 + 1.9 * (1.0 - torch.rand(n - n_cluster, dtype=torch.float64, device=device,
                                       generator=g))
    return torch.sort(torch.cat([lo, hi])).values


def spectrum_dft(n: int, seed: int, device="cpu") -> torch.Tensor:
    """DFT-like density: n/4 values U[-2, 0] (dense low band) and 3n/4 values
    ``50 u^2``, u ~ U(0, 1] (sparse tail up to 50, no gap); ascending."""
    g = generator(seed, device)
    nb = n // 4
    band = -2.0 + 2.0 * torch.rand(nb, dtype=torch.float64, device=device, generator=g)
    u = 1.0 - torch.rand(n - nb, dtype=torch.float64, device=device, generator=g)
    return torch.sort(torch.cat([band, 50.0 * u * u])).values


def spectrum_uniform(n: int, seed: int, device="cpu") -> torch.Tensor:
    g = generator(seed, device)
    return torch.sort(-1.0 + 2.0 * torch.rand(n, dtype=torch.float64, device=device,
                                              generator=g)).values


def hermitian_from(q: torch.Tensor, lam: torch.Tensor) -> torch.Tensor:
    """``H = Q diag(lam) Q^H`` as a full (both triangles) Hermitian matrix,
    stored column-major (the returned tensor is the transpose view of a
    contiguous row-major array, so its columns are contiguous)."""
    h = (q * lam.to(q.dtype)[None, :]) @ q.conj().t()
    h = 0.5 * (h + h.conj().t())
    # column-major storage: element (i, j) at j*n + i
    return h.t().contiguous().t()


def hermitian_dft(lam: torch.Tensor, seed: int, chunk: int = 2048) -> torch.Tensor:
    """``Q diag(lam) Q^H`` for the unitary ``Q = D1 F D2 F D3`` of
    ``unitary_dft(n, seed)`` without forming Q: ``D3 diag(lam) D3^H`` is
    ``diag(lam)``, ``F diag(lam) F^H`` is circulant with first column
    ``fft(lam) / n``, and the remaining factors are FFTs along the two axes
    and phase scalings.  O(n^2 log n); column-major full storage.  Works in
    place on one n x n buffer, ``chunk`` columns or rows at a time, so that
    n = 30000 (14.4 GB) also builds in host memory."""
    n = lam.numel()
    device = lam.device
    g = generator(seed, device)
    ph = torch.rand(3, n, dtype=torch.float64, device=device, generator=g) * (2.0 * math.pi)
    d = torch.polar(torch.ones_like(ph), ph)
    with _FFT_LOCK:
        c = torch.fft.fft(lam.to(torch.complex128)) / n       # circulant column
    t = torch.empty((n, n), dtype=torch.complex128, device=device)
    rows = torch.arange(n, device=device)
    for j0 in range(0, n, chunk):                              # F diag(lam) F^H, D2 . D2^H, F .
        j1 = min(n, j0 + chunk)
        blk = c[(rows[:, None] - rows[None, j0:j1]) % n]
        blk.mul_(d[1][:, None]).mul_(d[1][j0:j1].conj()[None, :])
        t[:, j0:j1] = _fft(blk, 0)
        del blk
    for i0 in range(0, n, chunk):                              # . F^H, D1 . D1^H
        i1 = min(n, i0 + chunk)
        blk = _fft(t[i0:i1, :], 1, inverse=True)
        blk.mul_(d[0][i0:i1, None]).mul_(d[0].conj()[None, :])
        t[i0:i1, :] = blk
        del blk
    # Hermitian part, tile pair by tile pair: t <- (t + t^H) / 2
    for i0 in range(0, n, chunk):
        i1 = min(n, i0 + chunk)
        for j0 in range(i0, n, chunk):
            j1 = min(n, j0 + chunk)
            a = t[i0:i1, j0:j1].clone()
            b = t[j0:j1, i0:i1].clone()
            t[i0:i1, j0:j1] = 0.5 * (a + b.conj().t())
            t[j0:j1, i0:i1] = 0.5 * (b + a.conj().t())
            del a, b
    # column-major storage of a Hermitian h is the row-major storage of conj(h)
    t.conj_physical_()
    return t.t()


def hermitian_noise(n: int, seed: int, device="cpu") -> torch.Tensor:
    """``E = (G + G^H) / (2 sqrt(2n))`` with G i.i.d. complex Gaussian of unit
    entry variance: off-diagonal variance 1/(4n), so the semicircle edge, and
    ``||E||_2``, is close to 1."""
    g = generator(seed, device)
    re = torch.randn(n, n, dtype=torch.float64, device=device, generator=g)
    im = torch.randn(n, n, dtype=torch.float64, device=device, generator=g)
    z = torch.complex(re, im).mul_(1.0 / math.sqrt(2.0))
    e = (z + z.conj().t()) * (1.0 / (2.0 * math.sqrt(2.0 * n)))
    return e.t().contiguous().t()


def batched_shapes(P: int, seed: int, n_lo: int = 256, n_hi: int = 2048,
                   nev_frac: float = 0.05, nex_frac: float = 0.02):
    """Sizes of a batch of independent problems: N uniform in [n_lo, n_hi],
    nev = ceil(nev_frac N), nex = ceil(nex_frac N); a list of (N, nev, nex)."""
    g = generator(seed, "cpu")
    ns = torch.randint(n_lo, n_hi + 1, (P,), generator=g).tolist()
    return [(int(n), int(math.ceil(nev_frac * n)), int(math.ceil(nex_frac * n))) for n in ns]


def orthogonal_qr(n: int, seed: int, device="cpu") -> torch.Tensor:
    """Random orthogonal matrix: QR of an i.i.d. real Gaussian, signs fixed
    so that R has a positive diagonal (Haar distributed)."""
    g = generator(seed, device)
    z = torch.randn(n, n, dtype=torch.float64, device=device, generator=g)
    q, r = torch.linalg.qr(z)
    return q * torch.sign(torch.diagonal(r))[None, :]


def symmetric_from(q: torch.Tensor, lam: torch.Tensor) -> torch.Tensor:
    """``H = Q diag(lam) Q^T`` (real symmetric, both triangles), column-major."""
    h = (q * lam[None, :]) @ q.t()
    h = 0.5 * (h + h.t())
    return h.t().contiguous().t()


def symmetric_noise(n: int, seed: int, device="cpu") -> torch.Tensor:
    """``E = (G + G^T) / (2 sqrt(2n))`` with G i.i.d. real Gaussian: the real
    counterpart of ``hermitian_noise`` (off-diagonal variance 1/(4n), so
    ``||E||_2`` is close to 1)."""
    g = generator(seed, device)
    z = torch.randn(n, n, dtype=torch.float64, device=device, generator=g)
    e = (z + z.t()) * (1.0 / (2.0 * math.sqrt(2.0 * n)))
    return e.t().contiguous().t()


def gaussian_block_real(n: int, b: int, seed: int, device="cpu") -> torch.Tensor:
    """n x b real Gaussian block, column-major."""
    g = generator(seed, device)
    return torch.randn(b, n, dtype=torch.float64, device=device, generator=g).t()
