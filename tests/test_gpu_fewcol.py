"""GPU parity of the few-column products (one to six active columns: the
Lanczos matvecs and the last degree steps of the filter) in all four scalar
kinds, through chase_filter* and chase_residuals* against the oracle.
Seven columns take the tensor-core tile path and are checked beside them.
n = 517 leaves a ragged tail in rows (8, 16 or 32 rows per block) and in
K (16, 8 or 4 K lanes times an unroll of 8 or 4)."""

import numpy as np
import pytest
import torch

import oracle
from paper_1805_10121_gb300 import chase, synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
KINDS = {
    # entry suffix, torch dtype, real?, filter tolerance, residual tolerance
    "c64": ("", torch.complex128, False, 1e-11, 1e-12),
    "f64": ("_real", torch.float64, True, 1e-11, 1e-12),
    "c32": ("_c32", torch.complex64, False, 1e-4, 1e-5),
    "f32": ("_f32", torch.float32, True, 1e-4, 1e-5),
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1805_10121_gb300 import build
    build.build()
    chase.lib()


def dcol(t, ld=None):
    n, b = t.shape
    if ld is None or ld == n:
        return t.to(DEV).t().contiguous().t()
    buf = torch.zeros(b, ld, dtype=t.dtype, device=DEV)
    buf[:, :n] = t.t().to(DEV)
    return buf.t()[:n, :]


def problem(n, seed, real):
    lam = synth.spectrum_clustered(n, seed + 1, n_cluster=max(2, n // 16))
    if real:
        return synth.symmetric_from(synth.orthogonal_qr(n, seed), lam), lam
    return synth.hermitian_from(synth.unitary_qr(n, seed), lam), lam


def col_rel_err(a, b):
    return np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0))


@pytest.mark.parametrize("kind", list(KINDS))
@pytest.mark.parametrize("b", [1, 2, 3, 5, 6, 7])
@pytest.mark.parametrize("ld", [None, 523])
def test_fewcol_filter_matches_oracle(kind, b, ld):
    suffix, dt, real, ftol, _ = KINDS[kind]
    n = 517
    H, lam = problem(n, 900 + b, real)
    V = synth.gaussian_block_real(n, b, 901 + b) if real else synth.gaussian_block(n, b, 901 + b)
    # distinct even degrees: the active block shrinks one column at a time
    deg = np.array([2, 4, 6, 8, 12, 16, 20][:b], dtype=np.int32)[::-1].copy()
    l = lam.numpy()
    b_sup, mu1, mu_nn = 1.02, float(l[0]), float(l[n // 8])
    Hd = H.to(dt)
    Vd = dcol(V.to(dt), ld)
    order = np.argsort(deg, kind="stable")
    ref = np.empty((n, b), dtype=np.complex128)
    Hn = Hd.cpu().to(torch.complex128 if not real else torch.float64).numpy()
    Vn = V.to(dt).cpu().to(torch.complex128 if not real else torch.float64).numpy()
    ref[:, order] = oracle.cheb_filter(Hn, Vn[:, order], deg[order], b_sup, mu1, mu_nn)
    getattr(chase, "chase_filter" + suffix)(dcol(Hd, ld), Vd, deg, b_sup, mu1, mu_nn)
    got = Vd.cpu().to(torch.complex128 if not real else torch.float64).numpy()
    assert col_rel_err(got, ref) <= ftol


@pytest.mark.parametrize("kind", list(KINDS))
@pytest.mark.parametrize("b", [1, 4, 6, 7])
def test_fewcol_residuals(kind, b):
    suffix, dt, real, _, rtol = KINDS[kind]
    n = 517
    H, _ = problem(n, 950 + b, real)
    V = synth.gaussian_block_real(n, b, 951) if real else synth.gaussian_block(n, b, 951)
    w = np.linspace(-1.0, 1.0, b) if b > 1 else np.array([0.3])
    got = getattr(chase, "chase_residuals" + suffix)(dcol(H.to(dt)), dcol(V.to(dt)), w)
    wide = torch.complex128 if not real else torch.float64
    Hn, Vn = H.to(dt).to(wide).numpy(), V.to(dt).to(wide).numpy()
    ref = np.linalg.norm(Hn @ Vn - Vn * w[None, :], axis=0)
    assert np.max(np.abs(got - ref) / ref) <= rtol
