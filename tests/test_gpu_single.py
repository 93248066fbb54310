"""GPU checks of the single-precision path (complex64 and float32 entry
points) against the oracle in double precision.  Tolerances follow FP32
arithmetic: a product with H carries about sqrt(N) 6e-8 relative error, a
degree-m filter about m times that, so filtered columns are compared at
1e-4 relative for degrees up to 20; solves use tol = 1e-5 (Table 1's
single-precision column) and eigenvalues must match the known spectrum to
1e-5 ||H||."""

import numpy as np
import pytest
import torch

import oracle
from paper_1805_10121_gb300 import chase, synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
FILTER_RTOL = 1e-4
EIG_RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1805_10121_gb300 import build
    build.build()
    chase.lib()


def dcol(t):
    return t.to(DEV).t().contiguous().t()


def problem(n, seed, real, n_cluster=None):
    lam = synth.spectrum_clustered(n, seed + 1, n_cluster=n_cluster or max(2, n // 16))
    if real:
        H = synth.symmetric_from(synth.orthogonal_qr(n, seed), lam)
    else:
        H = synth.hermitian_from(synth.unitary_qr(n, seed), lam)
    return H, lam


def block(n, b, seed, real):
    return synth.gaussian_block_real(n, b, seed) if real else synth.gaussian_block(n, b, seed)


def oracle_filter_any_order(H, V, deg, b_sup, mu1, mu_nn):
    order = np.argsort(deg, kind="stable")
    out = np.empty(V.shape, dtype=np.complex128)
    out[:, order] = oracle.cheb_filter(H, V[:, order], np.asarray(deg)[order], b_sup, mu1, mu_nn)
    return out


def col_rel_err(a, b):
    return np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0))


@pytest.mark.parametrize("real", [False, True])
@pytest.mark.parametrize("n,b", [(300, 37), (517, 70), (129, 1), (1000, 33)])
def test_single_filter_matches_oracle(real, n, b):
    H, lam = problem(n, 411 + n, real)
    V = block(n, b, 412 + b, real)
    rng = np.random.default_rng(n + 7 * b)
    deg = (2 * rng.integers(1, 11, size=b)).astype(np.int32)
    l = lam.numpy()
    b_sup, mu1, mu_nn = 1.02, float(l[0]), float(l[min(n - 1, max(1, n // 8))])
    ref = oracle_filter_any_order(H.numpy(), V.numpy(), deg, b_sup, mu1, mu_nn)
    if real:
        Vd = dcol(V.to(torch.float32))
        chase.chase_filter_f32(dcol(H.to(torch.float32)), Vd, deg, b_sup, mu1, mu_nn)
    else:
        Vd = dcol(V.to(torch.complex64))
        chase.chase_filter_c32(dcol(H.to(torch.complex64)), Vd, deg, b_sup, mu1, mu_nn)
    got = Vd.cpu().numpy().astype(np.complex128)
    assert col_rel_err(got, ref) <= FILTER_RTOL


@pytest.mark.parametrize("real", [False, True])
def test_single_residuals(real):
    n, b = 333, 20
    H, lam = problem(n, 431, real)
    V = block(n, b, 432, real)
    w = np.linspace(-1, 1, b)
    if real:
        got = chase.chase_residuals_f32(dcol(H.to(torch.float32)), dcol(V.to(torch.float32)), w)
        Hn, Vn = H.to(torch.float32).double().numpy(), V.to(torch.float32).double().numpy()
    else:
        got = chase.chase_residuals_c32(dcol(H.to(torch.complex64)), dcol(V.to(torch.complex64)), w)
        Hn = H.to(torch.complex64).to(torch.complex128).numpy()
        Vn = V.to(torch.complex64).to(torch.complex128).numpy()
    ref = np.linalg.norm(Hn @ Vn - Vn * w[None, :], axis=0)
    assert np.max(np.abs(got - ref) / ref) <= 1e-5


@pytest.mark.parametrize("precision", [chase.CHASE_FP64, chase.CHASE_SPLIT_BF16])
@pytest.mark.parametrize("real", [False, True])
@pytest.mark.parametrize("n,nev,nex", [(1000, 50, 20), (601, 30, 11)])
def test_single_solve_known_spectrum(real, n, nev, nex, precision):
    """FP32 products throughout, or (CHASE_SPLIT_BF16) the filter on the
    four-slice split product over widened copies of the block."""
    tol = 1e-5
    H, lam = problem(n, 441 + n, real, n_cluster=60)
    V0 = block(n, nev + nex, 442, real)
    S = block(n, 5, 443, real)
    dt = torch.float32 if real else torch.complex64
    Vd = dcol(V0.to(dt))
    solve = chase.chase_solve_f32 if real else chase.chase_solve_c32
    st, ritz, resid, stats = solve(dcol(H.to(dt)), nev, nex, tol, Vd, dcol(S.to(dt)),
                                   opts=chase.chase_opts_default(precision=precision))
    assert st == chase.CHASE_OK
    if precision != chase.CHASE_FP64:
        assert stats["filter_slices_low"] == stats["iterations"]  # 4 slices every iteration
    l = lam.numpy()
    hn = float(np.abs(l).max())
    assert np.max(np.abs(ritz[:nev] - l[:nev])) <= EIG_RTOL * hn
    assert np.all(resid[:nev] <= tol * hn)
    V = Vd.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(V.conj().T @ V - np.eye(nev + nex)) < 1e-4
    r = oracle.residuals(H.numpy(), V[:, :nev], ritz[:nev])
    assert np.all(r <= tol * hn * 1.5)
