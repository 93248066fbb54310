"""GPU parity of the real-symmetric path (float64 H and blocks) against the
oracle, which treats a real symmetric matrix as a Hermitian one (its results
are then real).  Same bars as the complex path: filter 1e-11 (FP64) and
max(1e-11, 4 m sqrt(N) 2^-49) (split-BF16, K = N terms per product;
``tests/tolerances.py``) relative per column; eigenvalues 1e-10 ||H||; residuals
tol ||H||.  Odd orders and odd leading dimensions exercise the staging of
real arrays into the even leading dimensions the TMA products need."""

import numpy as np
import pytest
import torch

import oracle
from paper_1805_10121_gb300 import chase, synth
from tests.tolerances import FP64_FILTER_RTOL, split_filter_rtol

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
EIG_RTOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1805_10121_gb300 import build
    build.build()
    chase.lib()


def dcol(t, ld=None):
    """Column-major device copy, optionally with a larger leading dimension."""
    n, b = t.shape
    if ld is None or ld == n:
        return t.to(DEV).t().contiguous().t()
    buf = torch.zeros(b, ld, dtype=t.dtype, device=DEV)
    buf[:, :n] = t.t().to(DEV)
    return buf.t()[:n, :]


def known_h(n, seed, n_cluster=None):
    q = synth.orthogonal_qr(n, seed)
    lam = synth.spectrum_clustered(n, seed + 1, n_cluster=n_cluster or max(2, n // 16))
    return synth.symmetric_from(q, lam), lam


def oracle_filter_any_order(H, V, deg, b_sup, mu1, mu_nn):
    order = np.argsort(deg, kind="stable")
    out = np.empty(V.shape, dtype=np.complex128)
    out[:, order] = oracle.cheb_filter(H, V[:, order], np.asarray(deg)[order], b_sup, mu1, mu_nn)
    assert np.max(np.abs(out.imag)) == 0.0
    return out.real


def col_rel_err(a, b):
    return np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0))


@pytest.mark.parametrize("precision", [chase.CHASE_FP64, chase.CHASE_SPLIT_BF16])
@pytest.mark.parametrize("n,b,ld", [(300, 37, None), (517, 70, None), (129, 1, None),
                                    (1001, 33, None), (400, 9, 403)])
def test_real_filter_matches_oracle(precision, n, b, ld):
    H, lam = known_h(n, 311 + n)
    V = synth.gaussian_block_real(n, b, 312 + b)
    rng = np.random.default_rng(n + 5 * b)
    deg = (2 * rng.integers(1, 19, size=b)).astype(np.int32)
    l = lam.numpy()
    b_sup, mu1, mu_nn = 1.02, float(l[0]), float(l[min(n - 1, max(1, n // 8))])
    ref = oracle_filter_any_order(H.numpy(), V.numpy(), deg, b_sup, mu1, mu_nn)
    Vd = dcol(V, ld)
    chase.chase_filter_real(dcol(H, ld), Vd, deg, b_sup, mu1, mu_nn, precision=precision)
    err = col_rel_err(Vd.cpu().numpy(), ref)
    bound = (FP64_FILTER_RTOL if precision == chase.CHASE_FP64
             else split_filter_rtol(n, int(deg.max()), real=True))
    assert err <= bound, err


def test_real_filter_host_arrays():
    n, b = 257, 12
    H, lam = known_h(n, 321)
    V = synth.gaussian_block_real(n, b, 322).contiguous().t().contiguous().t()
    deg = np.full(b, 10, dtype=np.int32)
    l = lam.numpy()
    ref = oracle_filter_any_order(H.numpy(), V.numpy(), deg, 1.02, float(l[0]), float(l[40]))
    Vh = V.clone()
    chase.chase_filter_real(H, Vh, deg, 1.02, float(l[0]), float(l[40]))
    assert col_rel_err(Vh.numpy(), ref) <= FP64_FILTER_RTOL


def test_real_residuals():
    n, b = 333, 20
    H, lam = known_h(n, 331)
    V = synth.gaussian_block_real(n, b, 332)
    w = np.linspace(-1, 1, b)
    got = chase.chase_residuals_real(dcol(H), dcol(V), w)
    Hn, Vn = H.numpy(), V.numpy()
    ref = np.linalg.norm(Hn @ Vn - Vn * w[None, :], axis=0)
    assert np.max(np.abs(got - ref) / ref) <= 1e-12


@pytest.mark.parametrize("precision", [chase.CHASE_FP64, chase.CHASE_SPLIT_BF16,
                                       chase.CHASE_SPLIT_BF16_RR])
@pytest.mark.parametrize("n,nev,nex", [(1000, 50, 20), (601, 30, 11)])
def test_real_solve_known_spectrum(precision, n, nev, nex):
    tol = 1e-10
    H, lam = known_h(n, 341 + n, n_cluster=60)
    V0 = synth.gaussian_block_real(n, nev + nex, 342)
    S = synth.gaussian_block_real(n, 5, 343)
    Vd = dcol(V0)
    o = chase.chase_opts_default(precision=precision)
    st, ritz, resid, stats = chase.chase_solve_real(dcol(H), nev, nex, tol, Vd, dcol(S), opts=o)
    assert st == chase.CHASE_OK
    l = lam.numpy()
    hn = float(np.abs(l).max())
    assert np.max(np.abs(ritz[:nev] - l[:nev])) <= EIG_RTOL * hn
    assert np.all(resid[:nev] <= tol * hn)
    V = Vd.cpu().numpy()
    assert np.linalg.norm(V.T @ V - np.eye(nev + nex)) < 1e-12
    r = oracle.residuals(H.numpy(), V[:, :nev], ritz[:nev])
    assert np.all(r <= tol * hn * 1.05)
    # a real problem takes 2 N^2 FLOPs per column product
    assert stats["flops_filter"] == pytest.approx(2.0 * n * n * stats["filter_matvecs"])


def test_real_solve_matches_complex_embedding():
    # the same symmetric matrix solved as a Hermitian one gives the same pairs
    n, nev, nex, tol = 500, 25, 10, 1e-10
    H, lam = known_h(n, 351)
    V0 = synth.gaussian_block_real(n, nev + nex, 352)
    S = synth.gaussian_block_real(n, 5, 353)
    st, rr, res_r, _ = chase.chase_solve_real(dcol(H), nev, nex, tol, dcol(V0), dcol(S))
    assert st == chase.CHASE_OK
    Hc = H.to(torch.complex128)
    st, rc, res_c, _ = chase.chase_solve(dcol(Hc), nev, nex, tol, dcol(V0.to(torch.complex128)),
                                         dcol(S.to(torch.complex128)))
    assert st == chase.CHASE_OK
    hn = float(lam.abs().max())
    assert np.max(np.abs(rr[:nev] - rc[:nev])) <= EIG_RTOL * hn
