"""GPU parity of the split-BF16 (tensor-core) filter and of full solves that
use it, against the CPU oracle and known spectra.

Tolerance of the filter: each split-BF16 product carries an error of about
2^-49 max|off-diagonal row of H| max|column| per term (7 slices of 7 bits);
the diagonal of H and the shift are applied exactly in FP64.  The K terms'
errors add like sqrt(K) and a degree-m filter chains m products, so each
column is held to the FP64 filter's bar of 1e-11, or to 4 m sqrt(K) 2^-49
where that is larger (``tolerances.split_filter_rtol``: 1e-11 up to
N = 1000, 3.2e-11 at N = 8000, 5.4e-11 at N = 22500 with m = 36).  Full solves
must meet the same eigenvalue (1e-10 ||H||) and residual (tol ||H||) bars as
the FP64 path, because Rayleigh-Ritz, QR and residuals stay FP64."""

import numpy as np
import pytest
import torch

import oracle
from paper_1805_10121_gb300 import chase, synth
from tests.tolerances import reduced_slice_rtol, split_filter_rtol

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
EIG_RTOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1805_10121_gb300 import build
    build.build()
    chase.lib()


def dcol(t):
    return t.to(DEV).t().contiguous().t()


def known_h(n, seed, n_cluster=None):
    q = synth.unitary_qr(n, seed)
    lam = synth.spectrum_clustered(n, seed + 1, n_cluster=n_cluster or max(2, n // 16))
    return synth.hermitian_from(q, lam), lam


def oracle_filter_any_order(H, V, deg, b_sup, mu1, mu_nn):
    order = np.argsort(deg, kind="stable")
    out = np.empty_like(V)
    out[:, order] = oracle.cheb_filter(H, V[:, order], np.asarray(deg)[order], b_sup, mu1, mu_nn)
    return out


def col_rel_err(a, b):
    return np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0))


@pytest.mark.parametrize("n,b", [(300, 37), (517, 70), (129, 1), (64, 64), (1000, 33)])
def test_split_filter_matches_oracle(n, b):
    H, lam = known_h(n, 211 + n)
    V = synth.gaussian_block(n, b, 212 + b)
    rng = np.random.default_rng(n + 3 * b)
    deg = (2 * rng.integers(1, 19, size=b)).astype(np.int32)
    l = lam.numpy()
    b_sup, mu1, mu_nn = 1.02, float(l[0]), float(l[min(n - 1, max(1, n // 8))])
    ref = oracle_filter_any_order(H.numpy(), V.numpy(), deg, b_sup, mu1, mu_nn)
    Vd = dcol(V)
    chase.chase_filter(dcol(H), Vd, deg, b_sup, mu1, mu_nn, precision=chase.CHASE_SPLIT_BF16)
    assert col_rel_err(Vd.cpu().numpy(), ref) <= split_filter_rtol(n, int(deg.max()))


def test_split_filter_full_size_sampled_columns():
    n, b = 8000, 480
    lam = synth.spectrum_dft(n, 221, device=DEV)
    q = synth.unitary_dft(n, 222, device=DEV)
    H = synth.hermitian_from(q, lam)
    del q
    V = synth.gaussian_block(n, b, 223, device=DEV)
    rng = np.random.default_rng(224)
    deg = (2 * rng.integers(1, 19, size=b)).astype(np.int32)
    l = lam.cpu().numpy()
    b_sup, mu1, mu_nn = 50.5, float(l[0]), float(l[b])
    Vin = V.clone()
    chase.chase_filter(H, V, deg, b_sup, mu1, mu_nn, precision=chase.CHASE_SPLIT_BF16)
    cols = [0, 7, 200, 333, 478, 479]
    ref = oracle_filter_any_order(H.cpu().numpy(), Vin[:, cols].cpu().numpy(), deg[cols], b_sup,
                                  mu1, mu_nn)
    assert col_rel_err(V[:, cols].cpu().numpy(), ref) <= split_filter_rtol(n, int(deg.max()))


def test_split_filter_narrow_block_uses_k_segments():
    # 8 columns at N = 4000 give 32 output tiles, so the product is split into
    # K segments whose partial sums are combined in FP64; degrees up to 36
    n, b = 4000, 8
    lam = synth.spectrum_dft(n, 251, device=DEV)
    q = synth.unitary_dft(n, 252, device=DEV)
    H = synth.hermitian_from(q, lam)
    del q
    V = synth.gaussian_block(n, b, 253, device=DEV)
    deg = np.array([36, 2, 20, 36, 8, 12, 36, 4], dtype=np.int32)
    l = lam.cpu().numpy()
    Vin = V.clone()
    chase.chase_filter(H, V, deg, 50.5, float(l[0]), float(l[240]),
                       precision=chase.CHASE_SPLIT_BF16)
    ref = oracle_filter_any_order(H.cpu().numpy(), Vin.cpu().numpy(), deg, 50.5, float(l[0]),
                                  float(l[240]))
    assert col_rel_err(V.cpu().numpy(), ref) <= split_filter_rtol(n, int(deg.max()))


def test_split_filter_beyond_one_launch_exact_range():
    # K = 2N = 45000 exceeds the exact int32 range of one launch (44000), so
    # the product runs as K segments combined in FP64; sampled columns
    n, b = 22500, 32
    lam = synth.spectrum_dft(n, 261, device=DEV)
    H = synth.hermitian_dft(lam, 262)
    V = synth.gaussian_block(n, b, 263, device=DEV)
    deg = np.array([2, 4, 8, 12, 16, 20, 24, 28, 32, 36] * 3 + [36, 2], dtype=np.int32)
    l = lam.cpu().numpy()
    Vin = V.clone()
    chase.chase_filter(H, V, deg, 50.5, float(l[0]), float(l[1350]),
                       precision=chase.CHASE_SPLIT_BF16)
    cols = [0, 9, 17, 31]
    ref = oracle_filter_any_order(H.cpu().numpy(), Vin[:, cols].cpu().numpy(), deg[cols], 50.5,
                                  float(l[0]), float(l[1350]))
    assert col_rel_err(V[:, cols].cpu().numpy(), ref) <= split_filter_rtol(n, int(deg.max()))
    del H, V, Vin
    torch.cuda.empty_cache()


def check_solution(H, lam_true, ritz, resid, V, nev, tol):
    hn = float(np.abs(lam_true).max())
    assert np.max(np.abs(ritz[:nev] - lam_true[:nev])) <= EIG_RTOL * hn
    assert np.all(resid[:nev] <= tol * hn)
    nx = V.shape[1]
    assert np.linalg.norm(V.conj().T @ V - np.eye(nx)) < 1e-12
    r = oracle.residuals(H, V[:, :nev], ritz[:nev])
    assert np.all(r <= tol * hn * 1.05)


def test_split_solve_single_problem_1000():
    n, nev, nex, tol = 1000, 50, 20, 1e-10
    H, lam = known_h(n, 231, n_cluster=60)
    V0 = synth.gaussian_block(n, nev + nex, 232)
    S = synth.gaussian_block(n, 5, 233)
    Vd = dcol(V0)
    o = chase.chase_opts_default(precision=chase.CHASE_SPLIT_BF16)
    st, ritz, resid, stats = chase.chase_solve(dcol(H), nev, nex, tol, Vd, dcol(S), opts=o)
    assert st == chase.CHASE_OK
    check_solution(H.numpy(), lam.numpy(), ritz, resid, Vd.cpu().numpy(), nev, tol)
    ref = oracle.solve(H.numpy(), nev, nex, V0.numpy(), S.numpy(), tol=tol)
    assert np.max(np.abs(ritz[:nev] - ref["ritz"][:nev])) <= EIG_RTOL


def test_split_solve_sequence_matches_fp64():
    n, nev, nex, tol = 600, 24, 8, 1e-10
    lam = synth.spectrum_dft(n, 241)
    q = synth.unitary_qr(n, 242)
    H = synth.hermitian_from(q, lam)
    V0 = synth.gaussian_block(n, nev + nex, 243)
    S = synth.gaussian_block(n, 5, 244)
    out = {}
    for prec in (chase.CHASE_FP64, chase.CHASE_SPLIT_BF16):
        Vd = dcol(V0)
        o = chase.chase_opts_default(precision=prec)
        st, r1, _, _ = chase.chase_solve(dcol(H), nev, nex, tol, Vd, dcol(S), opts=o)
        assert st == chase.CHASE_OK
        E = synth.hermitian_noise(n, 245)
        H2 = (H + 1e-3 * float(lam.abs().max()) * E).t().contiguous().t()
        o2 = chase.chase_opts_default(precision=prec, approx=1)
        st, r2, res2, s2 = chase.chase_solve(dcol(H2), nev, nex, tol, Vd,
                                             dcol(S[:, :1].contiguous()), Lambda=r1, opts=o2)
        assert st == chase.CHASE_OK
        w2 = np.linalg.eigvalsh(H2.numpy())
        check_solution(H2.numpy(), w2, r2, res2, Vd.cpu().numpy(), nev, tol)
        out[prec] = r2
    hn = float(lam.abs().max())
    assert np.max(np.abs(out[chase.CHASE_FP64][:nev] - out[chase.CHASE_SPLIT_BF16][:nev])) \
        <= EIG_RTOL * hn


@pytest.mark.parametrize("n,nev,nex", [(1000, 50, 20), (700, 35, 14)])
def test_split_rr_solve_matches_fp64(n, nev, nex):
    # Rayleigh-Ritz's H Q on the split product as well: same eigenpairs as
    # the FP64 solve, residuals re-checked by the oracle in FP64
    tol = 1e-10
    H, lam = known_h(n, 271 + n, n_cluster=60)
    V0 = synth.gaussian_block(n, nev + nex, 272)
    S = synth.gaussian_block(n, 5, 273)
    out = {}
    for prec in (chase.CHASE_FP64, chase.CHASE_SPLIT_BF16_RR):
        Vd = dcol(V0)
        o = chase.chase_opts_default(precision=prec)
        st, ritz, resid, stats = chase.chase_solve(dcol(H), nev, nex, tol, Vd, dcol(S), opts=o)
        assert st == chase.CHASE_OK
        check_solution(H.numpy(), lam.numpy(), ritz, resid, Vd.cpu().numpy(), nev, tol)
        out[prec] = ritz
    hn = float(lam.abs().max())
    assert np.max(np.abs(out[chase.CHASE_FP64][:nev] - out[chase.CHASE_SPLIT_BF16_RR][:nev])) \
        <= EIG_RTOL * hn


def test_split_rr_batched_solve():
    shapes = [(300, 15, 6), (800, 40, 16), (129, 7, 3)]
    tol = 1e-10
    Hs, lams, Vs, Ss = [], [], [], []
    for k, (n, nev, nex) in enumerate(shapes):
        H, lam = known_h(n, 281 + k)
        Hs.append(dcol(H))
        lams.append(lam.numpy())
        Vs.append(dcol(synth.gaussian_block(n, nev + nex, 282 + k)))
        Ss.append(dcol(synth.gaussian_block(n, 5, 283 + k)))
    o = chase.chase_opts_default(precision=chase.CHASE_SPLIT_BF16_RR)
    st, sts, ritz, res, stats, bst = chase.chase_solve_batched(
        Hs, [s[1] for s in shapes], [s[2] for s in shapes], tol, Vs, Ss, opts=o)
    assert st == chase.CHASE_OK
    for k, (n, nev, nex) in enumerate(shapes):
        check_solution(Hs[k].cpu().numpy(), lams[k], ritz[k], res[k], Vs[k].cpu().numpy(), nev,
                       tol)


# Per filtered column the error is a few hundred times the per-product
# truncation 2^-(7 S) over degrees up to 20 (measured: 2e-6 with 4 slices,
# 2e-4 with 3, 1e-12 with 7); the bound allows 4000 x 2^-(7 S).
@pytest.mark.parametrize("precision,rtol", [(chase.CHASE_SPLIT_BF16_4, reduced_slice_rtol(4)),
                                            (chase.CHASE_SPLIT_BF16_3, reduced_slice_rtol(3))])
@pytest.mark.parametrize("n,b", [(300, 37), (1000, 33)])
def test_reduced_slice_filter_accuracy(precision, rtol, n, b):
    # the leading 4 (3) slices: about 2^-28 (2^-21) relative per product;
    # the FP64 diagonal term is unchanged
    H, lam = known_h(n, 291 + n)
    V = synth.gaussian_block(n, b, 292 + b)
    rng = np.random.default_rng(n + 11 * b)
    deg = (2 * rng.integers(1, 11, size=b)).astype(np.int32)
    l = lam.numpy()
    b_sup, mu1, mu_nn = 1.02, float(l[0]), float(l[min(n - 1, max(1, n // 8))])
    ref = oracle_filter_any_order(H.numpy(), V.numpy(), deg, b_sup, mu1, mu_nn)
    Vd = dcol(V)
    chase.chase_filter(dcol(H), Vd, deg, b_sup, mu1, mu_nn, precision=precision)
    err = col_rel_err(Vd.cpu().numpy(), ref)
    assert err <= rtol
    # and it is a genuinely reduced precision: well above the 7-slice error
    assert err >= 1e-12


@pytest.mark.parametrize("n,nev,nex", [(1000, 50, 20), (700, 35, 14)])
def test_adaptive_slices_solve_matches_fp64(n, nev, nex):
    tol = 1e-10
    H, lam = known_h(n, 301 + n, n_cluster=60)
    V0 = synth.gaussian_block(n, nev + nex, 302)
    S = synth.gaussian_block(n, 5, 303)
    out = {}
    for prec in (chase.CHASE_SPLIT_BF16, chase.CHASE_SPLIT_BF16_ADAPT):
        Vd = dcol(V0)
        o = chase.chase_opts_default(precision=prec)
        st, ritz, resid, stats = chase.chase_solve(dcol(H), nev, nex, tol, Vd, dcol(S), opts=o)
        assert st == chase.CHASE_OK
        check_solution(H.numpy(), lam.numpy(), ritz, resid, Vd.cpu().numpy(), nev, tol)
        out[prec] = (ritz, stats)
    st_ad = out[chase.CHASE_SPLIT_BF16_ADAPT][1]
    assert st_ad["filter_slices_low"] >= 1
    # per column: some products ran on fewer slices, not all of them
    assert 0 < st_ad["filter_matvecs_low"] < st_ad["filter_matvecs"]
    hn = float(lam.abs().max())
    assert np.max(np.abs(out[chase.CHASE_SPLIT_BF16][0][:nev] -
                         out[chase.CHASE_SPLIT_BF16_ADAPT][0][:nev])) <= EIG_RTOL * hn


@pytest.mark.parametrize("n,b", [(1000, 61), (517, 9)])
def test_filter_with_a_precision_per_column(n, b):
    H, lam = known_h(n, 401 + n)
    V = synth.gaussian_block(n, b, 402 + b)
    rng = np.random.default_rng(403 + n)
    deg = (2 * rng.integers(1, 19, size=b)).astype(np.int32)
    ns = rng.choice([3, 4, 7], size=b).astype(np.int32)
    l = lam.numpy()
    b_sup, mu1, mu_nn = 1.02, float(l[0]), float(l[n // 8])
    ref = oracle_filter_any_order(H.numpy(), V.numpy(), deg, b_sup, mu1, mu_nn)
    Vd = dcol(V)
    chase.chase_filter_mixed(dcol(H), Vd, deg, ns, b_sup, mu1, mu_nn)
    got = Vd.cpu().numpy()
    err = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    for a in range(b):
        bound = (split_filter_rtol(n, int(deg.max())) if ns[a] == 7
                 else reduced_slice_rtol(int(ns[a])))
        assert err[a] <= bound, (a, int(ns[a]), float(err[a]))
    # all columns at 7 slices: the uniform split filter's result
    Vm = dcol(V)
    chase.chase_filter_mixed(dcol(H), Vm, deg, np.full(b, 7, np.int32), b_sup, mu1, mu_nn)
    Vu = dcol(V)
    chase.chase_filter(dcol(H), Vu, deg, b_sup, mu1, mu_nn, precision=chase.CHASE_SPLIT_BF16)
    assert col_rel_err(Vm.cpu().numpy(), Vu.cpu().numpy()) <= 1e-12


def test_filter_mixed_rejects_bad_slices():
    H, lam = known_h(64, 411)
    V = dcol(synth.gaussian_block(64, 3, 412))
    l = lam.numpy()
    with pytest.raises(chase.ChaseError) as ei:
        chase.chase_filter_mixed(dcol(H), V, [2, 4, 6], [3, 5, 7], 1.02, float(l[0]), float(l[8]))
    assert ei.value.status == chase.CHASE_INVALID_ARG
