"""GPU parity: every step of the ChASE path through the C ABI against the CPU
oracle on the same seeded inputs (sizes span several tiles and ragged
tails), plus full-size checks on sampled outputs."""

import numpy as np
import pytest
import torch

import oracle
from paper_1805_10121_gb300 import chase, synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
FILTER_RTOL = 1e-11   # filtered block, relative per column (FP64 throughout)
EIG_RTOL = 1e-10      # eigenvalues, relative to ||H||


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1805_10121_gb300 import build
    build.build()
    chase.lib()


def dcol(t):
    """Copy a column-major CPU tensor to the GPU, column-major."""
    return t.to(DEV).t().contiguous().t()


def known_h(n, seed, n_cluster=None, kind="clustered"):
    q = synth.unitary_qr(n, seed)
    if kind == "clustered":
        lam = synth.spectrum_clustered(n, seed + 1, n_cluster=n_cluster or max(2, n // 16))
    else:
        lam = synth.spectrum_uniform(n, seed + 1)
    return synth.hermitian_from(q, lam), lam, q


def oracle_filter_any_order(H, V, deg, b_sup, mu1, mu_nn):
    order = np.argsort(deg, kind="stable")
    out = np.empty_like(V)
    out[:, order] = oracle.cheb_filter(H, V[:, order], np.asarray(deg)[order], b_sup, mu1, mu_nn)
    return out


def col_rel_err(a, b):
    return np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0))


# ------------------------------------------------------------------ filter ---

@pytest.mark.parametrize("n,b", [(300, 37), (64, 64), (129, 1), (517, 70), (5, 3)])
def test_filter_matches_oracle(n, b):
    H, lam, _ = known_h(n, 11 + n)
    V = synth.gaussian_block(n, b, 12 + b)
    rng = np.random.default_rng(n * 7 + b)
    deg = (2 * rng.integers(1, 19, size=b)).astype(np.int32)  # even, 2..36, unsorted
    l = lam.numpy()
    b_sup, mu1, mu_nn = 1.02, float(l[0]), float(l[min(n - 1, max(1, n // 8))])
    ref = oracle_filter_any_order(H.numpy(), V.numpy(), deg, b_sup, mu1, mu_nn)
    Vd = dcol(V)
    chase.chase_filter(dcol(H), Vd, deg, b_sup, mu1, mu_nn)
    assert col_rel_err(Vd.cpu().numpy(), ref) <= FILTER_RTOL


def test_filter_device_degrees_and_workspace():
    n, b = 260, 45
    H, lam, _ = known_h(n, 21)
    V = synth.gaussian_block(n, b, 22)
    deg = np.array([36, 2, 10, 10, 4] * 9, dtype=np.int32)
    l = lam.numpy()
    ref = oracle_filter_any_order(H.numpy(), V.numpy(), deg, 1.01, l[0], l[30])
    Vd = dcol(V)
    work = torch.empty(b, n, dtype=torch.complex128, device=DEV).t()
    chase.chase_filter(dcol(H), Vd, torch.from_numpy(deg).to(DEV), 1.01, l[0], l[30], work=work)
    assert col_rel_err(Vd.cpu().numpy(), ref) <= FILTER_RTOL


def test_filter_host_arrays_match_device():
    n, b = 200, 19
    H, lam, _ = known_h(n, 31)
    V = synth.gaussian_block(n, b, 32)
    deg = [2 * (1 + (j % 9)) for j in range(b)]
    l = lam.numpy()
    Vh = V.clone()
    chase.chase_filter(H, Vh, deg, 1.05, l[0], l[25])
    Vd = dcol(V)
    chase.chase_filter(dcol(H), Vd, deg, 1.05, l[0], l[25])
    assert torch.equal(Vh, Vd.cpu())
    ref = oracle_filter_any_order(H.numpy(), V.numpy(), np.array(deg), 1.05, l[0], l[25])
    assert col_rel_err(Vh.numpy(), ref) <= FILTER_RTOL


def test_filter_diagonal_closed_form():
    # Chebyshev closed form (Eq. 2, Eq. 5) on a diagonal matrix, no oracle
    n, b, m = 150, 8, 24
    d = np.linspace(-1.0, 1.0, n)
    H = torch.diag(torch.from_numpy(d).to(torch.complex128)).t().contiguous().t()
    V = synth.gaussian_block(n, b, 41)
    b_sup, mu1, mu_nn = 1.0, -1.0, -0.7
    c, e = (b_sup + mu_nn) / 2, (b_sup - mu_nn) / 2

    def cm(t):
        t = np.asarray(t, dtype=float)
        out = np.where(np.abs(t) <= 1, np.cos(m * np.arccos(np.clip(t, -1, 1))),
                       np.sign(t) ** m * np.cosh(m * np.arccosh(np.maximum(np.abs(t), 1))))
        return out

    p = cm((d - c) / e) / cm((mu1 - c) / e)
    Vd = dcol(V)
    chase.chase_filter(dcol(H), Vd, [m] * b, b_sup, mu1, mu_nn)
    ref = p[:, None] * V.numpy()
    assert col_rel_err(Vd.cpu().numpy(), ref) <= FILTER_RTOL


def test_filter_rejects_bad_input():
    n = 40
    H, lam, _ = known_h(n, 51)
    Vd = dcol(synth.gaussian_block(n, 3, 52))
    for deg in ([2, 3, 4], [0, 2, 2], [2, 2, 2000]):
        with pytest.raises(chase.ChaseError) as ei:
            chase.chase_filter(dcol(H), Vd, deg, 1.0, -1.0, 0.0)
        assert ei.value.status == chase.CHASE_INVALID_ARG
    with pytest.raises(chase.ChaseError):
        chase.chase_filter(dcol(H), Vd, [2, 2, 2], 1.0, 0.5, 0.0)  # mu1 > mu_nevnex


def test_filter_empty_is_noop():
    n = 16
    H, _, _ = known_h(n, 61)
    V = torch.empty(0, n, dtype=torch.complex128, device=DEV).t()
    chase.chase_filter(dcol(H), V, [], 1.0, -1.0, 0.0)


def test_filter_full_size_sampled_columns():
    # N = 8000, b = 480 (the sequence workload's block), a realistic unsorted
    # degree mix; the oracle recomputes 6 sampled columns one by one (the
    # recurrence is column independent).
    n, b = 8000, 480
    g = synth.generator(71, "cpu")
    lam = synth.spectrum_dft(n, 72, device=DEV)
    q = synth.unitary_dft(n, 73, device=DEV)
    H = synth.hermitian_from(q, lam)
    del q
    V = synth.gaussian_block(n, b, 74, device=DEV)
    rng = np.random.default_rng(75)
    deg = (2 * rng.integers(1, 19, size=b)).astype(np.int32)
    l = lam.cpu().numpy()
    b_sup, mu1, mu_nn = 50.5, float(l[0]), float(l[b])
    Vin = V.clone()
    chase.chase_filter(H, V, deg, b_sup, mu1, mu_nn)
    cols = [0, 1, 123, 250, 401, 479]
    Hh = H.cpu().numpy()
    ref = oracle_filter_any_order(Hh, Vin[:, cols].cpu().numpy(), deg[cols], b_sup, mu1, mu_nn)
    assert col_rel_err(V[:, cols].cpu().numpy(), ref) <= FILTER_RTOL
    del g


# ----------------------------------------------------------------- Lanczos ---

def test_lanczos_matches_oracle():
    n, k, nvec, nev, nex = 400, 25, 4, 20, 8
    H, lam, _ = known_h(n, 81)
    S = synth.gaussian_block(n, 1 + nvec, 82)
    V = synth.gaussian_block(n, nev + nex, 83)
    ref = oracle.lanczos_estimates(H.numpy(), S.numpy(), k, nvec, False, nev, nex,
                                   V=V.numpy(), sigma=0.25)
    Vd = dcol(V)
    got = chase.chase_lanczos(dcol(H), k, nvec, 0, nev, nex, dcol(S), V=Vd)
    hn = float(lam.abs().max())
    assert abs(got["b_sup"] - ref["b_sup"]) <= 1e-10 * hn
    assert abs(got["mu1"] - ref["mu1"]) <= 1e-10 * hn
    assert abs(got["mu_nevnex"] - ref["mu_nevnex"]) <= 1e-10 * hn
    assert got["b_sup"] >= float(lam.max())
    # replaced leading columns equal the oracle's Ritz vectors up to sign
    Vg, Vr = Vd.cpu().numpy(), ref["V"]
    same = np.all(np.abs(Vg - V.numpy()) == 0, axis=0)
    nrep = int(np.argmax(same)) if same.any() else nev + nex
    assert nrep >= 1
    assert np.array_equal(same, np.all(Vr == V.numpy(), axis=0))
    for j in range(nrep):
        ip = abs(np.vdot(Vg[:, j], Vr[:, j]))
        assert abs(ip - 1.0) < 1e-8


def test_lanczos_approx_bound_only():
    n = 300
    H, lam, _ = known_h(n, 91)
    S = synth.gaussian_block(n, 1, 92)
    got = chase.chase_lanczos(dcol(H), 25, 4, 1, 10, 5, dcol(S))
    ref = oracle.lanczos_estimates(H.numpy(), S.numpy(), 25, 4, True, 10, 5)
    assert abs(got["b_sup"] - ref["b_sup"]) <= 1e-10
    assert "mu1" not in got


# ---------------------------------------------------- orthonormalisation ---

def test_orthonormalize_against_locked_matches_householder():
    n, nconv, b = 500, 7, 40
    Y = torch.from_numpy(oracle.householder_qr(synth.gaussian_block(n, nconv, 101).numpy())[0])
    Y = Y.t().contiguous().t()
    V = synth.gaussian_block(n, b, 102)
    Vd = dcol(V)
    chase.chase_orthonormalize(dcol(Y), Vd)
    Q = Vd.cpu().numpy()
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(b)) < 1e-13
    assert np.linalg.norm(Y.numpy().conj().T @ Q) < 1e-13
    Qr = oracle.householder_qr(np.hstack([Y.numpy(), V.numpy()]))[0][:, nconv:]
    M = Q.conj().T @ Qr
    assert np.allclose(np.abs(np.diag(M)), 1.0, atol=1e-10)
    assert np.linalg.norm(M - np.diag(np.diag(M))) < 1e-10


@pytest.mark.parametrize("n,nconv,b", [(700, 0, 100), (900, 33, 97), (300, 5, 32)])
def test_orthonormalize_blocked_panels(n, nconv, b):
    # several 32-wide panels of the blocked Cholesky and triangular solve
    Y = None
    if nconv:
        Y = torch.from_numpy(oracle.householder_qr(synth.gaussian_block(n, nconv, 105).numpy())[0])
        Y = Y.t().contiguous().t()
    scales = torch.logspace(-3, 3, b, dtype=torch.float64).to(torch.complex128)
    V = synth.gaussian_block(n, b, 106) * scales[None, :]
    Vd = dcol(V)
    chase.chase_orthonormalize(dcol(Y) if Y is not None else None, Vd)
    Q = Vd.cpu().numpy()
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(b)) < 1e-13
    full = V.numpy() if Y is None else np.hstack([Y.numpy(), V.numpy()])
    Qr = oracle.householder_qr(full)[0][:, nconv:]
    M = Q.conj().T @ Qr
    assert np.allclose(np.abs(np.diag(M)), 1.0, atol=1e-10)


def test_orthonormalize_ill_conditioned_block():
    # nearly dependent columns force the shifted Cholesky QR path
    n, b = 400, 24
    base = synth.gaussian_block(n, 4, 111).numpy()
    mix = synth.gaussian_block(4, b, 112).numpy()
    V = base @ mix + 1e-9 * synth.gaussian_block(n, b, 113).numpy()
    V = torch.from_numpy(V).t().contiguous().t()
    Vd = dcol(V)
    chase.chase_orthonormalize(None, Vd)
    Q = Vd.cpu().numpy()
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(b)) < 1e-12
    P = V.numpy() - Q @ (Q.conj().T @ V.numpy())
    assert np.linalg.norm(P) <= 1e-8 * np.linalg.norm(V.numpy())


# ---------------------------------------------------- Rayleigh-Ritz, resid ---

def test_rayleigh_ritz_matches_oracle():
    n, b = 300, 20
    H, lam, q = known_h(n, 121, kind="uniform")
    Hn = H.numpy()
    X = q.numpy()[:, :b] + 1e-3 * synth.gaussian_block(n, b, 122).numpy()
    Q = oracle.householder_qr(X)[0]
    Vr, wr = oracle.rayleigh_ritz(Hn, Q)
    rr = oracle.residuals(Hn, Vr, wr)
    Qd = dcol(torch.from_numpy(Q).t().contiguous().t())
    w, r = chase.chase_rayleigh_ritz(dcol(H), Qd)
    hn = float(lam.abs().max())
    assert np.max(np.abs(w - wr)) <= 1e-12 * hn
    assert np.max(np.abs(r - rr)) <= 1e-12 * hn
    Vg = Qd.cpu().numpy()
    for j in range(b):
        assert abs(abs(np.vdot(Vg[:, j], Vr[:, j])) - 1.0) < 1e-8


def test_residuals_match_oracle():
    n, b = 333, 13
    H, _, _ = known_h(n, 131)
    V = synth.gaussian_block(n, b, 132)
    lam = np.linspace(-1, 1, b)
    got = chase.chase_residuals(dcol(H), dcol(V), lam)
    ref = oracle.residuals(H.numpy(), V.numpy(), lam)
    assert np.max(np.abs(got - ref) / ref) < 1e-13


# -------------------------------------------------------------- full solve ---

def check_solution(H, lam_true, ritz, resid, V, nev, tol):
    hn = float(np.abs(lam_true).max())
    assert np.max(np.abs(ritz[:nev] - lam_true[:nev])) <= EIG_RTOL * hn
    assert np.all(resid[:nev] <= tol * hn)
    nx = V.shape[1]
    assert np.linalg.norm(V.conj().T @ V - np.eye(nx)) < 1e-12
    r = oracle.residuals(H, V[:, :nev], ritz[:nev])
    assert np.all(r <= tol * hn * 1.05)


def test_solve_single_problem_1000():
    # the N = 1000 workload: nev 50, nex 20, deg 20, tol 1e-10, random start
    n, nev, nex, tol = 1000, 50, 20, 1e-10
    H, lam, _ = known_h(n, 141, n_cluster=60)
    V0 = synth.gaussian_block(n, nev + nex, 142)
    S = synth.gaussian_block(n, 5, 143)
    Vd = dcol(V0)
    st, ritz, resid, stats = chase.chase_solve(dcol(H), nev, nex, tol, Vd, dcol(S))
    assert st == chase.CHASE_OK
    Hn = H.numpy()
    check_solution(Hn, lam.numpy(), ritz, resid, Vd.cpu().numpy(), nev, tol)
    ref = oracle.solve(Hn, nev, nex, V0.numpy(), S.numpy(), tol=tol)
    assert np.max(np.abs(ritz[:nev] - ref["ritz"][:nev])) <= EIG_RTOL
    assert stats["filter_matvecs"] > 0 and stats["iterations"] >= 1


@pytest.mark.parametrize("precision", [chase.CHASE_FP64, chase.CHASE_SPLIT_BF16])
def test_solve_raised_degree_caps_match_oracle(precision):
    # DEGEXTRA 6 and DEGMAX 64, the caps of the benchmarked split-filter
    # solves: the same eigenpairs as the oracle's solve with the same caps,
    # in the same number of iterations (the degrees follow Alg. 5 exactly)
    n, nev, nex, tol = 1000, 50, 20, 1e-10
    H, lam, _ = known_h(n, 145, n_cluster=60)
    V0 = synth.gaussian_block(n, nev + nex, 146)
    S = synth.gaussian_block(n, 5, 147)
    Vd = dcol(V0)
    o = chase.chase_opts_default(precision=precision, deg_extra=6, deg_max=64)
    st, ritz, resid, stats = chase.chase_solve(dcol(H), nev, nex, tol, Vd, dcol(S), opts=o)
    assert st == chase.CHASE_OK
    Hn = H.numpy()
    check_solution(Hn, lam.numpy(), ritz, resid, Vd.cpu().numpy(), nev, tol)
    ref = oracle.solve(Hn, nev, nex, V0.numpy(), S.numpy(), tol=tol, deg_extra=6, deg_max=64)
    assert ref["converged"]
    assert np.max(np.abs(ritz[:nev] - ref["ritz"][:nev])) <= EIG_RTOL
    assert abs(stats["iterations"] - ref["iterations"]) <= 1


def test_solve_host_arrays_equal_device():
    n, nev, nex, tol = 300, 12, 6, 1e-10
    H, lam, _ = known_h(n, 151)
    V0 = synth.gaussian_block(n, nev + nex, 152)
    S = synth.gaussian_block(n, 5, 153)
    Vh = V0.clone()
    st1, r1, s1, _ = chase.chase_solve(H, nev, nex, tol, Vh, S)
    Vd = dcol(V0)
    st2, r2, s2, _ = chase.chase_solve(dcol(H), nev, nex, tol, Vd, dcol(S))
    assert st1 == st2 == chase.CHASE_OK
    assert np.array_equal(r1, r2) and np.array_equal(s1, s2)
    assert torch.equal(Vh, Vd.cpu())


def test_solve_sequence_warm_start():
    n, nev, nex, tol = 500, 20, 8, 1e-10
    H, lam, _ = known_h(n, 161, n_cluster=30)
    V0 = synth.gaussian_block(n, nev + nex, 162)
    S = synth.gaussian_block(n, 5, 163)
    Vd = dcol(V0)
    st, r1, _, s1 = chase.chase_solve(dcol(H), nev, nex, tol, Vd, dcol(S))
    assert st == chase.CHASE_OK
    E = synth.hermitian_noise(n, 164)
    H2 = H + 1e-3 * float(lam.abs().max()) * E
    H2 = H2.t().contiguous().t()
    o = chase.chase_opts_default(approx=1)
    st, r2, res2, s2 = chase.chase_solve(dcol(H2), nev, nex, tol, Vd, dcol(S[:, :1].contiguous()),
                                         Lambda=r1, opts=o)
    assert st == chase.CHASE_OK
    assert s2["iterations"] < s1["iterations"]
    w2 = np.linalg.eigvalsh(H2.numpy())
    check_solution(H2.numpy(), w2, r2, res2, Vd.cpu().numpy(), nev, tol)


@pytest.mark.parametrize("optim,mode", [(0, chase.CHASE_CONV_REL), (1, chase.CHASE_CONV_ABS)])
def test_solve_options(optim, mode):
    n, nev, nex, tol = 400, 16, 8, 1e-10
    H, lam, _ = known_h(n, 171)
    V0 = synth.gaussian_block(n, nev + nex, 172)
    S = synth.gaussian_block(n, 5, 173)
    Vd = dcol(V0)
    o = chase.chase_opts_default(optim=optim, conv_mode=mode)
    st, ritz, resid, _ = chase.chase_solve(dcol(H), nev, nex, tol, Vd, dcol(S), opts=o)
    assert st == chase.CHASE_OK
    check_solution(H.numpy(), lam.numpy(), ritz, resid, Vd.cpu().numpy(), nev, tol)


def test_solve_max_iter_not_converged():
    n, nev, nex = 200, 10, 4
    H, lam, _ = known_h(n, 181)
    Vd = dcol(synth.gaussian_block(n, nev + nex, 182))
    o = chase.chase_opts_default(max_iter=1)
    st, ritz, resid, stats = chase.chase_solve(dcol(H), nev, nex, 1e-14, Vd,
                                               dcol(synth.gaussian_block(n, 5, 183)), opts=o)
    assert st == chase.CHASE_NOT_CONVERGED
    assert stats["iterations"] == 1
    V = Vd.cpu().numpy()
    assert np.linalg.norm(V.conj().T @ V - np.eye(nev + nex)) < 1e-12
    assert np.all(np.diff(ritz) >= 0)
