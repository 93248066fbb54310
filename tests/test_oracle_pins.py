"""Pins of the CPU oracle against facts that the paper and the mathematics fix
(closed forms, hand-worked values, library routines on special cases,
invariants).  CPU only."""

import math
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1805_10121_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cheb_closed(mdeg, t):
    """C_m(t) by Eq. 2: cosh(m acosh t) for t >= 1, cos(m acos t) on [-1, 1],
    (-1)^m cosh(m acosh |t|) for t <= -1."""
    t = np.asarray(t, dtype=np.float64)
    out = np.empty_like(t)
    inside = np.abs(t) <= 1.0
    out[inside] = np.cos(mdeg * np.arccos(t[inside]))
    up = t > 1.0
    out[up] = np.cosh(mdeg * np.arccosh(t[up]))
    dn = t < -1.0
    out[dn] = (-1.0) ** mdeg * np.cosh(mdeg * np.arccosh(-t[dn]))
    return out


def p_m(mdeg, x, b_sup, mu1, mu_nn):
    """The normalised filter polynomial of Eq. 5 with gamma = mu_1,
    [alpha, beta] = [mu_nev+nex, b_sup]."""
    c = (b_sup + mu_nn) / 2.0
    e = (b_sup - mu_nn) / 2.0
    return cheb_closed(mdeg, (np.asarray(x) - c) / e) / cheb_closed(mdeg, np.array([(mu1 - c) / e]))[0]


def rand_block(n, b, seed):
    return synth.gaussian_block(n, b, seed).numpy()


# ---------------------------------------------------------------- filter ---

@pytest.mark.parametrize("mdeg", [2, 4, 10, 20, 36])
def test_filter_diagonal_closed_form(mdeg):
    rng = np.random.default_rng(1)
    n, b = 64, 5
    d = np.sort(rng.uniform(-1.0, 1.0, n))
    H = np.diag(d).astype(np.complex128)
    V = rand_block(n, b, 2)
    b_sup, mu1, mu_nn = 1.05, -1.0, -0.6
    out = oracle.cheb_filter(H, V, [mdeg] * b, b_sup, mu1, mu_nn)
    ref = p_m(mdeg, d, b_sup, mu1, mu_nn)[:, None] * V
    err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    assert err < 1e-12


def test_filter_known_eigenbasis_per_column_degrees():
    n, b = 80, 7
    q = synth.unitary_qr(n, 3).numpy()
    lam = synth.spectrum_clustered(n, 4, n_cluster=6).numpy()
    H = (q * lam[None, :]) @ q.conj().T
    H = 0.5 * (H + H.conj().T)
    V = rand_block(n, b, 5)
    m = [2, 2, 4, 8, 8, 14, 20]
    b_sup, mu1, mu_nn = 1.02, lam[0], lam[b + 2]
    out = oracle.cheb_filter(H, V, m, b_sup, mu1, mu_nn)
    for a in range(b):
        ref = q @ (p_m(m[a], lam, b_sup, mu1, mu_nn) * (q.conj().T @ V[:, a]))
        assert np.linalg.norm(out[:, a] - ref) <= 1e-11 * np.linalg.norm(ref)


def test_filter_normalisation_at_mu1():
    # p_m(mu_1) = 1 (Eq. 5 normalisation): an eigenvector at mu_1 is unchanged
    n = 40
    d = np.linspace(-1.0, 1.0, n)
    H = np.diag(d).astype(np.complex128)
    V = np.zeros((n, 1), dtype=np.complex128)
    V[0, 0] = 1.0 + 0.5j
    out = oracle.cheb_filter(H, V, [16], 1.0, d[0], d[5])
    assert abs(out[0, 0] - V[0, 0]) < 1e-12
    assert np.linalg.norm(out[1:, 0]) == 0.0


def test_filter_matvec_count_is_sum_of_degrees():
    # a column leaves the products once it reaches its degree (Alg. 4 lines
    # 12-14), so the number of column products is exactly sum(m_a)
    n = 30
    H = np.diag(np.linspace(-1, 1, n)).astype(np.complex128)
    V = rand_block(n, 6, 3)
    for m in ([2] * 6, [2, 4, 4, 6, 10, 10], [8] * 6, [2, 2, 2, 2, 2, 36]):
        st = {}
        oracle.cheb_filter(H, V, m, 1.0, -1.0, -0.5, stats=st)
        assert st["matvecs"] == sum(m)


def test_filter_rejects_unsorted_or_odd():
    H = np.eye(4, dtype=np.complex128)
    V = np.ones((4, 2), dtype=np.complex128)
    with pytest.raises(ValueError):
        oracle.cheb_filter(H, V, [4, 2], 1.0, -1.0, 0.0)
    with pytest.raises(ValueError):
        oracle.cheb_filter(H, V, [3, 4], 1.0, -1.0, 0.0)


def test_filter_convergence_rate_eq6():
    # Eq. 6: the damped components shrink like |rho|^-m relative to mu_1's
    n = 30
    d = np.linspace(-1.0, 1.0, n)
    H = np.diag(d).astype(np.complex128)
    V = np.ones((n, 1), dtype=np.complex128)
    b_sup, mu1, mu_nn = 1.0, -1.0, -0.5
    c, e = (b_sup + mu_nn) / 2, (b_sup - mu_nn) / 2
    t = (mu1 - c) / e
    rho = abs(t) + math.sqrt(t * t - 1)
    out = oracle.cheb_filter(H, V, [30], b_sup, mu1, mu_nn)
    inside = np.abs((d - c) / e) <= 1.0
    # inside the damped interval |C_m| <= 1, so |p_m| <= 1/C_m(t(mu1)) ~ 2 rho^-m
    assert np.max(np.abs(out[inside, 0])) <= 2.0 * rho ** -30 * (1 + 1e-9)


# --------------------------------------------------------------- degrees ---

def load_degree_cases():
    rows = []
    with open(os.path.join(GOLDEN, "degrees_alg5.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tol, res, lam, c, e, dx, dm, exp = line.split()
            rows.append((float(tol), float(res), float(lam), float(c), float(e),
                         int(dx), int(dm), int(exp)))
    return rows


@pytest.mark.parametrize("case", load_degree_cases())
def test_degrees_golden(case):
    tol, res, lam, c, e, dx, dm, exp = case
    assert oracle.degree_one(tol, res, lam, c, e, dx, dm) == exp


def test_degrees_eq8_meets_tolerance():
    # Eq. 8: Res / |rho|^m <= tol for the returned degree (when below DEGMAX)
    rng = np.random.default_rng(7)
    for _ in range(200):
        c, e = 0.3, 0.7
        lam = rng.uniform(-3.0, -1.01)
        res = 10 ** rng.uniform(-9, -2)
        tol = 1e-10
        deg = oracle.degree_one(tol, res, lam, c, e, 0, 1000)
        t = (lam - c) / e
        rho = abs(t) + math.sqrt(t * t - 1)
        assert deg % 2 == 0
        assert res / rho ** deg <= tol * (1 + 1e-12)
        assert res / rho ** max(deg - 2, 0) > tol * (1 - 1e-12) or deg <= 2


# ------------------------------------------------------------ eigensolver ---

@pytest.mark.parametrize("n", [1, 2, 3, 8, 33])
def test_jacobi_matches_lapack(n):
    rng = np.random.default_rng(n)
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    G = a + a.conj().T
    w, Z = oracle.jacobi_eigh(G)
    wl = np.linalg.eigvalsh(G)
    assert np.allclose(w, wl, rtol=0, atol=1e-12 * max(1.0, np.abs(wl).max()))
    assert np.linalg.norm(Z.conj().T @ Z - np.eye(n)) < 1e-12
    assert np.linalg.norm(G @ Z - Z * w[None, :]) < 1e-11 * np.linalg.norm(G)


def test_jacobi_2x2_closed_form():
    a, d, b = 0.3, -1.2, 0.7 - 0.4j
    G = np.array([[a, b], [np.conj(b), d]])
    w, _ = oracle.jacobi_eigh(G)
    mid, rad = (a + d) / 2, math.sqrt(((a - d) / 2) ** 2 + abs(b) ** 2)
    assert np.allclose(w, [mid - rad, mid + rad], atol=1e-15)


def test_jacobi_known_spectrum():
    n = 24
    q = synth.unitary_qr(n, 11).numpy()
    lam = np.linspace(-2.0, 3.0, n)
    G = (q * lam) @ q.conj().T
    w, _ = oracle.jacobi_eigh(0.5 * (G + G.conj().T))
    assert np.max(np.abs(w - lam)) < 1e-13


# --------------------------------------------------------------------- QR ---

@pytest.mark.parametrize("shape", [(10, 1), (50, 7), (64, 64), (200, 30)])
def test_householder_qr(shape):
    n, b = shape
    X = rand_block(n, b, 9)
    Q, R = oracle.householder_qr(X)
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(b)) < 1e-13
    assert np.linalg.norm(Q @ R - X) < 1e-13 * np.linalg.norm(X)
    assert np.allclose(np.tril(R, -1), 0)
    Ql, _ = np.linalg.qr(X)
    # same column spaces, column by column, up to a unit phase
    assert np.allclose(np.abs(np.diag(Ql.conj().T @ Q)), 1.0, atol=1e-12)


def test_householder_qr_near_unit_columns():
    # columns already close to e_j: the reflector must not cancel (the sign of
    # alpha is chosen against x_1)
    n, b = 40, 6
    X = np.eye(n, b, dtype=np.complex128) * (1.0 + 0.5j) + 1e-9 * rand_block(n, b, 5)
    Q, R = oracle.householder_qr(X)
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(b)) < 1e-13
    assert np.linalg.norm(Q @ R - X) < 1e-14 * np.linalg.norm(X)


# ------------------------------------------------- RR, residuals, locking ---

def test_rayleigh_ritz_exact_subspace():
    n, b = 60, 6
    q = synth.unitary_qr(n, 21).numpy()
    lam = np.linspace(-1, 1, n)
    H = (q * lam) @ q.conj().T
    H = 0.5 * (H + H.conj().T)
    # a basis of the invariant subspace of the 6 lowest eigenvalues, mixed
    mix = np.linalg.qr(rand_block(b, b, 22))[0]
    Qs = q[:, :b] @ mix
    V, w = oracle.rayleigh_ritz(H, Qs)
    assert np.max(np.abs(w - lam[:b])) < 1e-13
    assert np.max(oracle.residuals(H, V, w)) < 1e-13


def test_residuals_definition():
    H = np.diag([1.0, 2.0, 3.0]).astype(np.complex128)
    V = np.array([[1, 0], [0, 0.6], [0, 0.8]], dtype=np.complex128)
    r = oracle.residuals(H, V, [1.0, 2.0])
    assert abs(r[0]) < 1e-16
    assert abs(r[1] - 0.8) < 1e-15  # ||(0, 1.2, 2.4) - 2 (0, .6, .8)|| = ||(0,0,0.8)||


def test_lock_prefix_rule():
    ritz = np.array([0.5, -1.0, 0.1, -0.5, 0.2])
    res = np.array([1e-12, 1e-12, 1e-3, 1e-11, 1e-12])
    order, n_new = oracle.deflate_and_lock(ritz, res, 1e-10)
    assert list(order) == [1, 3, 2, 4, 0]
    assert n_new == 2  # -1.0, -0.5 lock; 0.1 stops the run though 0.2, 0.5 converged
    order, n_new = oracle.deflate_and_lock(ritz, res, 1e-2)
    assert n_new == 5
    # ties keep the input order (stable sort)
    order, _ = oracle.deflate_and_lock(np.array([1.0, 1.0, 0.0]), np.zeros(3), 1.0)
    assert list(order) == [2, 0, 1]
    # boundary: Res == tol locks (Alg. 3 line 4 returns only on Res > tol)
    _, n_new = oracle.deflate_and_lock(np.array([0.0]), np.array([1e-10]), 1e-10)
    assert n_new == 1


# ---------------------------------------------------------------- Lanczos ---

def test_lanczos_relation_and_bound():
    n, k = 120, 25
    q = synth.unitary_qr(n, 31).numpy()
    lam = synth.spectrum_clustered(n, 32, n_cluster=8).numpy()
    H = (q * lam) @ q.conj().T
    H = 0.5 * (H + H.conj().T)
    v0 = rand_block(n, 1, 33)[:, 0]
    theta, Z, fnorm, U = oracle.lanczos_run(H, v0, k)
    # U^H A U = T_k up to rounding for a short run
    T = U.conj().T @ H @ U
    assert np.allclose(np.triu(T, 2), 0, atol=1e-8)
    w = np.linalg.eigvalsh(0.5 * (T + T.conj().T))
    assert np.allclose(np.sort(w), theta, atol=1e-8)
    # Ritz values inside the spectrum; b_sup bounds lambda_max (Sec. 4.2)
    assert theta.min() >= lam.min() - 1e-12 and theta.max() <= lam.max() + 1e-12
    assert fnorm + theta.max() >= lam.max()
    # weights |Z_1i|^2 sum to one
    assert abs(np.sum(np.abs(Z[0, :]) ** 2) - 1.0) < 1e-12


def test_lanczos_estimates_bound_and_mu1():
    n, k = 200, 6
    H, lam, _ = known_problem(n, 35, 10)
    starts = rand_block(n, 5, 36)
    est = oracle.lanczos_estimates(H, starts, k, 4, True, 10, 5)
    theta0, _, f0, _ = oracle.lanczos_run(H, starts[:, 0], k)
    # Alg. 6 line 3 with a short run: max theta alone is below lambda_max
    assert theta0.max() < lam.max()
    assert est["b_sup"] == f0 + theta0.max()
    assert est["b_sup"] >= lam.max()
    est = oracle.lanczos_estimates(H, starts, k, 4, False, 10, 5, V=rand_block(n, 15, 37))
    mins = [oracle.lanczos_run(H, starts[:, 1 + j], k)[0].min() for j in range(4)]
    assert est["mu1"] == min(mins) and min(mins) < max(mins)
    assert est["mu1"] >= lam.min() - 1e-12
    assert est["b_sup"] >= lam.max()
    assert lam.min() <= est["mu_nevnex"] <= lam.max()


def test_lanczos_invariant_subspace_breakdown():
    H = np.diag([-2.0, 1.0, 5.0, 7.0]).astype(np.complex128)
    v0 = np.array([1.0, 1.0, 0.0, 0.0], dtype=np.complex128)
    theta, Z, fnorm, U = oracle.lanczos_run(H, v0, 4)
    assert np.allclose(theta, [-2.0, 1.0])
    assert fnorm <= 1e-13 * 7.0
    assert np.allclose(np.abs(Z[0, :]) ** 2, [0.5, 0.5])


def test_dos_single_cluster_closed_form():
    # H = lambda0 I: every run stops after one step with theta = lambda0 and
    # weight 1, so the integral of Eq. 10 is Phi((t - lambda0)/sigma) and its
    # quantile is lambda0 + sigma Phi^-1(target).
    from scipy.stats import norm
    n, nev, nex = 50, 3, 2
    lam0 = 0.7
    H = lam0 * np.eye(n, dtype=np.complex128)
    starts = rand_block(n, 5, 41)
    runs = [oracle.lanczos_run(H, starts[:, 1 + j], 10) for j in range(4)]
    assert all(len(th) == 1 and abs(th[0] - lam0) < 1e-14 for th, _, _, _ in runs)
    nodes = [(th, np.abs(Z[0, :]) ** 2) for th, Z, _, _ in runs]
    for sig in (0.25, 0.05):
        q = oracle.dos_quantile(nodes, (nev + nex) / n, sig)
        assert abs(q - (lam0 + sig * norm.ppf((nev + nex) / n))) < 1e-9
    # the estimate itself must stay inside (mu_1, b_sup); with a collapsed
    # spectrum the interval is empty and the uniform fallback returns mu_1
    est = oracle.lanczos_estimates(H, starts, 10, 4, False, nev, nex, V=None, sigma=0.25)
    assert abs(est["b_sup"] - lam0) < 1e-14 and abs(est["mu1"] - lam0) < 1e-14


def test_dos_estimate_kept_inside_interval():
    # a band holding the lowest 6 % of the spectrum: with the width of Eq. 10
    # measured on [mu_1, b_sup] the raw quantile falls below mu_1; the
    # estimate must still land strictly between mu_1 and b_sup
    n, nev, nex = 400, 16, 8
    H, lam, _ = known_problem(n, 171, 25)
    starts = rand_block(n, 5, 173)
    est = oracle.lanczos_estimates(H, starts, 25, 4, False, nev, nex, V=None, sigma=0.25)
    runs = [oracle.lanczos_run(H, starts[:, 1 + j], 25) for j in range(4)]
    nodes = [(th, np.abs(Z[0, :]) ** 2) for th, Z, _, _ in runs]
    raw = oracle.dos_quantile(nodes, (nev + nex) / n, 0.25 * (est["b_sup"] - est["mu1"]) / 2)
    assert raw < est["mu1"]
    assert est["mu1"] < est["mu_nevnex"] < est["b_sup"]
    assert lam[0] <= est["mu_nevnex"] <= lam[nev + nex + 40]


def load_dos_golden():
    """Cases of tests/golden/dos_safeguard.txt: (name, target, mu1, b_sup,
    expected mu, expected halvings, nodes)."""
    cases = []
    with open(os.path.join(GOLDEN, "dos_safeguard.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, target, mu1, b_sup, mu, halv, runs = line.split()
            nodes = []
            for run in runs.split("|"):
                th, w = run.split(":")
                nodes.append((np.array([float(x) for x in th.split(",")]),
                              np.array([float(x) for x in w.split(",")])))
            cases.append((name, float(target), float(mu1), float(b_sup), float(mu), int(halv),
                          nodes))
    return cases


@pytest.mark.parametrize("case", load_dos_golden(), ids=lambda c: c[0])
def test_dos_safeguard_golden(case):
    # hand-worked values of Alg. 6 line 11 with the width safeguard (Sec. 4.2)
    name, target, mu1, b_sup, mu, halv, nodes = case
    got = oracle.dos_estimate(nodes, target, mu1, b_sup, sigma=0.25)
    assert got["mu"] == pytest.approx(mu, abs=1e-9), name
    if halv < 0:
        assert got["fallback"] and got["halvings"] == 40
    else:
        assert not got["fallback"] and got["halvings"] == halv


def test_dos_safeguard_golden_file_covers_each_branch():
    halvings = sorted({c[5] for c in load_dos_golden()})
    assert halvings == [-1, 0, 1, 2]


def test_dos_two_clusters_quantile():
    # two eigenvalues with multiplicity: the Krylov space is 2-dimensional,
    # theta = {a, b}, weights = the start vector's mass on each eigenspace.
    from scipy.stats import norm
    from scipy.optimize import brentq
    n = 40
    d = np.array([-1.0] * 10 + [1.0] * 30)
    H = np.diag(d).astype(np.complex128)
    starts = rand_block(n, 5, 51)
    nev, nex = 6, 2
    est = oracle.lanczos_estimates(H, starts, 6, 4, False, nev, nex, V=None, sigma=0.25)
    sig = 0.25 * (est["b_sup"] - est["mu1"]) / 2.0
    ws = []
    for j in range(4):
        v = starts[:, 1 + j]
        ws.append(np.sum(np.abs(v[:10]) ** 2) / np.sum(np.abs(v) ** 2))
    f = lambda t: np.mean([w * norm.cdf((t + 1) / sig) + (1 - w) * norm.cdf((t - 1) / sig)
                           for w in ws]) - (nev + nex) / n
    assert abs(est["mu_nevnex"] - brentq(f, -5, 5)) < 1e-9


# --------------------------------------------------------------- inputs ---

def test_hermitian_dft_equals_dense_construction():
    # the FFT construction of Q diag(lam) Q^H equals the dense product
    n = 96
    lam = synth.spectrum_dft(n, 5)
    dense = synth.hermitian_from(synth.unitary_dft(n, 6), lam).numpy()
    fast = synth.hermitian_dft(lam, 6).numpy()
    assert np.linalg.norm(dense - fast) <= 1e-13 * np.linalg.norm(dense)
    assert np.allclose(np.linalg.eigvalsh(fast), lam.numpy(), atol=1e-12 * 50)
    assert np.array_equal(fast, fast.conj().T)


# ------------------------------------------------------------- full solve ---

def known_problem(n, seed, n_cluster):
    q = synth.unitary_qr(n, seed).numpy()
    lam = synth.spectrum_clustered(n, seed + 1, n_cluster=n_cluster).numpy()
    H = (q * lam) @ q.conj().T
    return 0.5 * (H + H.conj().T), lam, q


@pytest.mark.parametrize("optim", [True, False])
def test_solve_known_spectrum(optim):
    n, nev, nex, tol = 150, 10, 6, 1e-10
    H, lam, q = known_problem(n, 61, 12)
    V0 = rand_block(n, nev + nex, 62)
    starts = rand_block(n, 5, 63)
    out = oracle.solve(H, nev, nex, V0, starts, tol=tol, optim=optim)
    assert out["converged"]
    hnorm = np.abs(lam).max()
    assert np.max(np.abs(out["ritz"][:nev] - lam[:nev])) <= 1e-10 * hnorm
    assert np.all(out["resid"][:nev] <= tol * hnorm)
    V = out["V"]
    assert np.linalg.norm(V.conj().T @ V - np.eye(nev + nex)) <= 1e-12
    r = oracle.residuals(H, V[:, :nev], out["ritz"][:nev])
    assert np.all(r <= tol * hnorm * 1.01)


def test_solve_warm_start_fewer_iterations():
    n, nev, nex, tol = 150, 10, 6, 1e-10
    H, lam, q = known_problem(n, 71, 12)
    V0 = rand_block(n, nev + nex, 72)
    starts = rand_block(n, 5, 73)
    first = oracle.solve(H, nev, nex, V0, starts, tol=tol)
    E = synth.hermitian_noise(n, 74).numpy()
    H2 = H + 1e-3 * np.abs(lam).max() * E
    second = oracle.solve(H2, nev, nex, first["V"], starts, tol=tol, Lam=first["ritz"],
                          approx=True)
    assert second["converged"]
    assert second["iterations"] < first["iterations"]
    w2 = np.linalg.eigvalsh(H2)
    assert np.max(np.abs(second["ritz"][:nev] - w2[:nev])) <= 1e-10 * np.abs(w2).max()


def test_solve_max_iter_returns_partial():
    n, nev, nex = 100, 8, 4
    H, lam, q = known_problem(n, 81, 10)
    out = oracle.solve(H, nev, nex, rand_block(n, nev + nex, 82), rand_block(n, 5, 83),
                       tol=1e-14, max_iter=1)
    assert out["iterations"] == 1
    assert not out["converged"]
    assert out["V"].shape == (n, nev + nex)


# ------------------------------------------------------- small helpers ---

def test_filter_bounds_hand_values():
    # Alg. 4 lines 2-3 with b_sup = 3, mu_nev+nex = 1, mu_1 = -1:
    # c = 2, e = 1, sigma_1 = e / (mu_1 - c) = -1/3
    c, e, s1 = oracle.filter_bounds(3.0, -1.0, 1.0)
    assert (c, e) == (2.0, 1.0)
    assert s1 == pytest.approx(-1.0 / 3.0, abs=1e-15)


def test_shifted_apply_is_h_minus_c_identity():
    rng = np.random.default_rng(5)
    n, b = 7, 3
    H = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    X = rng.standard_normal((n, b)) + 1j * rng.standard_normal((n, b))
    out = oracle.shifted_apply(H, X, 0.75)
    assert np.allclose(out, (H - 0.75 * np.eye(n)) @ X, rtol=0, atol=1e-13)


def test_degrees_is_degree_one_per_column():
    rng = np.random.default_rng(9)
    res = 10.0 ** rng.uniform(-12, 0, 20)
    ritz = rng.uniform(-2.0, 0.4, 20)
    c, e, tol = 0.5, 0.5, 1e-10
    got = oracle.degrees(res, ritz, c, e, tol)
    ref = [oracle.degree_one(tol, r, l, c, e, 2, 36) for r, l in zip(res, ritz)]
    assert list(got) == ref
    assert all(d % 2 == 0 and 2 <= d <= 36 for d in got)


def test_dos_cdf_single_node_is_the_normal_cdf():
    # one run, one Ritz value at 0 with unit weight: the integral of Eq. 10
    # is the Gaussian CDF Phi(t / sigma)
    nodes = [(np.array([0.0]), np.array([1.0]))]
    for t, ref in ((0.0, 0.5), (0.25, 0.5 * (1 + math.erf(1.0 / math.sqrt(2)))),
                   (-0.5, 0.5 * (1 + math.erf(-2.0 / math.sqrt(2))))):
        assert oracle.dos_cdf(nodes, t, 0.25) == pytest.approx(ref, abs=1e-15)
    # two runs are averaged; weights summing to one give a CDF from 0 to 1
    nodes2 = [(np.array([-1.0, 1.0]), np.array([0.5, 0.5])), (np.array([0.0]), np.array([1.0]))]
    assert oracle.dos_cdf(nodes2, -50.0, 0.1) == pytest.approx(0.0, abs=1e-15)
    assert oracle.dos_cdf(nodes2, 50.0, 0.1) == pytest.approx(1.0, abs=1e-15)
    assert oracle.dos_cdf(nodes2, 0.0, 0.1) == pytest.approx(0.5, abs=1e-12)
