"""C ABI checks that need no GPU: the library loads, exports every function
declared in include/chase.h, and its host-side steps (Alg. 5 degrees, Alg. 3
locking, the tridiagonal eigensolve of Alg. 6) agree with the oracle."""

import os

import numpy as np
import pytest

import oracle
from paper_1805_10121_gb300 import chase

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def lib():
    from paper_1805_10121_gb300 import build
    build.build()
    return chase.lib()


def test_exports_every_declared_symbol(lib):
    names = chase.declared_symbols()
    assert "chase_solve" in names and "chase_filter" in names
    for name in names:
        assert hasattr(lib, name), name


def test_opts_default_table1(lib):
    o = chase.chase_opts_default()
    assert (o.deg, o.deg_extra, o.deg_max, o.max_iter, o.lanczos_iter, o.num_lanczos) == \
        (20, 2, 36, 25, 25, 4)
    assert o.approx == 0 and o.dos_sigma == 0.25 and o.optim == 1
    assert o.conv_mode == chase.CHASE_CONV_REL and o.precision == chase.CHASE_FP64


def test_degrees_golden(lib):
    with open(os.path.join(GOLDEN, "degrees_alg5.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            tol, res, lam, c, e, dx, dm, exp = line.split()
            got = chase.chase_degrees([float(res)], [float(lam)], float(c), float(e), float(tol),
                                      int(dx), int(dm))
            assert got[0] == int(exp), line


def test_degrees_match_oracle_random(lib):
    rng = np.random.default_rng(5)
    n = 2000
    ritz = rng.uniform(-3.0, 2.0, n)
    res = 10 ** rng.uniform(-14, 1, n)
    c, e, tol = 0.4, 0.8, 1e-10
    got = chase.chase_degrees(res, ritz, c, e, tol, 2, 36)
    ref = oracle.degrees(res, ritz, c, e, tol, 2, 36)
    assert np.array_equal(got, ref)
    # edge cases: zero / inf / nan residual, Ritz value at the centre
    ed = chase.chase_degrees([0.0, np.inf, np.nan, 1e-3], [-2.0, -2.0, -2.0, c], c, e, tol)
    assert list(ed) == [36, 36, 36, 36]


@pytest.mark.parametrize("deg_extra,deg_max", [(6, 64), (10, 64), (6, 63), (10, 96)])
def test_degrees_match_oracle_raised_caps(lib, deg_extra, deg_max):
    # the split-filter solves raise DEGEXTRA and DEGMAX above Table 1's 2 and
    # 36; an odd cap exercises the even rounding after the clamp (Alg. 5)
    rng = np.random.default_rng(deg_extra * 1000 + deg_max)
    n = 3000
    ritz = rng.uniform(-3.0, 2.0, n)
    res = 10 ** rng.uniform(-14, 1, n)
    c, e, tol = 0.4, 0.8, 1e-10
    got = chase.chase_degrees(res, ritz, c, e, tol, deg_extra, deg_max)
    ref = oracle.degrees(res, ritz, c, e, tol, deg_extra, deg_max)
    assert np.array_equal(got, ref)
    assert np.all(got % 2 == 0) and got.max() <= deg_max
    assert np.any(got > 36)  # the raised cap is reached by some columns


def test_lock_matches_oracle(lib):
    rng = np.random.default_rng(9)
    for _ in range(200):
        b = int(rng.integers(1, 40))
        ritz = np.round(rng.normal(size=b), 1)  # ties exercise stability
        res = 10 ** rng.uniform(-12, -8, b)
        order, n = chase.chase_lock(ritz, res, 1e-10)
        o_ref, n_ref = oracle.deflate_and_lock(ritz, res, 1e-10)
        assert list(order) == list(o_ref) and n == n_ref


def test_tridiag_eigh_against_lapack_and_oracle(lib):
    rng = np.random.default_rng(3)
    for k in (1, 2, 3, 7, 25, 60):
        d = rng.normal(size=k)
        off = np.abs(rng.normal(size=k - 1)) if k > 1 else np.zeros(0)
        w, z = chase.chase_tridiag_eigh(d, off)
        T = np.diag(d) + np.diag(off, 1) + np.diag(off, -1)
        assert np.allclose(w, np.linalg.eigvalsh(T), atol=1e-13 * max(1, np.abs(d).max() + 2))
        assert np.linalg.norm(z.T @ z - np.eye(k)) < 1e-12
        assert np.linalg.norm(T @ z - z * w) < 1e-12 * max(1.0, np.linalg.norm(T))
        wo, zo = oracle.jacobi_eigh(T.astype(np.complex128))
        assert np.allclose(w, wo, atol=1e-12)
        # Eq. 10 weights: squared first components
        assert np.allclose(z[0, :] ** 2, np.abs(zo[0, :]) ** 2, atol=1e-10)


def test_tridiag_eigh_degenerate(lib):
    # zero off-diagonal: already diagonal; repeated eigenvalues
    w, z = chase.chase_tridiag_eigh([3.0, 1.0, 1.0, 2.0], [0.0, 0.0, 0.0])
    assert list(w) == [1.0, 1.0, 2.0, 3.0]
    assert np.allclose(np.abs(z), np.abs(z).round())


def test_invalid_arguments_return_status(lib):
    with pytest.raises(chase.ChaseError) as ei:
        chase.chase_degrees([1.0], [0.0], 0.0, -1.0, 1e-10)
    assert ei.value.status == chase.CHASE_INVALID_ARG
    assert "chase_degrees" in chase.chase_last_error()


def _dos_golden():
    from tests.test_oracle_pins import load_dos_golden
    return load_dos_golden()


def test_dos_estimate_golden(lib):
    # the library's Alg. 6 line 11 (the host step of chase_lanczos) against the
    # hand-worked cases, safeguard branches included
    for name, target, mu1, b_sup, mu, halv, nodes in _dos_golden():
        got, h = chase.chase_dos_estimate(nodes, target, mu1, b_sup, 0.25)
        assert got == pytest.approx(mu, abs=1e-9), name
        assert h == halv, name


def test_dos_estimate_matches_oracle_on_lanczos_runs(lib):
    n, nev, nex = 400, 16, 8
    rng = np.random.default_rng(41)
    lam = np.sort(np.concatenate([rng.uniform(-1, -0.95, 25), rng.uniform(-0.95, 1, n - 25)]))
    q, _ = np.linalg.qr(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    H = (q * lam) @ q.conj().T
    H = 0.5 * (H + H.conj().T)
    starts = (rng.normal(size=(n, 4)) + 1j * rng.normal(size=(n, 4))) / np.sqrt(2)
    runs = [oracle.lanczos_run(H, starts[:, j], 25) for j in range(4)]
    nodes = [(th, np.abs(Z[0, :]) ** 2) for th, Z, _, _ in runs]
    mu1 = min(float(th.min()) for th, _ in nodes)
    b_sup = max(f + float(th.max()) for th, _, f, _ in runs)
    ref = oracle.dos_estimate(nodes, (nev + nex) / n, mu1, b_sup, 0.25)
    got, h = chase.chase_dos_estimate(nodes, (nev + nex) / n, mu1, b_sup, 0.25)
    assert got == pytest.approx(ref["mu"], abs=1e-12 * max(1.0, abs(b_sup)))
    assert h == (-1 if ref["fallback"] else ref["halvings"])


def test_dos_estimate_invalid_arguments(lib):
    with pytest.raises(chase.ChaseError) as ei:
        chase.chase_dos_estimate([([0.0], [1.0])], 1.5, 0.0, 1.0)
    assert ei.value.status == chase.CHASE_INVALID_ARG
    with pytest.raises(chase.ChaseError):
        chase.chase_dos_estimate([([0.0], [1.0])], 0.5, 2.0, 1.0)


def test_wait_selftest_rejects_a_budget_out_of_range(lib):
    # validated before any device work, so this runs without a GPU
    assert chase.chase_wait_selftest(-1) == chase.CHASE_INVALID_ARG
    assert chase.chase_wait_selftest(3_000_000_000) == chase.CHASE_INVALID_ARG
