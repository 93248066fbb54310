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
