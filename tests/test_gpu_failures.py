"""Failure detection on the GPU, in forms that fault, trap or hang nothing.

Every failure here is made on the host (a non-finite input, a block with a
zero column, bounds out of order) or by a bounded wait that is meant to run
out (a barrier that nothing arrives at).  Each case must come back as a
status, not a hang, and the library must keep working afterwards in the same
process (the context stays usable)."""

import numpy as np
import pytest
import torch

import oracle
from paper_1805_10121_gb300 import chase, synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1805_10121_gb300 import build
    build.build()
    chase.lib()


def dcol(t):
    return t.to(DEV).t().contiguous().t()


def problem(n, seed):
    q = synth.unitary_qr(n, seed)
    lam = synth.spectrum_clustered(n, seed + 1, n_cluster=max(2, n // 16))
    return synth.hermitian_from(q, lam), lam


def filter_still_works():
    """A small FP64 filter matches the oracle: the context is usable."""
    H, lam = problem(200, 7)
    V = synth.gaussian_block(200, 9, 8)
    deg = np.array([2, 4, 6, 8, 10, 12, 14, 16, 18], dtype=np.int32)
    l = lam.numpy()
    Vd = dcol(V)
    chase.chase_filter(dcol(H), Vd, deg, 1.02, float(l[0]), float(l[20]))
    ref = oracle.cheb_filter(H.numpy(), V.numpy(), deg, 1.02, float(l[0]), float(l[20]))
    err = np.max(np.linalg.norm(Vd.cpu().numpy() - ref, axis=0) / np.linalg.norm(ref, axis=0))
    assert err <= 1e-11


def test_bounded_wait_gives_up_with_timeout_status():
    # one second at most: 2e6 cycles is about a millisecond at 2 GHz
    st = chase.chase_wait_selftest(2_000_000)
    assert st == chase.CHASE_TIMEOUT
    assert "bounded wait" in chase.chase_last_error()
    filter_still_works()
    # a second run behaves the same (the error flag is per call)
    assert chase.chase_wait_selftest(0) == chase.CHASE_TIMEOUT
    filter_still_works()


@pytest.mark.parametrize("where", ["H", "V", "lanczos_starts"])
@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_non_finite_solve_input_is_rejected(where, bad):
    n, nev, nex = 160, 6, 4
    H, lam = problem(n, 31)
    V = synth.gaussian_block(n, nev + nex, 32)
    S = synth.gaussian_block(n, 5, 33)
    arrays = {"H": H.clone(), "V": V.clone(), "lanczos_starts": S.clone()}
    a = arrays[where]
    a[17, 3] = complex(bad, 0.0)
    if where == "H":
        a[3, 17] = complex(bad, 0.0)  # keep it Hermitian in shape
    with pytest.raises(chase.ChaseError) as ei:
        chase.chase_solve(dcol(arrays["H"]), nev, nex, 1e-10, dcol(arrays["V"]),
                          dcol(arrays["lanczos_starts"]))
    assert ei.value.status == chase.CHASE_INVALID_ARG
    assert where in chase.chase_last_error() and "non-finite" in chase.chase_last_error()
    # the same process solves the clean problem
    st, ritz, res, _ = chase.chase_solve(dcol(H), nev, nex, 1e-10, dcol(V), dcol(S))
    assert st == chase.CHASE_OK
    assert np.max(np.abs(ritz[:nev] - lam.numpy()[:nev])) <= 1e-10


def test_non_finite_filter_block_is_rejected():
    H, lam = problem(200, 41)
    V = synth.gaussian_block(200, 12, 42)
    V[5, 7] = complex(0.0, float("nan"))
    l = lam.numpy()
    for prec in (chase.CHASE_FP64, chase.CHASE_SPLIT_BF16):
        with pytest.raises(chase.ChaseError) as ei:
            chase.chase_filter(dcol(H), dcol(V), [4] * 12, 1.02, float(l[0]), float(l[20]),
                               precision=prec)
        assert ei.value.status == chase.CHASE_INVALID_ARG
    filter_still_works()


def test_zero_column_breaks_the_qr_down():
    # A zero column defeats Cholesky QR and its shifted retry (the shift keeps
    # the column at zero), so the orthonormalisation reports a breakdown
    # (Sec. 4.1.3: rank deficiency of the filtered block).
    n, b = 300, 16
    V = synth.gaussian_block(n, b, 51)
    V[:, 5] = 0
    with pytest.raises(chase.ChaseError) as ei:
        chase.chase_orthonormalize(None, dcol(V))
    assert ei.value.status == chase.CHASE_QR_BREAKDOWN
    W = dcol(synth.gaussian_block(n, b, 52))
    chase.chase_orthonormalize(None, W)
    Wh = W.cpu().numpy()
    assert np.linalg.norm(Wh.conj().T @ Wh - np.eye(b)) < 1e-12


def test_warm_start_values_above_the_upper_bound():
    # approx = 1 takes mu_1 and mu_nev+nex from the caller's Lambda; values
    # above the Lanczos upper bound b_sup leave mu_nev+nex >= b_sup, which
    # Alg. 4's interval cannot use: the solve stops with a bound violation.
    n, nev, nex = 200, 6, 4
    H, lam = problem(n, 61)
    V = synth.gaussian_block(n, nev + nex, 62)
    S = synth.gaussian_block(n, 1, 63)
    Lam = np.linspace(-1.0, 5.0, nev + nex)  # the spectrum ends at 1
    o = chase.chase_opts_default(approx=1)
    with pytest.raises(chase.ChaseError) as ei:
        chase.chase_solve(dcol(H), nev, nex, 1e-10, dcol(V), dcol(S), Lambda=Lam, opts=o)
    assert ei.value.status == chase.CHASE_BOUND_VIOLATION
    Lam[3] = float("nan")
    with pytest.raises(chase.ChaseError) as ei:
        chase.chase_solve(dcol(H), nev, nex, 1e-10, dcol(V), dcol(S), Lambda=Lam, opts=o)
    assert ei.value.status == chase.CHASE_INVALID_ARG


def test_filter_bounds_out_of_order():
    H, lam = problem(100, 71)
    V = dcol(synth.gaussian_block(100, 4, 72))
    for b_sup, mu1, mu_nn in ((0.5, -1.0, 0.7), (1.0, 0.2, 0.1), (float("nan"), -1.0, 0.0)):
        with pytest.raises(chase.ChaseError) as ei:
            chase.chase_filter(dcol(H), V, [2, 2, 2, 2], b_sup, mu1, mu_nn)
        assert ei.value.status == chase.CHASE_INVALID_ARG
    filter_still_works()
