"""Solver modes of Table 1 beyond the defaults, on the GPU against the
oracle: the constant-degree filter (optim = false, Alg. 1 line 1 degree for
every column in every iteration) and odd initial degrees (rounded up to
even, Sec. 4.1.3)."""

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


@pytest.mark.parametrize("precision", [chase.CHASE_FP64, chase.CHASE_SPLIT_BF16])
@pytest.mark.parametrize("deg", [8, 13, 24])
def test_constant_degree_mode(precision, deg):
    n, nev, nex, tol = 600, 30, 12, 1e-10
    q = synth.unitary_qr(n, 901)
    lam = synth.spectrum_clustered(n, 902, n_cluster=40)
    H = synth.hermitian_from(q, lam)
    V0 = synth.gaussian_block(n, nev + nex, 903)
    S = synth.gaussian_block(n, 5, 904)
    Vd = dcol(V0)
    o = chase.chase_opts_default(precision=precision, optim=0, deg=deg)
    st, ritz, res, stats = chase.chase_solve(dcol(H), nev, nex, tol, Vd, dcol(S), opts=o)
    assert st == chase.CHASE_OK
    d0 = deg + deg % 2
    # every filtered column ran exactly d0 products in every iteration
    assert stats["filter_matvecs"] % d0 == 0
    hn = float(lam.abs().max())
    l = lam.numpy()
    assert np.max(np.abs(ritz[:nev] - l[:nev])) <= 1e-10 * hn
    assert np.all(res[:nev] <= tol * hn)
    ref = oracle.solve(H.numpy(), nev, nex, V0.numpy(), S.numpy(), tol=tol, deg=deg, optim=False)
    assert np.max(np.abs(ritz[:nev] - ref["ritz"][:nev])) <= 1e-10 * hn


@pytest.mark.parametrize("real", [False, True])
def test_lower_storage_reads_only_the_lower_triangle(real):
    # the strict upper triangle holds NaN: with CHASE_STORAGE_LOWER the solve
    # must not read it, and must match the full-storage solve
    n, nev, nex, tol = 500, 24, 10, 1e-10
    if real:
        q = synth.orthogonal_qr(n, 921)
        lam = synth.spectrum_clustered(n, 922, n_cluster=30)
        H = synth.symmetric_from(q, lam)
        V0 = synth.gaussian_block_real(n, nev + nex, 923)
        S = synth.gaussian_block_real(n, 5, 924)
        solve = chase.chase_solve_real
    else:
        q = synth.unitary_qr(n, 921)
        lam = synth.spectrum_clustered(n, 922, n_cluster=30)
        H = synth.hermitian_from(q, lam)
        V0 = synth.gaussian_block(n, nev + nex, 923)
        S = synth.gaussian_block(n, 5, 924)
        solve = chase.chase_solve
    Hd = dcol(H)
    Hl = Hd.clone()
    iu = torch.triu_indices(n, n, offset=1, device=DEV)
    Hl[iu[0], iu[1]] = float("nan")
    out = {}
    for storage, Hx in ((chase.CHASE_STORAGE_FULL, Hd), (chase.CHASE_STORAGE_LOWER, Hl)):
        o = chase.chase_opts_default(storage=storage)
        st, ritz, res, stats = solve(Hx, nev, nex, tol, dcol(V0), dcol(S), opts=o)
        assert st == chase.CHASE_OK
        out[storage] = (ritz, stats["iterations"])
    rf, itf = out[chase.CHASE_STORAGE_FULL]
    rl, itl = out[chase.CHASE_STORAGE_LOWER]
    assert itf == itl
    hn = float(lam.abs().max())
    assert np.max(np.abs(rf[:nev] - rl[:nev])) <= 1e-12 * hn
    assert np.max(np.abs(rl[:nev] - lam.numpy()[:nev])) <= 1e-10 * hn
