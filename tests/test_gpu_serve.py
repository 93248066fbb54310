"""Continuous batching on the GPU: each request's results are the same when
it runs alone and when it shares the device with others, and they are right:
the final Ritz values of every request equal the exact lowest eigenvalues of
the last problem of its sequence (and the oracle's solve of that problem)."""

import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_1805_10121_gb300 import chase, serve, synth

pytestmark = pytest.mark.gpu

EIG_RTOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1805_10121_gb300 import build
    build.build()
    chase.lib()


@pytest.mark.parametrize("precision", [chase.CHASE_SPLIT_BF16, chase.CHASE_FP64])
def test_alone_equals_in_the_mix_and_the_exact_spectrum(precision):
    dev = torch.device("cuda:0")
    trace = serve.poisson_trace(5, 200.0, 11, sizes=(256, 384, 512), weights=(1, 1, 1),
                                nprob_range=(3, 3))
    fp = lambda r: serve.footprint_bytes(r.n, r.nev, r.nex, precision == chase.CHASE_SPLIT_BF16)
    mixed = serve.Server(serve.gpu_sequence_solver(dev, precision, keep_last_h=True), 64e9, 3,
                         fp).run(trace)
    assert len(mixed) == 5
    solver = serve.gpu_sequence_solver(dev, precision)
    for r, m in zip(trace, mixed):
        alone = serve.Server(solver, 64e9, 1, fp).run([dataclasses.replace(r, arrival=0.0)])[0]
        assert m.statuses == alone.statuses == [0] * r.nprob
        for a, b in zip(m.ritz, alone.ritz):
            # the kernels are deterministic: identical, well inside 1e-10 ||H||
            assert np.max(np.abs(a - b)) <= 1e-12 * 50
        assert max(m.resid_max_over_norm) <= 1e-10
        # ground truth: the exact spectrum of the request's last problem
        lam = np.linalg.eigvalsh(m.last_h)
        hn = float(np.abs(lam).max())
        assert np.max(np.abs(m.ritz[-1] - lam[:r.nev])) <= EIG_RTOL * hn


def test_served_request_matches_the_oracle():
    # one small request: the oracle solves its last problem from its own cold
    # start; the eigenvalues are unique, so both must give the same nev values
    dev = torch.device("cuda:0")
    req = serve.Request(0, 200, 8, 2, 3, 12345, 0.0)
    fp = lambda r: serve.footprint_bytes(r.n, r.nev, r.nex, True)
    res = serve.Server(serve.gpu_sequence_solver(dev, chase.CHASE_SPLIT_BF16, keep_last_h=True),
                       64e9, 1, fp).run([req])[0]
    H = res.last_h
    nx = req.nev + req.nex
    V = synth.gaussian_block(req.n, nx, 7).numpy()
    S = synth.gaussian_block(req.n, 5, 8).numpy()
    ref = oracle.solve(H, req.nev, req.nex, V, S, tol=1e-10)
    hn = float(np.abs(np.linalg.eigvalsh(H)).max())
    assert np.max(np.abs(res.ritz[-1] - ref["ritz"][:req.nev])) <= EIG_RTOL * hn


def test_warm_eigensolver_runs_every_size_class():
    # the start-up warm-up: one Rayleigh-Ritz per width from 100 down to 16
    dev = torch.device("cuda:0")
    n0 = chase.chase_kernel_launches()
    serve.warm_eigensolver(dev, [100])
    # widths 100, 70, 50, 35, 25, 17: six Rayleigh-Ritz calls, each several launches
    assert chase.chase_kernel_launches() - n0 >= 6
