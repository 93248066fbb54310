"""Continuous batching on the GPU: each request's results are the same when
it runs alone and when it shares the device with others."""

import dataclasses

import numpy as np
import pytest
import torch

from paper_1805_10121_gb300 import chase, serve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1805_10121_gb300 import build
    build.build()
    chase.lib()


@pytest.mark.parametrize("precision", [chase.CHASE_SPLIT_BF16, chase.CHASE_FP64])
def test_alone_equals_in_the_mix(precision):
    dev = torch.device("cuda:0")
    trace = serve.poisson_trace(5, 200.0, 11, sizes=(256, 384, 512), weights=(1, 1, 1),
                                nprob_range=(3, 3))
    fp = lambda r: serve.footprint_bytes(r.n, r.nev, r.nex, precision == chase.CHASE_SPLIT_BF16)
    mixed = serve.Server(serve.gpu_sequence_solver(dev, precision), 64e9, 3, fp).run(trace)
    assert len(mixed) == 5
    solver = serve.gpu_sequence_solver(dev, precision)
    for r, m in zip(trace, mixed):
        alone = serve.Server(solver, 64e9, 1, fp).run([dataclasses.replace(r, arrival=0.0)])[0]
        assert m.statuses == alone.statuses == [0] * r.nprob
        for a, b in zip(m.ritz, alone.ritz):
            # the kernels are deterministic: identical, well inside 1e-10 ||H||
            assert np.max(np.abs(a - b)) <= 1e-12 * 50
        assert max(m.resid_max_over_norm) <= 1e-10
