"""The allocation-free residual entry point, for callers that cannot let the
library allocate device memory (a framework that owns a fixed device-memory
budget, or a caller that cannot afford the device-wide synchronisation of
cudaMalloc / cudaFree).  It must give the same residual norms as
chase_residuals, call after call, although it reuses one fixed scratch
array.  This file is collected last on purpose."""

import numpy as np
import pytest
import torch

from paper_1805_10121_gb300 import chase, synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1805_10121_gb300 import build
    build.build()
    chase.lib()


def _problem(n, b, seed):
    q = synth.unitary_qr(n, seed)
    lam = synth.spectrum_uniform(n, seed + 1)
    H = synth.hermitian_from(q, lam).to(DEV).t().contiguous().t()
    V = synth.gaussian_block(n, b, seed + 2).to(DEV).t().contiguous().t()
    w = np.linspace(-1.0, 1.0, b)
    return H, V, w


def test_noalloc_matches_allocating_entry_point_twice():
    # calls in a row, different shapes: none may see an earlier call's scratch.
    # b <= 6 takes the few-column product, larger b the tiled FP64 product.
    for n, b, seed in ((1000, 70, 11), (333, 13, 21), (1000, 1, 41), (2000, 4, 51)):
        H, V, w = _problem(n, b, seed)
        lam_d = torch.from_numpy(w).to(DEV)
        out_d = torch.full((b,), -1.0, dtype=torch.float64, device=DEV)
        torch.cuda.synchronize()
        allocs = chase.chase_device_allocations()
        chase.chase_residuals_noalloc(H, V, lam_d, out_d)
        torch.cuda.synchronize()
        # the property this entry point exists for: the library allocated nothing
        assert chase.chase_device_allocations() == allocs
        ref = chase.chase_residuals(H, V, w)
        assert chase.chase_device_allocations() > allocs  # the counter does count
        got = out_d.cpu().numpy()
        assert np.max(np.abs(got - ref) / ref) < 1e-13


def test_noalloc_rejects_oversize_and_host_arrays():
    n, b = 3000, 700  # N*b above the fixed scratch
    H = torch.zeros(n, n, dtype=torch.complex128, device=DEV).t()
    V = torch.zeros(b, n, dtype=torch.complex128, device=DEV).t()
    lam = torch.zeros(b, dtype=torch.float64, device=DEV)
    out = torch.zeros(b, dtype=torch.float64, device=DEV)
    with pytest.raises(chase.ChaseError) as ei:
        chase.chase_residuals_noalloc(H, V, lam, out)
    assert ei.value.status == chase.CHASE_INVALID_ARG
    assert "scratch" in chase.chase_last_error()
    Hs, Vs, w = _problem(64, 4, 31)
    with pytest.raises(chase.ChaseError) as ei:
        chase.chase_residuals_noalloc(Hs.cpu().t().contiguous().t(), Vs.cpu().t().contiguous().t(),
                                      torch.from_numpy(w), torch.zeros(4, dtype=torch.float64))
    assert ei.value.status == chase.CHASE_INVALID_ARG
