"""Results do not depend on what else runs on the device.

The FP64 product kernels stage operand tiles with TMA and read them with
ordinary shared-memory loads; a stage is handed back to the TMA producer
only after those reads are ordered before the next asynchronous copy.  A
missing proxy fence there let a copy overwrite a stage before a warp's last
loads had returned whenever other kernels kept the SM's load pipe busy,
which corrupted 8 x 8 fragments of the product (and, through the filter,
whole columns).  Each case here runs a product-heavy call alone, then again
while other streams run memory-bound kernels, and demands bit-identical
results."""

import threading

import numpy as np
import pytest
import torch

from paper_1805_10121_gb300 import chase, synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
REPS = 6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1805_10121_gb300 import build
    build.build()
    chase.lib()


def cm(t):
    return t.t().contiguous().t()


class Load:
    """Memory-bound elementwise kernels on three other streams."""

    def __init__(self):
        self.streams = [torch.cuda.Stream(device=DEV) for _ in range(3)]
        self.bufs = [torch.randn(4096, 4096, device=DEV) for _ in range(3)]
        torch.cuda.synchronize()
        self.stop = False
        self.threads = [threading.Thread(target=self._run, args=(k,)) for k in range(3)]

    def _run(self, k):
        with torch.cuda.stream(self.streams[k]):
            while not self.stop:
                for _ in range(20):
                    self.bufs[k].mul_(1.0000001).add_(1e-7)
                self.streams[k].synchronize()

    def __enter__(self):
        for t in self.threads:
            t.start()
        return self

    def __exit__(self, *exc):
        self.stop = True
        for t in self.threads:
            t.join()


def alone_then_loaded(fn):
    s = torch.cuda.Stream(device=DEV)
    ref = fn(s)
    bad = []
    with Load():
        for r in range(REPS):
            out = fn(s)
            d = max(float(np.max(np.abs(a - b))) for a, b in zip(out, ref))
            if d != 0.0:
                bad.append((r, d))
    assert not bad, f"results changed under concurrent load: {bad}"


def problem(n, seed, dtype=torch.complex128):
    lam = synth.spectrum_dft(n, seed, device=DEV)
    H = synth.hermitian_dft(lam, seed + 1)
    if dtype == torch.float64:
        H = cm(H.real)
    return H, lam.cpu().numpy()


def test_fp64_filter_and_residuals_unchanged_by_other_streams():
    n, b = 2048, 99  # 99 columns: the 64 x 8 tile shape, the one that showed the race
    H, l = problem(n, 11)
    V0 = cm(synth.gaussian_block(n, b, 12, device=DEV))
    deg = np.array([2 + 2 * (j % 6) for j in range(b)], dtype=np.int32)
    torch.cuda.synchronize()

    def run(s):
        with torch.cuda.stream(s):
            V = V0.clone()
            chase.chase_filter(H, V, deg, 1.01 * l[-1], float(l[0]), float(l[b]),
                               stream=s.cuda_stream)
            r = chase.chase_residuals(H, V0, np.zeros(b), stream=s.cuda_stream)
            s.synchronize()
            return V.cpu().numpy(), r

    alone_then_loaded(run)


def test_real_fp64_filter_unchanged_by_other_streams():
    n, b = 2048, 99
    H, l = problem(n, 21, torch.float64)
    V0 = synth.gaussian_block_real(n, b, 22, device=DEV).contiguous().t().contiguous().t()
    deg = np.full(b, 4, dtype=np.int32)
    torch.cuda.synchronize()

    def run(s):
        with torch.cuda.stream(s):
            V = V0.clone()
            chase.chase_filter_real(H, V, deg, 1.01 * l[-1], float(l[0]), float(l[b]),
                                    stream=s.cuda_stream)
            s.synchronize()
            return (V.cpu().numpy(),)

    alone_then_loaded(run)


def test_batched_fp64_filter_unchanged_by_other_streams():
    sizes = [700, 1024, 333]
    Hs, Vs, ls = [], [], []
    for q, n in enumerate(sizes):
        H, l = problem(n, 31 + 2 * q)
        Hs.append(H)
        ls.append(l)
        Vs.append(cm(synth.gaussian_block(n, 40, 50 + q, device=DEV)))
    degs = [np.array([2 + 2 * (j % 5) for j in range(40)], dtype=np.int32) for _ in sizes]
    torch.cuda.synchronize()

    def run(s):
        with torch.cuda.stream(s):
            W = [v.clone() for v in Vs]
            chase.chase_filter_batched(Hs, W, degs, [1.01 * l[-1] for l in ls],
                                       [float(l[0]) for l in ls], [float(l[40]) for l in ls],
                                       tile=0, stream=s.cuda_stream)
            s.synchronize()
            return [w.cpu().numpy() for w in W]

    alone_then_loaded(run)
