"""Serving loop: continuous batching of sequence-solve requests on one GPU.

A request is a correlated sequence of Hermitian problems (as in the
benchmark's sequence workload: H_{k+1} = H_k + 1e-3 ||H_1|| E_k), solved
problem after problem with ChASE, each problem warm-started from the
previous one's Ritz vectors and values (Sec. 3.3: the approx flag), which
stay resident on the device for the request's lifetime.

Continuous batching: requests arrive over time (a seeded Poisson trace);
the dispatcher admits a waiting request as soon as a slot is free and its
estimated device footprint fits under the memory cap (first fit, so a
large request at the head does not block smaller ones behind it; waiting
requests are taken in arrival order, or shortest job first with an aging
limit).  Every slot owns a CUDA stream and a host thread; the solves of
admitted requests run concurrently and overlap on the device.  Every step
of every solve runs in libchase's kernels through the C ABI; this module
only schedules, generates inputs and records latencies.
"""

from __future__ import annotations

import dataclasses
import heapq
import math
import threading
import time
from typing import Callable, List, Optional

import numpy as np

__all__ = ["Request", "Result", "poisson_trace", "footprint_bytes", "Server", "gpu_sequence_solver",
           "percentile", "warm_eigensolver"]


@dataclasses.dataclass(frozen=True)
class Request:
    rid: int
    n: int
    nev: int
    nex: int
    nprob: int
    seed: int
    arrival: float  # seconds after the start of the trace


@dataclasses.dataclass
class Result:
    rid: int
    n: int
    nprob: int
    arrival: float
    admitted: float
    finished: float
    slot: int
    statuses: List[int]
    iterations: List[int]
    ritz: List[np.ndarray]
    resid_max_over_norm: List[float]
    flops: float
    last_h: Optional[np.ndarray] = None  # the last problem's H (host), when kept for checks

    @property
    def latency(self) -> float:
        return self.finished - self.arrival

    @property
    def queueing(self) -> float:
        return self.admitted - self.arrival


def poisson_trace(n_requests: int, rate: float, seed: int,
                  sizes=(2048, 4096, 8192, 16384), weights=(4, 3, 2, 1),
                  nprob_range=(5, 10), nev_frac=0.04, nex_frac=0.2) -> List[Request]:
    """Seeded trace: exponential inter-arrival times (rate per second), N drawn
    with the given weights, 5-10 problems, nev = ceil(nev_frac N),
    nex = ceil(nex_frac nev)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    p = np.asarray(weights, dtype=float)
    p /= p.sum()
    for i in range(n_requests):
        t += float(rng.exponential(1.0 / rate))
        n = int(rng.choice(sizes, p=p))
        nev = int(math.ceil(nev_frac * n))
        nex = int(math.ceil(nex_frac * nev))
        nprob = int(rng.integers(nprob_range[0], nprob_range[1] + 1))
        out.append(Request(i, n, nev, nex, nprob, int(rng.integers(1, 2**31)), t))
    return out


def footprint_bytes(n: int, nev: int, nex: int, split: bool) -> int:
    """Device bytes a request holds while it runs: the current and next H
    (complex128), the FFT generator's temporaries, the split slices of H,
    the resident block and the solver's N x (nev+nex) workspaces."""
    nx = nev + nex
    h = 16 * n * n
    gen = 3 * h                                   # construction temporaries
    slices = 28 * n * n if split else 0          # 7 BF16 slice planes of [Re H | Im H]
    blocks = 16 * n * nx * 10                    # V, filter buffer, RR/QR work, slices of V
    return int(2 * h + gen + slices + blocks)


def percentile(xs, q):
    if not xs:
        return float("nan")
    return float(np.percentile(np.asarray(xs, dtype=float), q))


def work_estimate(r: Request) -> float:
    """Relative cost of a request for shortest-job-first admission: its
    problems times the N^2 (nev + nex) of one filter product."""
    return float(r.nprob) * float(r.n) ** 2 * float(r.nev + r.nex)


class Server:
    """Admission by device footprint, slots with their own streams and threads.

    ``solve_fn(request, slot) -> Result-like dict`` runs one whole request
    (all its problems) on the slot's stream; it is injected so that the
    scheduling logic can be exercised without a GPU.

    ``policy`` orders the waiting requests for first-fit admission:
    ``"fifo"`` by arrival, ``"sjf"`` by ``cost_fn`` (shortest job first),
    except that a request that has waited ``max_wait_s`` seconds or more
    goes ahead of every request that has not (no request starves)."""

    def __init__(self, solve_fn: Callable, mem_cap_bytes: float, max_slots: int,
                 footprint_fn: Callable[[Request], int], policy: str = "fifo",
                 cost_fn: Callable[[Request], float] = work_estimate,
                 max_wait_s: Optional[float] = None):
        if policy not in ("fifo", "sjf"):
            raise ValueError(f"unknown admission policy {policy!r}")
        self.solve_fn = solve_fn
        self.mem_cap = float(mem_cap_bytes)
        self.max_slots = int(max_slots)
        self.footprint_fn = footprint_fn
        self.policy = policy
        self.cost_fn = cost_fn
        self.max_wait_s = max_wait_s
        self._cv = threading.Condition()
        self._waiting: List[Request] = []
        self._mem_used = 0.0
        self._free_slots = list(range(self.max_slots))
        self._results: List[Result] = []
        self._errors: List[BaseException] = []
        self.peak_mem = 0.0
        self.peak_concurrency = 0
        self._running = 0
        self._t0 = 0.0

    def _now(self) -> float:
        return time.perf_counter() - self._t0

    def _order_locked(self):
        """Indices into the waiting list in admission order."""
        idx = list(range(len(self._waiting)))
        if self.policy == "fifo":
            return idx
        now = self._now()

        def key(i):
            r = self._waiting[i]
            aged = self.max_wait_s is not None and now - r.arrival >= self.max_wait_s
            # aged requests first (oldest first), then the cheapest
            return (0, r.arrival, 0.0) if aged else (1, 0.0, self.cost_fn(r))

        return sorted(idx, key=key)

    def _admit_locked(self):
        """First fit in the policy's order; returns (request, slot) or None."""
        if not self._free_slots:
            return None
        for i in self._order_locked():
            r = self._waiting[i]
            fp = self.footprint_fn(r)
            if fp > self.mem_cap:
                raise ValueError(f"request {r.rid} needs {fp} bytes, above the cap")
            if self._mem_used + fp <= self.mem_cap:
                self._waiting.pop(i)
                self._mem_used += fp
                self.peak_mem = max(self.peak_mem, self._mem_used)
                slot = self._free_slots.pop(0)
                self._running += 1
                self.peak_concurrency = max(self.peak_concurrency, self._running)
                return r, slot
        return None

    def _worker(self, req: Request, slot: int, admitted: float):
        try:
            out = self.solve_fn(req, slot)
            res = Result(rid=req.rid, n=req.n, nprob=req.nprob, arrival=req.arrival,
                         admitted=admitted, finished=self._now(), slot=slot, **out)
            with self._cv:
                self._results.append(res)
        except BaseException as e:  # surfaced by run()
            with self._cv:
                self._errors.append(e)
        finally:
            with self._cv:
                self._mem_used -= self.footprint_fn(req)
                self._free_slots.append(slot)
                self._free_slots.sort()
                self._running -= 1
                self._cv.notify_all()

    def run(self, trace: List[Request], realtime: bool = True) -> List[Result]:
        """Replay the trace (arrivals in real time when ``realtime``) and
        return one Result per request, in request order."""
        pending = [(r.arrival, r.rid, r) for r in trace]
        heapq.heapify(pending)
        threads = []
        self._t0 = time.perf_counter()
        with self._cv:
            while pending or self._waiting or self._running:
                if self._errors:
                    break
                now = self._now()
                while pending and (not realtime or pending[0][0] <= now):
                    _, _, r = heapq.heappop(pending)
                    self._waiting.append(r)
                while True:
                    adm = self._admit_locked()
                    if adm is None:
                        break
                    r, slot = adm
                    t = threading.Thread(target=self._worker, args=(r, slot, self._now()),
                                         daemon=True)
                    threads.append(t)
                    t.start()
                timeout = None
                if pending and realtime:
                    timeout = max(0.0, pending[0][0] - self._now())
                if not pending and not self._waiting and not self._running:
                    break
                self._cv.wait(timeout=timeout if timeout is not None else 0.5)
        for t in threads:
            t.join()
        if self._errors:
            raise self._errors[0]
        return sorted(self._results, key=lambda x: x.rid)


def gpu_sequence_solver(device, precision: int, tol: float = 1e-10, seq_scale: float = 1e-3,
                        keep_last_h: bool = False, deg_extra: Optional[int] = None,
                        deg_max: Optional[int] = None):
    """solve_fn for Server: builds the request's sequence on the slot's
    stream and solves it problem after problem with warm starts.  With
    ``keep_last_h`` the result also carries the last problem's H on the host
    (for checks against its exact spectrum).  ``deg_extra`` and ``deg_max``
    override DEGEXTRA and DEGMAX of Alg. 5 (Table 1: 2 and 36)."""
    import torch

    from . import chase, synth

    streams = {}

    def solve(req: Request, slot: int):
        if slot not in streams:
            streams[slot] = torch.cuda.Stream(device=device)
        s = streams[slot]
        nx = req.nev + req.nex
        statuses, iters, ritz, rmax = [], [], [], []
        flops = 0.0
        with torch.cuda.stream(s):
            lam = synth.spectrum_dft(req.n, req.seed, device=device)
            H = synth.hermitian_dft(lam, req.seed + 1)
            hnorm = float(lam.abs().max())
            V = synth.gaussian_block(req.n, nx, req.seed + 7, device=device)
            S = synth.gaussian_block(req.n, 5, req.seed + 8, device=device)
            Lam = None
            for k in range(req.nprob):
                if k > 0:
                    E = synth.hermitian_noise(req.n, req.seed + 100 + k, device=device)
                    H = (H + (seq_scale * hnorm) * E).t().contiguous().t()
                    del E
                o = chase.chase_opts_default(approx=0 if k == 0 else 1, precision=precision)
                if deg_extra is not None:
                    o.deg_extra = int(deg_extra)
                if deg_max is not None:
                    o.deg_max = int(deg_max)
                st, Lam, res, stats = chase.chase_solve(
                    H, req.nev, req.nex, tol, V, S if k == 0 else S[:, :1].contiguous(),
                    Lambda=Lam, opts=o, stream=s.cuda_stream)
                statuses.append(int(st))
                iters.append(int(stats["iterations"]))
                ritz.append(Lam[:req.nev].copy())
                rmax.append(float(np.max(res[:req.nev])) / hnorm)
                flops += float(stats["flops_total"])
            s.synchronize()
            last = H.cpu().numpy() if keep_last_h else None
            del H, V, S
        return {"statuses": statuses, "iterations": iters, "ritz": ritz,
                "resid_max_over_norm": rmax, "flops": flops, "last_h": last}

    return solve


def warm_eigensolver(device, widths, seed: int = 77):
    """Run Rayleigh-Ritz (and so its projected eigensolve) once at each width
    and at the widths below it down to 16 (factor sqrt 2).  On a fresh
    machine the first eigensolve of a size class in a process costs seconds
    (measured on GB300: 9.5 s for the first 1500 x 1500 solve, 0.32 s for
    every later one) while the solver prepares its kernels for the device;
    a server calls this once at start-up with the widths (nev + nex) it
    expects, so that no request pays that cost."""
    import torch

    from . import chase, synth

    ws = set()
    for w in widths:
        w = float(w)
        while w >= 16:
            ws.add(int(w))
            w /= 1.4142
    for w in sorted(ws, reverse=True):
        n = max(2 * w, 64)
        lam = synth.spectrum_uniform(n, seed, device=device)
        H = synth.hermitian_dft(lam, seed + 1)
        Q = synth.gaussian_block(n, w, seed + 2, device=device).t().contiguous().t()
        chase.chase_orthonormalize(None, Q)
        chase.chase_rayleigh_ritz(H, Q)
        del H, Q
    torch.cuda.synchronize(device)
