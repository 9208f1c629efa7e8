"""Continuous-batching server for forward + reverse Cholesky solves.

Each request carries one SPD covariance Sigma (squared-exponential kernel on
seeded points) and a reverse-mode seed L_bar; serving it means
L = cd_chol_fwd(Sigma) followed by tril(Sigma_bar) = cd_chol_rev(L, L_bar)
(Sec. 4.2), with L kept resident on the device between the two.

The loop replays the arrival times in real time.  Requests that have arrived
wait in a FIFO queue; whenever a lane (a CUDA stream with its own library
handle and workspace) is free and the HBM budget allows, the queue's head is
admitted as one ragged batch: its requests run together inside the same
grouped kernels (cd_chol_*_batched), and batches of different lanes overlap
on the device.  A batch completes when its CUDA event does; its memory then
returns to the budget and newly arrived requests are admitted.  Precision is
per request (FP64 or split-BF16); requests of one precision in a batch share
one call.
"""
import collections
import dataclasses
import math
import time
from typing import List, Optional

import numpy as np
import torch

from . import native

SE_ELL = 0.3
SE_JITTER = 1e-2   # keeps the mixed-precision requests well conditioned (cond < 1e5 at N = 4096)


@dataclasses.dataclass
class Request:
    rid: int
    t_arrival: float          # seconds after the start of the stream
    n: int
    prec: str                 # "fp64", "bf16x6" or "bf16x3"
    seed: int
    t_admit: Optional[float] = None
    t_done: Optional[float] = None
    sigma_bar: Optional[torch.Tensor] = None
    info: Optional[torch.Tensor] = None


def requests_from_stream(stream, mixed_prec="bf16x6"):
    """Requests from workloads.serving_stream tuples (t, n, mixed, seed)."""
    return [Request(rid=i, t_arrival=t, n=n, prec=(mixed_prec if mixed else "fp64"), seed=seed)
            for i, (t, n, mixed, seed) in enumerate(stream)]


def request_bytes(n: int, prec: str) -> int:
    """HBM held by one request in flight: its Sigma/L and L_bar/Sigma_bar
    buffers, plus the split-BF16 operand copies of a mixed request."""
    b = 2 * n * n * 8
    if prec != "fp64":
        b += (3 if prec == "bf16x6" else 2) * 2 * 2 * n * (n + 72)
    return b


def build_inputs(req: Request, device, ell=SE_ELL, jitter=SE_JITTER):
    """The request's payload: Sigma from its seeded points, L_bar from its seed."""
    rng = np.random.default_rng([req.seed, 0])
    X = torch.tensor(rng.uniform(size=(req.n, 3)), device=device)
    S = torch.cdist(X, X).square_().mul_(-0.5 / (ell * ell)).exp_()
    S.diagonal().add_(jitter)
    g = torch.Generator(device=device)
    g.manual_seed(int(req.seed) & 0x7FFFFFFFFFFFFFFF)
    Lb = torch.randn(req.n, req.n, generator=g, device=device, dtype=torch.float64).tril_()
    return S, Lb


def solve_alone(req: Request, device, nb=0):
    """One request by itself on the shared handle: returns (L, tril(Sigma_bar), info)."""
    A, Ab = build_inputs(req, device)
    info = native.chol_fwd(A, nb=nb, prec=req.prec)
    native.chol_rev(A, Ab, nb=nb, prec=req.prec)
    return A, Ab, info


class _Lane:
    def __init__(self, device):
        self.stream = torch.cuda.Stream(device)
        self.handle = native.Handle(device)
        self.batch: List[Request] = []
        self.event = None
        self.bytes = 0


class Server:
    def __init__(self, device="cuda:0", mem_cap=40e9, lanes=2, max_batch=64, nb=0, keep_results=False):
        self.device = torch.device(device)
        self.mem_cap = float(mem_cap)
        self.max_batch = int(max_batch)
        self.nb = nb
        self.keep = keep_results
        self.lanes = [_Lane(self.device) for _ in range(lanes)]
        self.peak_bytes = 0.0

    def close(self):
        for ln in self.lanes:
            ln.handle.close()

    def _launch(self, lane: _Lane, batch: List[Request]):
        with torch.cuda.stream(lane.stream):
            bufs = {}
            for r in batch:
                bufs[r.rid] = build_inputs(r, self.device)
            for prec in ("fp64", "bf16x6", "bf16x3"):
                grp = [r for r in batch if r.prec == prec]
                if not grp:
                    continue
                As = [bufs[r.rid][0] for r in grp]
                Abs = [bufs[r.rid][1] for r in grp]
                info = native.chol_fwd_batched(As, nb=self.nb, prec=prec, handle_=lane.handle)
                native.chol_rev_batched(As, Abs, nb=self.nb, prec=prec, handle_=lane.handle)
                for i, r in enumerate(grp):
                    if self.keep:
                        r.sigma_bar = Abs[i]
                        r.info = info[i:i + 1]
            lane.event = torch.cuda.Event()
            lane.event.record(lane.stream)
        lane.batch = batch
        lane.bytes = sum(request_bytes(r.n, r.prec) for r in batch)

    def run(self, requests: List[Request], realtime: bool = True):
        """Serve `requests` (arrival times replayed in real time unless
        realtime=False, which releases every request at t = 0).  Returns the
        list of completed requests with t_admit / t_done filled in."""
        reqs = sorted(requests, key=lambda r: r.t_arrival)
        for r in reqs:
            if request_bytes(r.n, r.prec) > self.mem_cap:
                raise ValueError(f"request {r.rid} alone exceeds the memory cap")
        pending = collections.deque()
        done: List[Request] = []
        in_use = 0.0
        i = 0
        t0 = time.perf_counter()
        while len(done) < len(reqs):
            now = time.perf_counter() - t0
            while i < len(reqs) and (not realtime or reqs[i].t_arrival <= now):
                pending.append(reqs[i])
                i += 1
            progressed = False
            for ln in self.lanes:
                if ln.batch and ln.event.query():
                    t = time.perf_counter() - t0
                    for r in ln.batch:
                        r.t_done = t
                    done.extend(ln.batch)
                    in_use -= ln.bytes
                    ln.batch, ln.bytes = [], 0
                    progressed = True
            for ln in self.lanes:
                if ln.batch or not pending:
                    continue
                batch, need = [], 0.0
                while pending and len(batch) < self.max_batch:
                    b = request_bytes(pending[0].n, pending[0].prec)
                    if in_use + need + b > self.mem_cap:
                        break
                    r = pending.popleft()
                    r.t_admit = time.perf_counter() - t0
                    batch.append(r)
                    need += b
                if not batch:
                    break
                in_use += need
                self.peak_bytes = max(self.peak_bytes, in_use)
                self._launch(ln, batch)
                progressed = True
            if not progressed:
                if i < len(reqs) and not pending and realtime:
                    time.sleep(max(0.0, min(1e-3, reqs[i].t_arrival - (time.perf_counter() - t0))))
                else:
                    time.sleep(5e-5)
        return done


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return float("nan")
    k = (len(xs) - 1) * q / 100.0
    lo, hi = int(math.floor(k)), int(math.ceil(k))
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


def summarize(done: List[Request], wall: Optional[float] = None):
    lat = [r.t_done - r.t_arrival for r in done]
    svc = [r.t_done - r.t_admit for r in done]
    span = wall if wall is not None else (max(r.t_done for r in done) - min(r.t_arrival for r in done))
    flops = sum(r.n ** 3 for r in done)  # n^3/3 (fwd) + 2 n^3/3 (rev)
    return {"requests": len(done), "p50_ms": 1e3 * percentile(lat, 50), "p99_ms": 1e3 * percentile(lat, 99),
            "service_p50_ms": 1e3 * percentile(svc, 50), "service_p99_ms": 1e3 * percentile(svc, 99),
            "solves_per_s": len(done) / span, "tflops": flops / span / 1e12, "span_s": span}
