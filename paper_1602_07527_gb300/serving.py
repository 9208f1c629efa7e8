"""Continuous-batching server for forward + reverse Cholesky solves.

Each request carries one SPD covariance Sigma (squared-exponential kernel on
seeded points) and a reverse-mode seed L_bar; serving it means
L = cd_chol_fwd(Sigma) followed by tril(Sigma_bar) = cd_chol_rev(L, L_bar)
(Sec. 4.2), with L kept resident on the device between the two.

The loop replays the arrival times in real time.  Requests that have arrived
wait in a FIFO queue per precision; whenever a lane of that precision (a CUDA
stream with its own library handle and workspace) has room and the HBM budget
allows, the queue's head is admitted as one ragged batch: its requests run
together inside the same grouped kernels (cd_chol_*_batched), and the
batches of all lanes overlap on the device.  Sub-batches complete through
their own CUDA events; their memory then returns to the budget and newly
arrived requests are admitted.

The HBM budget covers everything the server holds on the device: each lane's
library workspace, reserved once when the server starts (the library then
never allocates during a call, because a batch is admitted to a lane only if
the workspace bound of its sizes, cd_workspace_size_batched, fits that
reservation), plus the buffers of the requests in flight.
"""
import collections
import dataclasses
import math
import queue
import threading
import time
from typing import List, Optional

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
    payload: Optional[tuple] = None   # (Sigma, L_bar) already on the device, if prepared


def requests_from_stream(stream, mixed_prec="bf16x6"):
    """Requests from workloads.serving_stream tuples (t, n, mixed, seed)."""
    return [Request(rid=i, t_arrival=t, n=n, prec=(mixed_prec if mixed else "fp64"), seed=seed)
            for i, (t, n, mixed, seed) in enumerate(stream)]


def request_bytes(n: int, prec: str) -> int:
    """HBM held by one request in flight: its Sigma/L and L_bar/Sigma_bar
    buffers (the split-BF16 operand copies of a mixed request live in the
    lane's workspace, counted separately)."""
    return 2 * n * n * 8


def lane_workspace_bytes(device, prec, nb=0, n_max=4096, ws_requests=2) -> int:
    """The workspace one lane of precision `prec` reserves: the library's
    bound for a batched call over ws_requests problems of size n_max."""
    return native.workspace_size_batched([int(n_max)] * int(ws_requests), nb=nb, prec=prec, device=device)


def build_inputs(req: Request, device, ell=SE_ELL, jitter=SE_JITTER):
    """The request's payload, drawn on the device from the request's seed
    (no host-to-device copy, which would block the launching thread):
    points uniform in [0,1]^3 -> SE covariance Sigma, and L_bar iid N(0,1)."""
    g = torch.Generator(device=device)
    g.manual_seed(int(req.seed) & 0x7FFFFFFFFFFFFFFF)
    X = torch.rand(req.n, 3, generator=g, device=device, dtype=torch.float64)
    S = torch.cdist(X, X).square_().mul_(-0.5 / (ell * ell)).exp_()
    S.diagonal().add_(jitter)
    Lb = torch.randn(req.n, req.n, generator=g, device=device, dtype=torch.float64).tril_()
    return S, Lb


def prepare(requests: List[Request], device):
    """Build every request's payload on the device ahead of a replay, so that
    the served timings cover the solves only (as if the data had arrived)."""
    for r in requests:
        r.payload = build_inputs(r, device)
    torch.cuda.synchronize(device)


def solve_alone(req: Request, device, nb=0):
    """One request by itself on the shared handle: returns (L, tril(Sigma_bar), info)."""
    A, Ab = req.payload if req.payload is not None else build_inputs(req, device)
    info = native.chol_fwd(A, nb=nb, prec=req.prec)
    native.chol_rev(A, Ab, nb=nb, prec=req.prec)
    return A, Ab, info


class _Lane:
    """One CUDA stream with its own library handle and host thread, serving
    one precision.  The thread turns admitted batches into launches (the
    library's host loop runs without holding the GIL), so lanes enqueue work
    in parallel while the scheduler thread keeps admitting and completing."""

    def __init__(self, device, prec, high, ws_bytes, nb):
        self.device = device
        self.prec = prec
        self.nb = nb
        lo, hi = torch.cuda.Stream.priority_range() if hasattr(torch.cuda.Stream, "priority_range") else (0, -5)
        self.stream = torch.cuda.Stream(device, priority=hi if high else 0)
        self.handle = native.Handle(device)
        # cheap (split-BF16) requests are scheduled ahead of FP64 ones on a shared GPU
        self.handle.set_priorities(hi if high else min(0, hi + 2), hi + 1 if high else 0)
        native.reserve(ws_bytes, device, handle_=self.handle)   # held for the server's life
        self.ws_bytes = native.workspace_bytes(self.handle, device)
        self.inflight = collections.deque()   # (event, requests, bytes, last), in stream order
        self.lock = threading.Lock()
        self.batches = 0                      # admitted batches not yet complete (scheduler thread only)
        self.launch_s = 0.0
        self.phase_s = {"inputs": 0.0, "fwd": 0.0, "rev": 0.0}
        self.work = queue.Queue()
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    def _loop(self):
        torch.cuda.set_device(self.device)
        while True:
            item = self.work.get()
            if item is None:
                return
            server, batch = item
            t = time.perf_counter()
            entries = server._launch(self, batch)
            self.launch_s += time.perf_counter() - t
            with self.lock:
                self.inflight.extend(entries)

    def close(self):
        self.work.put(None)
        self.thread.join()
        self.handle.close()


class Server:
    """Continuous batching over `lanes_per_prec` lanes per precision.

    A lane accepts a new batch while up to `depth` earlier batches are still
    queued or running on its stream, so the stream never idles between
    batches.  An admitted batch is sorted by size and launched as size-class
    sub-batches (sizes within a factor of two), each with its own completion
    event, so that small requests finish without waiting for large ones.
    """

    def __init__(self, device="cuda:0", mem_cap=40e9, lanes_per_prec=2, max_batch=64, nb=0, depth=2,
                 keep_results=False, precisions=("fp64", "bf16x6", "bf16x3"), n_max=4096, ws_requests=2):
        self.device = torch.device(device)
        self.mem_cap = float(mem_cap)
        self.max_batch = int(max_batch)
        self.nb = nb
        self.depth = int(depth)
        self.keep = keep_results
        self.n_max = int(n_max)
        # each lane's workspace: the bound for ws_requests problems of the largest size
        ws = {p: lane_workspace_bytes(self.device, p, nb, self.n_max, ws_requests) for p in precisions}
        self.lanes = [_Lane(self.device, p, p != "fp64", ws[p], nb) for p in precisions
                      for _ in range(lanes_per_prec)]
        self.ws_total = float(sum(ln.ws_bytes for ln in self.lanes))
        if self.ws_total >= self.mem_cap:
            raise ValueError("the lanes' workspaces alone exceed the memory cap")
        self.peak_bytes = 0.0

    @property
    def host_launch_s(self):
        return sum(ln.launch_s for ln in self.lanes)

    @property
    def host_phase_s(self):
        return {k: sum(ln.phase_s[k] for ln in self.lanes) for k in ("inputs", "fwd", "rev")}

    def close(self):
        for ln in self.lanes:
            ln.close()

    def _ws_need(self, ns, prec):
        """Workspace bound of one batched call over sizes ns (host arithmetic)."""
        return native.workspace_size_batched(ns, nb=self.nb, prec=prec, device=self.device)

    def _launch(self, lane: _Lane, batch: List[Request]):
        """Enqueue one admitted batch on the lane (lane thread); returns its entries."""
        out = []
        batch = sorted(batch, key=lambda r: r.n)
        classes = collections.OrderedDict()
        for r in batch:
            classes.setdefault(max(1, r.n).bit_length(), []).append(r)
        with torch.cuda.stream(lane.stream):
            for grp in classes.values():
                t = time.perf_counter()
                bufs = [r.payload if r.payload is not None else build_inputs(r, self.device) for r in grp]
                As = [b[0] for b in bufs]
                Abs = [b[1] for b in bufs]
                t1 = time.perf_counter()
                info = native.chol_fwd_batched(As, nb=self.nb, prec=lane.prec, handle_=lane.handle)
                t2 = time.perf_counter()
                native.chol_rev_batched(As, Abs, nb=self.nb, prec=lane.prec, handle_=lane.handle)
                t3 = time.perf_counter()
                lane.phase_s["inputs"] += t1 - t
                lane.phase_s["fwd"] += t2 - t1
                lane.phase_s["rev"] += t3 - t2
                if self.keep:
                    for i, r in enumerate(grp):
                        r.sigma_bar = Abs[i]
                        r.info = info[i:i + 1]
                ev = torch.cuda.Event()
                ev.record(lane.stream)
                out.append((ev, grp, sum(request_bytes(r.n, r.prec) for r in grp), False))
        out[-1] = out[-1][:3] + (True,)
        return out

    def run(self, requests: List[Request], realtime: bool = True):
        """Serve `requests` (arrival times replayed in real time unless
        realtime=False, which releases every request at t = 0).  Returns the
        list of completed requests with t_admit / t_done filled in."""
        reqs = sorted(requests, key=lambda r: r.t_arrival)
        precs = {ln.prec for ln in self.lanes}
        lane_ws = {ln.prec: ln.ws_bytes for ln in self.lanes}
        for r in reqs:
            if request_bytes(r.n, r.prec) > self.mem_cap - self.ws_total:
                raise ValueError(f"request {r.rid} alone exceeds the memory cap")
            if r.prec in lane_ws and self._ws_need([r.n], r.prec) > lane_ws[r.prec]:
                raise ValueError(f"request {r.rid} needs more workspace than a lane holds")
            if r.prec not in precs:
                raise ValueError(f"no lane serves precision {r.prec}")
        pending = {p: collections.deque() for p in precs}
        done: List[Request] = []
        in_use = self.ws_total   # the lanes' workspaces, then the requests in flight
        i = 0
        t0 = time.perf_counter()
        while len(done) < len(reqs):
            now = time.perf_counter() - t0
            while i < len(reqs) and (not realtime or reqs[i].t_arrival <= now):
                pending[reqs[i].prec].append(reqs[i])
                i += 1
            progressed = False
            for ln in self.lanes:                      # completions, in stream order
                with ln.lock:
                    while ln.inflight and ln.inflight[0][0].query():
                        _, grp, b, last = ln.inflight.popleft()
                        t = time.perf_counter() - t0
                        for r in grp:
                            r.t_done = t
                        done.extend(grp)
                        in_use -= b
                        if last:
                            ln.batches -= 1
                        progressed = True
            for ln in self.lanes:                      # admissions
                q = pending[ln.prec]
                while q and ln.batches < self.depth:
                    batch, need = [], 0.0
                    while q and len(batch) < self.max_batch:
                        b = request_bytes(q[0].n, q[0].prec)
                        if in_use + need + b > self.mem_cap:
                            break
                        if batch and self._ws_need([r.n for r in batch] + [q[0].n], ln.prec) > ln.ws_bytes:
                            break
                        r = q.popleft()
                        r.t_admit = time.perf_counter() - t0
                        batch.append(r)
                        need += b
                    if not batch:
                        break
                    in_use += need
                    self.peak_bytes = max(self.peak_bytes, in_use)
                    ln.batches += 1
                    ln.work.put((self, batch))
                    progressed = True
            if not progressed:
                if i < len(reqs) and realtime and not any(pending.values()):
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
