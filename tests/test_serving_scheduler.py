"""The continuous-batching scheduler of serving.Server on the host, with fake
lanes in place of CUDA streams (no GPU): a fake launch completes a batch
after a delay proportional to its work, so admissions, completions and the
memory budget interleave as they do on the device.

Checked: every request completes exactly once; the HBM budget is never
exceeded (at every launch the admitted bytes in flight stay within the cap);
no lane holds more than `depth` batches; batches hold at most `max_batch`
requests of the lane's precision; each precision's queue is admitted in
arrival order; requests that cannot fit or have no lane are refused.
"""
import collections
import queue
import threading
import time

import pytest

from paper_1602_07527_gb300 import serving
from paper_1602_07527_gb300 import workloads as W


class _Event:
    def __init__(self, t_done):
        self.t_done = t_done

    def query(self):
        return time.perf_counter() >= self.t_done


class _FakeLane:
    def __init__(self, prec):
        self.prec = prec
        self.inflight = collections.deque()
        self.lock = threading.Lock()
        self.batches = 0
        self.launch_s = 0.0
        self.phase_s = {"inputs": 0.0, "fwd": 0.0, "rev": 0.0}
        self.work = queue.Queue()
        self.free_at = 0.0           # the fake stream runs batches one after another
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    def _loop(self):
        while True:
            item = self.work.get()
            if item is None:
                return
            server, batch = item
            entries = server._launch(self, batch)
            with self.lock:
                self.inflight.extend(entries)

    def close(self):
        self.work.put(None)
        self.thread.join()


class _FakeServer(serving.Server):
    def __init__(self, mem_cap, lanes_per_prec, max_batch, depth, precisions=("fp64", "bf16x6")):
        self.device = None
        self.mem_cap = float(mem_cap)
        self.max_batch = int(max_batch)
        self.nb = 0
        self.depth = int(depth)
        self.keep = False
        self.lanes = [_FakeLane(p) for p in precisions for _ in range(lanes_per_prec)]
        for ln in self.lanes:
            ln.ws_bytes = 3 * 8 * 1024 * 1024   # a fake workspace: room for three n = 1024 problems
        self.ws_total = 0.0
        self.peak_bytes = 0.0
        self.log_lock = threading.Lock()
        self.launches = []           # (lane, [rid], bytes in flight incl. this batch, outstanding batches)
        self.flight = 0.0

    def _ws_need(self, ns, prec):  # a fake workspace bound: 8 bytes an element of each problem
        return sum(8 * n * n for n in ns)

    def _launch(self, lane, batch):
        b = sum(serving.request_bytes(r.n, r.prec) for r in batch)
        work = sum(r.n ** 3 for r in batch) * 2e-13 + 2e-4   # seconds of fake device time
        now = time.perf_counter()
        lane.free_at = max(lane.free_at, now) + work
        with self.log_lock:
            self.flight += b
            outstanding = sum(1 for _ in lane.inflight) + 1
            self.launches.append((lane, [r.rid for r in batch], self.flight, outstanding))
        return [(_Done(self, lane.free_at, b), list(batch), b, True)]


class _Done(_Event):
    def __init__(self, server, t_done, b):
        super().__init__(t_done)
        self.server, self.b, self.seen = server, b, False

    def query(self):
        done = super().query()
        if done and not self.seen:
            self.seen = True
            with self.server.log_lock:
                self.server.flight -= self.b
        return done


def _requests(count=300, seed=11):
    st = W.serving_stream(seed=seed, rate=2000.0, duration=count / 2000.0, n_lo=32, n_hi=1024)
    return serving.requests_from_stream(st)


@pytest.mark.parametrize("cap,lanes,max_batch,depth", [(64e6, 2, 8, 2), (20e6, 1, 4, 1), (1e9, 2, 64, 3)])
def test_admission_respects_budget_depth_and_order(cap, lanes, max_batch, depth):
    reqs = _requests()
    reqs = [r for r in reqs if serving.request_bytes(r.n, r.prec) <= cap]
    srv = _FakeServer(cap, lanes, max_batch, depth)
    try:
        done = srv.run(reqs, realtime=False)
    finally:
        srv.close()
    assert sorted(r.rid for r in done) == sorted(r.rid for r in reqs)         # each exactly once
    assert srv.peak_bytes <= cap
    by_id = {r.rid: r for r in reqs}
    for lane, rids, flight, outstanding in srv.launches:
        assert flight <= cap * (1 + 1e-12)
        assert 1 <= len(rids) <= max_batch
        assert srv._ws_need([by_id[rid].n for rid in rids], lane.prec) <= lane.ws_bytes  # fits the workspace
        assert outstanding <= depth
        assert all(by_id[rid].prec == lane.prec for rid in rids)
    for prec in ("fp64", "bf16x6"):
        mine = sorted((r for r in reqs if r.prec == prec), key=lambda r: r.rid)
        admits = [r.t_admit for r in mine]
        assert admits == sorted(admits)                                        # FIFO per precision
        assert all(r.t_done >= r.t_admit for r in mine)


def test_refuses_what_cannot_be_served():
    srv = _FakeServer(1e6, 1, 4, 1, precisions=("fp64",))
    try:
        with pytest.raises(ValueError):
            srv.run([serving.Request(rid=0, t_arrival=0.0, n=4096, prec="fp64", seed=1)], realtime=False)
        with pytest.raises(ValueError):
            srv.run([serving.Request(rid=1, t_arrival=0.0, n=32, prec="bf16x6", seed=1)], realtime=False)
    finally:
        srv.close()
