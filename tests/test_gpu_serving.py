"""Continuous batching: every served result is bitwise the result of the same
request solved alone (each problem's launch parameters depend on its own
shape only, in FP64 and in split-BF16), the HBM budget is respected, and
results match the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_1602_07527_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def srv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_07527_gb300 import serving
    return serving


def _stream(serving, count, n_hi, seed=5):
    st = W.serving_stream(seed=seed, rate=2000.0, duration=count / 2000.0, n_lo=32, n_hi=n_hi)
    return serving.requests_from_stream(st)


def test_served_equals_alone(srv):
    reqs = _stream(srv, 48, 600)
    assert {r.prec for r in reqs} == {"fp64", "bf16x6"}
    # a 24 MB budget for requests in flight on top of the four lanes' workspaces
    ws = sum(2 * srv.lane_workspace_bytes(DEV, p, n_max=600) for p in ("fp64", "bf16x6"))
    cap = ws + 24e6
    server = srv.Server(DEV, mem_cap=cap, lanes_per_prec=2, max_batch=8, keep_results=True,
                        precisions=("fp64", "bf16x6"), n_max=600)
    done = server.run(reqs)
    torch.cuda.synchronize()
    assert len(done) == len(reqs)
    assert server.ws_total <= ws * (1 + 1e-9) + 4096
    assert server.peak_bytes <= cap
    batches = {r.t_admit for r in done}
    assert len(batches) > 2          # requests were admitted over several batches
    for r in done:
        assert int(r.info.item()) == 0
        _, alone, info = srv.solve_alone(r, DEV)
        assert int(info.item()) == 0
        assert torch.equal(r.sigma_bar, alone), (r.rid, r.n, r.prec)
    server.close()


def test_served_matches_oracle(srv):
    reqs = [r for r in _stream(srv, 30, 300, seed=9) if r.prec == "fp64"][:6]
    server = srv.Server(DEV, mem_cap=4e9, lanes_per_prec=2, max_batch=4, keep_results=True, n_max=300)
    done = server.run(reqs, realtime=False)
    torch.cuda.synchronize()
    for r in done:
        S, Lb = srv.build_inputs(r, DEV)
        Sn = S.cpu().numpy()
        L, info = oracle.chol_unblocked(Sn)
        assert info == 0
        ref = oracle.chol_unblocked_rev(L, np.tril(Lb.cpu().numpy()))
        assert oracle.rel_fro(r.sigma_bar.cpu().numpy(), ref) <= 1e-11
    server.close()


def test_admission_with_tight_budget(srv):
    reqs = _stream(srv, 12, 400, seed=11)
    ws = sum(srv.lane_workspace_bytes(DEV, p, n_max=400) for p in ("fp64", "bf16x6"))
    cap = ws + 4096 + max(srv.request_bytes(r.n, r.prec) for r in reqs) * 1.01
    server = srv.Server(DEV, mem_cap=cap, lanes_per_prec=1, max_batch=16, precisions=("fp64", "bf16x6"),
                        n_max=400)
    done = server.run(reqs, realtime=False)
    assert len(done) == len(reqs)
    assert server.peak_bytes <= cap
    s = srv.summarize(done)
    assert s["p99_ms"] >= s["p50_ms"] > 0
    server.close()


def test_large_requests_served_equal_alone(srv):
    # sizes up to the stream's maximum, where the split-BF16 passes take
    # 256-wide blocks and the products split K: served bitwise equal to alone
    sizes = [4096, 3000, 2100, 4096, 1500, 2600, 3500, 1100]
    reqs = [srv.Request(rid=i, t_arrival=0.0, n=n, prec=("bf16x6" if i % 2 == 0 else "fp64"), seed=700 + i)
            for i, n in enumerate(sizes)]
    ws = sum(2 * srv.lane_workspace_bytes(DEV, p, n_max=4096) for p in ("fp64", "bf16x6"))
    server = srv.Server(DEV, mem_cap=ws + 3e9, lanes_per_prec=2, max_batch=3, keep_results=True,
                        precisions=("fp64", "bf16x6"), n_max=4096)
    done = server.run(reqs, realtime=False)
    torch.cuda.synchronize()
    assert len(done) == len(reqs)
    assert server.peak_bytes <= ws + 3e9
    for r in done:
        assert int(r.info.item()) == 0
        _, alone, info = srv.solve_alone(r, DEV)
        assert int(info.item()) == 0
        assert torch.equal(r.sigma_bar, alone), (r.rid, r.n, r.prec)
    server.close()
