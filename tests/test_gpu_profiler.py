"""The kernel profiler (cd_profile_enable / cd_profile_timeline / cd_profile_read):
measurement support of the library, checked for consistency, not for speed.

A split-BF16 reverse pass runs its bulk products on the handle's side stream,
so its timeline must show launches on both streams; every record has
start <= end, starts are measured from the first launch, and the per-kind
totals of cd_profile_read agree with the timeline's own sums.  Profiling
changes no result: the profiled pass is bitwise equal to an unprofiled one.
"""
import collections

import numpy as np
import pytest

from paper_1602_07527_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_07527_gb300 import native
    return native


def test_timeline_and_totals(nat):
    n, nb = 1024, 256
    L = torch.tensor(np.tril(W.wishart(n, 7)), device=DEV)
    nat.chol_fwd(L)
    Lb = torch.tensor(W.lbar(n, 7), device=DEV)
    ref = Lb.clone()
    nat.chol_rev(L, ref, nb=nb, prec="bf16x6")
    torch.cuda.synchronize()
    nat.profile_read()                       # drop anything recorded before
    nat.profile_enable(True)
    X = Lb.clone()
    nat.chol_rev(L, X, nb=nb, prec="bf16x6")
    tl = nat.profile_timeline()
    stats = nat.profile_read()
    nat.profile_enable(False)
    assert torch.equal(X, ref)              # profiling changes no result
    assert len(tl) > 0
    assert tl[0]["start_ms"] == 0.0
    assert all(r["end_ms"] >= r["start_ms"] >= 0.0 for r in tl)
    assert {r["stream"] for r in tl} == {0, 1}
    sums = collections.Counter()
    counts = collections.Counter()
    for r in tl:
        sums[r["name"]] += r["end_ms"] - r["start_ms"]
        counts[r["name"]] += 1
    assert {k["name"] for k in stats} == set(counts)
    for k in stats:
        assert k["launches"] == counts[k["name"]]
        assert k["ms"] == pytest.approx(sums[k["name"]], rel=1e-3, abs=1e-3)
    assert nat.profile_timeline() == []     # cd_profile_read cleared the record
