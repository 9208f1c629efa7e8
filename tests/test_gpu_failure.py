"""Device-side failure detection without faulting the GPU: a bounded wait
that runs out reports CD_ETIMEOUT through the handle's error word, and the
context stays usable (a normal call afterwards is correct)."""
import numpy as np
import pytest

import oracle
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


def test_bounded_wait_reports_timeout_and_context_survives(nat):
    h = nat.Handle(DEV)
    try:
        assert nat.device_error_of(h) == nat.CD_OK
        nat.debug_wait_timeout(DEV, handle_=h)
        torch.cuda.synchronize()
        assert nat.device_error_of(h) == nat.CD_ETIMEOUT
        assert nat.device_error_of(h) == nat.CD_OK          # reading clears the word
        # the context still computes correctly, on the same handle, in both precisions
        n = 300
        S = W.wishart(n, 1500)
        L, _ = oracle.chol_unblocked(S)
        Lb = W.lbar(n, 1500)
        ref = oracle.chol_unblocked_rev(L, Lb)
        for prec, tol in (("fp64", 1e-11), ("bf16x6", 1e-6)):
            Ab = torch.tensor(Lb, device=DEV)
            nat.chol_rev(torch.tensor(L, device=DEV), Ab, nb=64, prec=prec, handle_=h)
            torch.cuda.synchronize()
            assert oracle.rel_fro(Ab.cpu().numpy(), ref) <= tol
        assert nat.device_error_of(h) == nat.CD_OK
    finally:
        h.close()
