"""cd_chol_rev_noalloc: the reverse pass for callers that cannot allocate.

Callers running where device allocation is not allowed (inside an
allocator's callbacks, or in an embedding that owns all device memory) use
this entry point; its scratch is a fixed array inside the library.  These
checks call it through the C ABI and compare it with cd_chol_rev, the
allocating entry point, on two calls in a row: the second call runs on the
scratch contents the first one left behind.  This file is collected last so
that a run stopping at the first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1602_07527_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-11
DEV = "cuda:0"


@pytest.fixture(scope="module")
def native():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1602_07527_gb300 import native as nat
    return nat


def _noalloc(nat, L, Abar, nb=0, out=0):
    n = L.shape[0]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return nat.lib().cd_chol_rev_noalloc(n, ctypes.c_void_p(L.data_ptr()), L.stride(0),
                                         ctypes.c_void_p(Abar.data_ptr()), Abar.stride(0), nb, out, stream)


def _case(n, seed):
    S = W.se(n, seed, 3, 0.3, 1e-2)
    L, info = oracle.chol_unblocked(S)
    assert info == 0
    return L, W.lbar(n, seed)


def test_noalloc_matches_allocating_entry_point_twice(native):
    # (n, nb, out): the largest allowed problem with its default block size
    # (the scratch is fullest there), a smaller one at nb = 64, a column-by-
    # column one at nb = 1 and the symmetric output form
    for n, nb, out, seed in ((2048, 128, 0, 30), (1500, 0, 0, 31), (700, 64, 1, 32), (40, 1, 0, 33)):
        L, Lb = _case(n, seed)
        Ld = torch.tensor(L, device=DEV)
        ref = torch.tensor(Lb, device=DEV)
        native.chol_rev(Ld, ref, nb=nb, out="sym" if out else "tril")  # allocating entry point
        got = torch.tensor(Lb, device=DEV)
        assert _noalloc(native, Ld, got, nb=nb, out=out) == 0
        torch.cuda.synchronize()
        g, r = got.cpu().numpy(), ref.cpu().numpy()
        if out:
            assert np.array_equal(g, g.T)
            g, r = np.tril(g), np.tril(r)
        err = oracle.rel_fro(g, r)
        assert err <= TOL, (n, nb, out, err)


def test_noalloc_matches_oracle_at_its_limit(native):
    n = 2048
    L, Lb = _case(n, 34)
    got = torch.tensor(Lb, device=DEV)
    assert _noalloc(native, torch.tensor(L, device=DEV), got, nb=128) == 0
    torch.cuda.synchronize()
    err = oracle.rel_fro(got.cpu().numpy(), oracle.chol_unblocked_rev(L, Lb))
    assert err <= TOL, err


def test_noalloc_rejects_sizes_beyond_its_scratch(native):
    n = 2049
    L = torch.eye(n, dtype=torch.float64, device=DEV)
    Ab = torch.zeros_like(L)
    assert _noalloc(native, L, Ab) == native.CD_ESCRATCH
    assert _noalloc(native, L[:4, :4], Ab[:4, :4], nb=129) == native.CD_EINVAL
    torch.cuda.synchronize()
    assert torch.count_nonzero(Ab).item() == 0
