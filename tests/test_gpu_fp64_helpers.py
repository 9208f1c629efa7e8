"""The diagonal factorisation's hand-written FP64 reciprocal and square root.

k_potrf_cluster takes each pivot's reciprocal (an FP32 seed refined by one
Householder step of order 2) and the panel's square roots and reciprocal
square roots (Goldschmidt's iteration from an FP32 seed) instead of FP64
division and square root.  These checks run them on values spanning every
exponent of the normal range and edge values (powers of two, values just
below them, the largest and smallest normals), against references computed
in extended precision (numpy longdouble: 64 or 113 significand bits), and
against CUDA's own correctly rounded division and square root: the error
bound asserted is one unit in the last place (faithful rounding).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ULP_BOUND = 1.0
DEV = "cuda:0"


@pytest.fixture(scope="module")
def native():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_07527_gb300 import native as nat
    return nat


def _inputs():
    g = np.random.default_rng(21)
    mant = 1.0 + g.random(200000)
    expo = g.integers(-1021, 1022, mant.size)
    x = np.ldexp(mant, expo)
    edges = [1.0, 2.0, 4.0, 0.5, 3.0, np.nextafter(2.0, 0.0), np.nextafter(1.0, 0.0), np.nextafter(1.0, 2.0),
             np.finfo(np.float64).max, np.finfo(np.float64).tiny, np.nextafter(np.finfo(np.float64).tiny, 1.0),
             2.0 ** 1022, 2.0 ** 1023, 2.0 ** -1022, 2.0 ** -1021, 1e-300, 1e300, 7.0, 1.0 / 3.0]
    for e in range(-1022, 1024, 7):
        edges += [2.0 ** e, np.nextafter(2.0 ** e, 0.0) if e > -1022 else 2.0 ** e]
    return np.concatenate([x, np.array(edges, dtype=np.float64)])


def _ulps(y, ref):
    r64 = ref.astype(np.float64)
    sp = np.spacing(np.abs(r64))
    return np.abs(y.astype(np.longdouble) - ref) / sp.astype(np.longdouble)


def test_reciprocal_and_square_roots_within_one_ulp(native):
    x = _inputs()
    xt = torch.tensor(x, device=DEV)
    recip, sq, rsq = (t.cpu().numpy() for t in native.fp64_helpers(xt))
    xl = x.astype(np.longdouble)
    ref_recip = 1.0 / xl
    ref_sq = np.sqrt(xl)
    ref_rsq = 1.0 / np.sqrt(xl)
    # 1 / x for x near the top of the range is subnormal: the helper takes the
    # platform's division there, which is checked with the rest below
    normal = np.abs(ref_recip.astype(np.float64)) >= np.finfo(np.float64).tiny
    e_recip = _ulps(recip[normal], ref_recip[normal]).max()
    e_sq = _ulps(sq, ref_sq).max()
    e_rsq = _ulps(rsq, ref_rsq).max()
    # CUDA's own division and square root, as a check of the references
    cuda_recip = (1.0 / xt).cpu().numpy()
    cuda_sq = torch.sqrt(xt).cpu().numpy()
    assert _ulps(cuda_recip[normal], ref_recip[normal]).max() <= 0.5 + 1e-12
    assert _ulps(cuda_sq, ref_sq).max() <= 0.5 + 1e-12
    print(f"max ulps: recip {float(e_recip):.3f} sqrt {float(e_sq):.3f} rsqrt {float(e_rsq):.3f}; "
          f"bit-equal to CUDA: recip {np.mean(recip == cuda_recip):.4f} sqrt {np.mean(sq == cuda_sq):.4f}")
    assert e_recip <= ULP_BOUND, e_recip
    assert e_sq <= ULP_BOUND, e_sq
    assert e_rsq <= ULP_BOUND, e_rsq


def test_special_inputs_take_the_platform_path(native):
    x = torch.tensor([5e-324, 1e-310, np.inf], dtype=torch.float64, device=DEV)
    recip, sq, rsq = native.fp64_helpers(x)
    assert torch.equal(recip, 1.0 / x)
    assert torch.equal(sq, torch.sqrt(x))
