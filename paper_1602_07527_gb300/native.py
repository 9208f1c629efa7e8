"""ctypes binding of libcholdiff (include/libcholdiff.h).

Argument marshalling only: every matrix operation runs in the CUDA library.
Tensors must be CUDA float64, 2-D, row-major with unit column stride (the
row stride is passed as the leading dimension).  Calls are enqueued on the
current torch CUDA stream of the tensor's device and return without waiting.
There is no CPU fallback: if the library is missing the first call raises.
"""
import ctypes
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcholdiff.so")

CD_OK, CD_EINVAL, CD_ENOMEM, CD_ECUDA, CD_ETIMEOUT, CD_ESCRATCH = 0, -1, -2, -3, -4, -5
_ERR = {CD_EINVAL: "invalid argument", CD_ENOMEM: "workspace allocation failed",
        CD_ECUDA: "CUDA error", CD_ETIMEOUT: "device-side wait timed out",
        CD_ESCRATCH: "problem larger than the fixed scratch of cd_chol_rev_noalloc"}
PREC = {"fp64": 0, "bf16x3": 1, "bf16x6": 2, "fixed4": 3}
DIAG = {"auto": 0, "level2": 1, "symbolic": 2}
OUT = {"tril": 0, "sym": 1}


class CholDiffError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {_ERR.get(code, 'error')} (code {code})")
        self.code = code


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_longlong), ("ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


class LaunchRec(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("stream", ctypes.c_int), ("start_ms", ctypes.c_double),
                ("end_ms", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int), ("prec", ctypes.c_int), ("out", ctypes.c_int), ("diag", ctypes.c_int),
                ("uplo", ctypes.c_int), ("spin_limit", ctypes.c_longlong)]


_lib = None
_lock = threading.Lock()
_handles = {}

_vp = ctypes.c_void_p
_ll = ctypes.c_longlong
_i = ctypes.c_int


def lib():
    """Load libcholdiff.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        L.cd_create.argtypes = [P(_vp), _i]
        L.cd_destroy.argtypes = [_vp]
        L.cd_options_default.argtypes = [P(Options)]
        L.cd_options_default.restype = None
        L.cd_workspace_size.argtypes = [_vp, _i, P(Options), P(ctypes.c_size_t)]
        L.cd_reserve.argtypes = [_vp, ctypes.c_size_t]
        L.cd_workspace_size_batched.argtypes = [_vp, _i, _vp, P(Options), P(ctypes.c_size_t)]
        L.cd_workspace_bytes.argtypes = [_vp, P(ctypes.c_size_t)]
        L.cd_chol_fwd.argtypes = [_vp, _i, _vp, _ll, P(Options), _vp, _vp]
        L.cd_chol_rev.argtypes = [_vp, _i, _vp, _ll, _vp, _ll, P(Options), _vp]
        L.cd_chol_fwd_sens.argtypes = [_vp, _i, _vp, _ll, _vp, _ll, P(Options), _vp]
        L.cd_chol_fwd_batched.argtypes = [_vp, _i, _vp, _vp, _vp, P(Options), _vp, _vp]
        L.cd_chol_rev_batched.argtypes = [_vp, _i, _vp, _vp, _vp, _vp, _vp, P(Options), _vp]
        L.cd_chol_fwd_sens_batched.argtypes = [_vp, _i, _vp, _vp, _vp, _vp, _vp, P(Options), _vp]
        L.cd_chol_fwd_and_sens.argtypes = [_vp, _i, _vp, _ll, _vp, _ll, P(Options), _vp, _vp]
        L.cd_chol_fwd_and_sens_batched.argtypes = [_vp, _i, _vp, _vp, _vp, _vp, _vp, P(Options), _vp, _vp]
        L.cd_chol_jacobian.argtypes = [_vp, _i, _vp, _ll, _vp, _vp]
        L.cd_get_last_device_error.argtypes = [_vp, P(_i)]
        L.cd_debug_fp64_probe.argtypes = [_vp, _i, _ll, _vp, P(ctypes.c_double)]
        L.cd_debug_fp64_helpers.argtypes = [_vp, _i, _vp, _vp, _vp, _vp, _vp]
        L.cd_launch_count.argtypes = [_vp]
        L.cd_launch_count.restype = _ll
        L.cd_version.restype = ctypes.c_char_p
        L.cd_profile_enable.argtypes = [_vp, _i]
        L.cd_profile_read.argtypes = [_vp, P(KernelStat), _i, P(_i)]
        L.cd_profile_timeline.argtypes = [_vp, P(LaunchRec), _i, P(_i)]
        L.cd_chol_rev_noalloc.argtypes = [_i, _vp, _ll, _vp, _ll, _i, _i, _vp]
        L.cd_set_priorities.argtypes = [_vp, _i, _i]
        L.cd_debug_wait_timeout.argtypes = [_vp, _vp]
        L.cd_mixed_gemm_debug.argtypes = [_vp, _i, _i, _i, _vp, _ll, _vp, _ll, _vp, _ll, _i, _i, _vp]
        _lib = L
    return _lib


def exported_symbols():
    """Names of every entry point the header declares (for load checks)."""
    return ["cd_create", "cd_destroy", "cd_options_default", "cd_workspace_size", "cd_reserve",
            "cd_chol_fwd", "cd_chol_rev", "cd_chol_fwd_sens", "cd_chol_fwd_batched",
            "cd_chol_rev_batched", "cd_chol_fwd_sens_batched", "cd_get_last_device_error",
            "cd_launch_count", "cd_version", "cd_profile_enable", "cd_profile_read", "cd_profile_timeline",
            "cd_chol_rev_noalloc", "cd_mixed_gemm_debug", "cd_set_priorities", "cd_debug_wait_timeout",
            "cd_chol_fwd_and_sens", "cd_chol_fwd_and_sens_batched", "cd_chol_jacobian", "cd_debug_fp64_probe",
            "cd_workspace_size_batched", "cd_workspace_bytes", "cd_debug_fp64_helpers"]


def handle(device=None):
    """The library handle of a CUDA device (created on first use, kept for the process)."""
    dev = torch.cuda.current_device() if device is None else torch.device(device).index
    if dev is None:
        dev = torch.cuda.current_device()
    h = _handles.get(dev)
    if h is None:
        with _lock:
            h = _handles.get(dev)
            if h is None:
                hp = _vp()
                rc = lib().cd_create(ctypes.byref(hp), dev)
                if rc != CD_OK:
                    raise CholDiffError(rc, "cd_create")
                h = hp.value
                _handles[dev] = h
    return h


class Handle:
    """An independent library handle (own workspace, streams and counters).

    Calls that may run concurrently on different streams need different
    handles; the module-level functions use one shared handle per device.
    """

    def __init__(self, device=None):
        dev = torch.cuda.current_device() if device is None else torch.device(device).index
        hp = _vp()
        rc = lib().cd_create(ctypes.byref(hp), dev)
        if rc != CD_OK:
            raise CholDiffError(rc, "cd_create")
        self.ptr = hp.value
        self.device = dev

    def set_priorities(self, chain, bulk):
        """CUDA priorities of the handle's internal streams (lower = higher priority)."""
        _check(lib().cd_set_priorities(_vp(self.ptr), int(chain), int(bulk)), "cd_set_priorities")

    def close(self):
        if self.ptr:
            lib().cd_destroy(_vp(self.ptr))
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _h(handle_, device):
    if handle_ is None:
        return handle(device)
    return handle_.ptr if isinstance(handle_, Handle) else handle_


UPLO = {"lower": 0, "upper": 1}


def options(nb=0, prec="fp64", out="tril", spin_limit=0, diag="auto", uplo="lower"):
    o = Options()
    lib().cd_options_default(ctypes.byref(o))
    o.nb = int(nb)
    o.uplo = UPLO[uplo] if isinstance(uplo, str) else int(uplo)
    o.diag = DIAG[diag] if isinstance(diag, str) else int(diag)
    o.prec = PREC[prec] if isinstance(prec, str) else int(prec)
    o.out = OUT[out] if isinstance(out, str) else int(out)
    o.spin_limit = int(spin_limit)
    return o


def _mat(t, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    if t.dim() != 2 or t.shape[0] != t.shape[1]:
        raise ValueError(f"{name} must be square 2-D, got {tuple(t.shape)}")
    if t.shape[0] > 0 and (t.stride(1) != 1 or t.stride(0) < t.shape[0]):
        raise ValueError(f"{name} must be row-major with unit column stride")
    return t.shape[0], max(1, t.stride(0))


def _stream(dev):
    return _vp(torch.cuda.current_stream(dev).cuda_stream)


def _check(rc, what):
    if rc != CD_OK:
        raise CholDiffError(rc, what)


def chol_fwd(A, nb=0, prec="fp64", info=None, handle_=None, uplo="lower"):
    """In place: tril(A) = tril(Sigma) -> L (Sec. 4.2 chol_blocked).

    Returns the device int32 tensor holding LAPACK-style info (0 = success,
    j = first non-positive pivot, 1-based).
    """
    n, lda = _mat(A, "A")
    dev = A.device
    if info is None:
        info = torch.zeros(1, dtype=torch.int32, device=dev)
    o = options(nb, prec, uplo=uplo)
    _check(lib().cd_chol_fwd(_h(handle_, dev), n, _vp(A.data_ptr()), lda, ctypes.byref(o), _stream(dev),
                             _vp(info.data_ptr())), "cd_chol_fwd")
    return info


def chol_rev(L, Abar, nb=0, prec="fp64", out="tril", handle_=None, diag="auto", uplo="lower"):
    """In place: tril(Abar) = L_bar -> tril(Sigma_bar) (Sec. 4.2 chol_blocked_rev)."""
    n, ldl = _mat(L, "L")
    n2, lda = _mat(Abar, "Abar")
    if n != n2 or L.device != Abar.device:
        raise ValueError("L and Abar must have the same size and device")
    o = options(nb, prec, out, diag=diag, uplo=uplo)
    _check(lib().cd_chol_rev(_h(handle_, L.device), n, _vp(L.data_ptr()), ldl, _vp(Abar.data_ptr()), lda,
                             ctypes.byref(o), _stream(L.device)), "cd_chol_rev")
    return Abar


def chol_fwd_sens(L, Adot, nb=0, prec="fp64", handle_=None, diag="auto", uplo="lower"):
    """In place: tril(Adot) = tril(Sigma_dot) -> L_dot (Sec. 4.2 chol_blocked_fwd)."""
    n, ldl = _mat(L, "L")
    n2, lda = _mat(Adot, "Adot")
    if n != n2 or L.device != Adot.device:
        raise ValueError("L and Adot must have the same size and device")
    o = options(nb, prec, diag=diag, uplo=uplo)
    _check(lib().cd_chol_fwd_sens(_h(handle_, L.device), n, _vp(L.data_ptr()), ldl, _vp(Adot.data_ptr()), lda,
                                  ctypes.byref(o), _stream(L.device)), "cd_chol_fwd_sens")
    return Adot


def chol_fwd_and_sens(A, Adot, nb=0, prec="fp64", info=None, handle_=None, diag="auto", uplo="lower"):
    """In place, in one pass: tril(A) = tril(Sigma) -> L and
    tril(Adot) = tril(Sigma_dot) -> L_dot (Sec. 4.1-4.2: the forward-mode
    updates accumulated in the factorisation's loop).  Returns the info tensor."""
    n, lda = _mat(A, "A")
    n2, ldd = _mat(Adot, "Adot")
    if n != n2 or A.device != Adot.device:
        raise ValueError("A and Adot must have the same size and device")
    dev = A.device
    if info is None:
        info = torch.zeros(1, dtype=torch.int32, device=dev)
    o = options(nb, prec, diag=diag, uplo=uplo)
    _check(lib().cd_chol_fwd_and_sens(_h(handle_, dev), n, _vp(A.data_ptr()), lda, _vp(Adot.data_ptr()), ldd,
                                      ctypes.byref(o), _stream(dev), _vp(info.data_ptr())), "cd_chol_fwd_and_sens")
    return info


def chol_jacobian(L, handle_=None):
    """Eq. delements: the n x n x n x n tensor J[i, j, k, l] = dL_ij / dSigma_kl
    (i >= j, k >= l; tied pairs Sigma_kl = Sigma_lk counted once), computed on
    the device from the factor L.  Theta(n^4) memory: for analysis."""
    n, ldl = _mat(L, "L")
    J = torch.empty((n, n, n, n), dtype=torch.float64, device=L.device)
    _check(lib().cd_chol_jacobian(_h(handle_, L.device), n, _vp(L.data_ptr()), ldl, _vp(J.data_ptr()),
                                  _stream(L.device)), "cd_chol_jacobian")
    return J


def _arrays(mats, name):
    ns, lds, ptrs = [], [], []
    for t in mats:
        n, ld = _mat(t, name)
        ns.append(n)
        lds.append(ld)
        ptrs.append(t.data_ptr())
    b = len(mats)
    return (b, (_i * b)(*ns), (_ll * b)(*lds), (_vp * b)(*ptrs), ns)


def chol_fwd_batched(As, nb=0, prec="fp64", info=None, handle_=None, uplo="lower"):
    b, n, ld, p, _ = _arrays(As, "A")
    if b == 0:
        return info
    dev = As[0].device
    if info is None:
        info = torch.zeros(b, dtype=torch.int32, device=dev)
    o = options(nb, prec, uplo=uplo)
    _check(lib().cd_chol_fwd_batched(_h(handle_, dev), b, n, p, ld, ctypes.byref(o), _stream(dev),
                                     _vp(info.data_ptr())), "cd_chol_fwd_batched")
    return info


def chol_rev_batched(Ls, Abars, nb=0, prec="fp64", out="tril", handle_=None, diag="auto", uplo="lower"):
    b, n, ldl, pl, ns = _arrays(Ls, "L")
    b2, n2, lda, pa, ns2 = _arrays(Abars, "Abar")
    if b != b2 or ns != ns2:
        raise ValueError("L and Abar lists must match")
    if b == 0:
        return Abars
    dev = Ls[0].device
    o = options(nb, prec, out, diag=diag, uplo=uplo)
    _check(lib().cd_chol_rev_batched(_h(handle_, dev), b, n, pl, ldl, pa, lda, ctypes.byref(o), _stream(dev)),
           "cd_chol_rev_batched")
    return Abars


def chol_fwd_sens_batched(Ls, Adots, nb=0, prec="fp64", handle_=None, diag="auto", uplo="lower"):
    b, n, ldl, pl, ns = _arrays(Ls, "L")
    b2, n2, lda, pa, ns2 = _arrays(Adots, "Adot")
    if b != b2 or ns != ns2:
        raise ValueError("L and Adot lists must match")
    if b == 0:
        return Adots
    dev = Ls[0].device
    o = options(nb, prec, diag=diag, uplo=uplo)
    _check(lib().cd_chol_fwd_sens_batched(_h(handle_, dev), b, n, pl, ldl, pa, lda, ctypes.byref(o), _stream(dev)),
           "cd_chol_fwd_sens_batched")
    return Adots


def chol_fwd_and_sens_batched(As, Adots, nb=0, prec="fp64", info=None, handle_=None, diag="auto", uplo="lower"):
    b, n, lda, pa, ns = _arrays(As, "A")
    b2, n2, ldd, pd, ns2 = _arrays(Adots, "Adot")
    if b != b2 or ns != ns2:
        raise ValueError("A and Adot lists must match")
    if b == 0:
        return info
    dev = As[0].device
    if info is None:
        info = torch.zeros(b, dtype=torch.int32, device=dev)
    o = options(nb, prec, diag=diag, uplo=uplo)
    _check(lib().cd_chol_fwd_and_sens_batched(_h(handle_, dev), b, n, pa, lda, pd, ldd, ctypes.byref(o),
                                              _stream(dev), _vp(info.data_ptr())), "cd_chol_fwd_and_sens_batched")
    return info


def mixed_gemm_debug(A, B, C, prec="bf16x3", lower=False):
    """C = A B^T through the split-BF16 tensor-core product of the mixed path."""
    for t, nm in ((A, "A"), (B, "B"), (C, "C")):
        if not t.is_cuda or t.dtype != torch.float64 or t.dim() != 2 or t.stride(1) != 1:
            raise TypeError(f"{nm} must be a row-major CUDA float64 matrix")
    M, K = A.shape
    N = B.shape[0]
    if B.shape[1] != K or tuple(C.shape) != (M, N):
        raise ValueError("shape mismatch")
    _check(lib().cd_mixed_gemm_debug(handle(A.device), M, N, K, _vp(A.data_ptr()), A.stride(0), _vp(B.data_ptr()),
                                     B.stride(0), _vp(C.data_ptr()), C.stride(0), PREC[prec], 1 if lower else 0,
                                     _stream(A.device)), "cd_mixed_gemm_debug")
    return C


def fp64_probe(kind="dfma", iters=200000, device=None):
    """Launch the FP64 peak probe (kind "dfma" or "dmma") on the current stream;
    returns the floating-point operations it performs."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    fl = ctypes.c_double(0.0)
    _check(lib().cd_debug_fp64_probe(handle(dev), 0 if kind == "dfma" else 1, ctypes.c_longlong(iters), _stream(dev),
                                     ctypes.byref(fl)), "cd_debug_fp64_probe")
    return fl.value


def fp64_helpers(x):
    """The diagonal factorisation's FP64 helpers on a CUDA float64 vector x > 0:
    returns (1/x, sqrt(x), 1/sqrt(x)) as computed on the device."""
    if not x.is_cuda or x.dtype != torch.float64 or x.dim() != 1 or not x.is_contiguous():
        raise TypeError("x must be a contiguous CUDA float64 vector")
    r, s, q = torch.empty_like(x), torch.empty_like(x), torch.empty_like(x)
    _check(lib().cd_debug_fp64_helpers(handle(x.device), x.numel(), _vp(x.data_ptr()), _vp(r.data_ptr()),
                                       _vp(s.data_ptr()), _vp(q.data_ptr()), _stream(x.device)), "cd_debug_fp64_helpers")
    return r, s, q


def launch_count(device=None, handle_=None):
    return int(lib().cd_launch_count(_h(handle_, device)))


def device_error(device=None):
    code = _i()
    _check(lib().cd_get_last_device_error(handle(device), ctypes.byref(code)), "cd_get_last_device_error")
    return code.value


def debug_wait_timeout(device=None, handle_=None):
    """Run the tensor-core kernel with a load barrier that never completes (test hook)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    _check(lib().cd_debug_wait_timeout(_h(handle_, dev), _stream(dev)), "cd_debug_wait_timeout")


def device_error_of(handle_):
    code = _i()
    _check(lib().cd_get_last_device_error(_vp(handle_.ptr), ctypes.byref(code)), "cd_get_last_device_error")
    return code.value


def workspace_size(n, nb=0, prec="fp64", device=None, uplo="lower"):
    o = options(nb, prec, uplo=uplo)
    out = ctypes.c_size_t()
    _check(lib().cd_workspace_size(handle(device), int(n), ctypes.byref(o), ctypes.byref(out)),
           "cd_workspace_size")
    return out.value


def workspace_size_batched(ns, nb=0, prec="fp64", handle_=None, device=None):
    """Workspace bytes a batched call over the problem sizes ns may use (host arithmetic)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    arr = (ctypes.c_int * max(1, len(ns)))(*[int(x) for x in ns])
    o = options(nb, prec)
    b = ctypes.c_size_t(0)
    _check(lib().cd_workspace_size_batched(_h(handle_, dev), len(ns), ctypes.cast(arr, _vp), ctypes.byref(o),
                                           ctypes.byref(b)), "cd_workspace_size_batched")
    return b.value


def workspace_bytes(handle_=None, device=None):
    """Bytes of workspace the handle holds now."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    b = ctypes.c_size_t(0)
    _check(lib().cd_workspace_bytes(_h(handle_, dev), ctypes.byref(b)), "cd_workspace_bytes")
    return b.value


def reserve(nbytes, device=None, handle_=None):
    """Grow the handle's workspace to at least nbytes now."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    _check(lib().cd_reserve(_h(handle_, dev), int(nbytes)), "cd_reserve")


def profile_enable(on=True, device=None):
    """Record a CUDA event pair around every library kernel launch (see profile_read)."""
    _check(lib().cd_profile_enable(handle(device), 1 if on else 0), "cd_profile_enable")


def profile_read(device=None, max_kinds=64):
    """Synchronise, aggregate and clear the recorded launches: list of dicts per kernel kind."""
    arr = (KernelStat * max_kinds)()
    cnt = _i()
    _check(lib().cd_profile_read(handle(device), arr, max_kinds, ctypes.byref(cnt)), "cd_profile_read")
    return [dict(name=arr[k].name.decode(), launches=int(arr[k].launches), ms=float(arr[k].ms),
                 flops=float(arr[k].flops), bytes=float(arr[k].bytes)) for k in range(cnt.value)]


def profile_timeline(device=None, max_launches=200000):
    """The recorded launches one by one (not cleared; call before profile_read):
    list of dicts with name, stream (0 caller's, 1 side), start_ms, end_ms."""
    arr = (LaunchRec * max_launches)()
    cnt = _i()
    _check(lib().cd_profile_timeline(handle(device), arr, max_launches, ctypes.byref(cnt)), "cd_profile_timeline")
    return [dict(name=arr[k].name.decode(), stream=int(arr[k].stream), start_ms=float(arr[k].start_ms),
                 end_ms=float(arr[k].end_ms)) for k in range(cnt.value)]


def version():
    return lib().cd_version().decode()
