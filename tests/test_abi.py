"""CPU checks of the C ABI: the library loads, exports every entry point the
header declares, and rejects bad arguments on the host without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "libcholdiff.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1602_07527_gb300 import build_native
    path = build_native.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cd_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_operations():
    names = declared_functions()
    for required in ("cd_chol_fwd", "cd_chol_rev", "cd_chol_fwd_sens", "cd_chol_fwd_batched",
                     "cd_chol_rev_batched", "cd_chol_fwd_sens_batched", "cd_create", "cd_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol(lib):
    from paper_1602_07527_gb300 import native
    assert sorted(native.exported_symbols()) == declared_functions()


def test_host_argument_checks_without_gpu(lib):
    vp = ctypes.c_void_p
    lib.cd_chol_rev.argtypes = [vp, ctypes.c_int, vp, ctypes.c_longlong, vp, ctypes.c_longlong, vp, vp]
    lib.cd_chol_fwd.argtypes = [vp, ctypes.c_int, vp, ctypes.c_longlong, vp, vp, vp]
    # NULL handle
    assert lib.cd_chol_rev(None, 4, None, 4, None, 4, None, None) == -1
    assert lib.cd_chol_fwd(None, 4, None, 4, None, None, None) == -1
    lib.cd_version.restype = ctypes.c_char_p
    assert b"libcholdiff" in lib.cd_version()
    lib.cd_destroy.argtypes = [vp]
    assert lib.cd_destroy(None) == 0


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_1602_07527_gb300 import native
    monkeypatch.setattr(native, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(native, "_lib", None)
    with pytest.raises(ImportError):
        native.lib()
