"""The C ABI library loads and exports every entry point include/*.h declares
(no GPU needed), and argument checks fail cleanly without a device."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(inc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", text, flags=re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "sizeof", "return"):
                names.add(name)
    return names


@pytest.fixture(scope="module")
def libmdx():
    from paper_2002_09561_gb300 import build

    build.build()
    return ctypes.CDLL(build.LIB)


def test_every_declared_symbol_is_exported(libmdx):
    declared = _declared()
    assert {"detect_sd", "detect_kbest", "detect_hybrid", "mdx_create"} <= declared
    for name in declared:
        assert hasattr(libmdx, name), name


def test_binding_lists_every_declared_symbol():
    from paper_2002_09561_gb300 import mdx

    assert set(mdx.EXPORTS) == _declared()


def test_strerror(libmdx):
    libmdx.mdx_strerror.restype = ctypes.c_char_p
    assert libmdx.mdx_strerror(0) == b"ok"
    assert libmdx.mdx_strerror(-1) == b"invalid argument"


def test_create_rejects_bad_sizes(libmdx):
    h = ctypes.c_void_p()
    assert libmdx.mdx_create(ctypes.byref(h), 0, 0, 4, 4) == -1
    assert libmdx.mdx_create(ctypes.byref(h), 0, 10, 2, 4) == -1
    assert libmdx.mdx_create(ctypes.byref(h), 0, 10, 128, 101) == -1
    assert libmdx.mdx_create(None, 0, 10, 4, 4) == -1


def test_null_context_is_rejected(libmdx):
    from paper_2002_09561_gb300 import mdx

    p = mdx.make_params(4, 4, 4)
    for name in ("detect_sd", "detect_kbest", "detect_hybrid"):
        f = getattr(libmdx, name)
        f.argtypes = [ctypes.c_void_p, ctypes.POINTER(mdx.Params)] + [ctypes.c_int] + [ctypes.c_void_p] * 8
        assert f(None, ctypes.byref(p), 1, *([None] * 8)) == -1


def test_measure_peaks_rejects_bad_arguments(libmdx):
    f = libmdx.mdx_measure_peaks
    f.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    out = (ctypes.c_double * 4)()
    assert f(0, None, None) == -1  # no output array
    assert f(-1, ctypes.cast(out, ctypes.c_void_p), None) == -1  # no such device


def test_no_cpu_fallback_without_library(tmp_path, monkeypatch):
    from paper_2002_09561_gb300 import mdx

    monkeypatch.setattr(mdx, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(mdx, "_lib", None)
    with pytest.raises(mdx.MdxError):
        mdx.lib()
