"""The C-ABI library builds, loads and exports every entry point include/pspec.h declares.

No compute call is made here (no GPU is needed): only symbol lookup and the pure host
helpers pspec_strerror / pspec_version / pspec_kernel_name.
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pspec.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pspec_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1704_02357_gb300 import build as B
    B.build()
    from paper_1704_02357_gb300 import pspec
    return pspec.load()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("pspec_paint", "pspec_multipoles", "pspec_wedges", "pspec_create", "pspec_destroy",
                 "pspec_strerror", "pspec_last_error", "pspec_workspace_size"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    import ctypes
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_binding_declares_every_symbol(lib):
    from paper_1704_02357_gb300 import pspec
    bound = {n for n, _, _ in pspec.SIGNATURES}
    assert set(declared_symbols()) == bound


def test_host_only_helpers(lib):
    assert lib.pspec_strerror(0) == b"ok"
    assert lib.pspec_strerror(6) == b"unsupported"
    assert b"sm_103a" in lib.pspec_version()
    assert lib.pspec_kernel_name(7) == b"bin_x"


def test_missing_library_fails_loudly(tmp_path):
    from paper_1704_02357_gb300 import pspec
    with pytest.raises(ImportError):
        saved = pspec._lib
        pspec._lib = None
        try:
            pspec.load(str(tmp_path / "nope.so"))
        finally:
            pspec._lib = saved
