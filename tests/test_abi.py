"""The C ABI library builds, loads and exports every declared entry point
(no compute call: these run without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2406_11185_gb300 import adft

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "adft.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(adft_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(adft.LIB_PATH):
        from paper_2406_11185_gb300 import build
        build.build()
    return adft.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "adft_jk_build" in names and "adft_basis_create" in names
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(adft.EXPORTED) == sorted(names)


def test_status_strings_and_version(lib):
    assert adft.status_string(0) == "ok"
    assert "symmetric" in adft.status_string(adft.ADFT_ERR_ASYM_D)
    assert lib.adft_version().decode().startswith("adft")


def test_null_arguments_rejected_without_gpu(lib):
    out = ctypes.c_void_p()
    assert lib.adft_basis_create(None, 0, None, 0, 1, ctypes.byref(out)) == adft.ADFT_ERR_ARG
    assert lib.adft_basis_create(None, 0, None, 0, 1, None) == adft.ADFT_ERR_ARG
    assert lib.adft_jk_build(None, None, None, None, None) == adft.ADFT_ERR_ARG
    n = ctypes.c_int()
    assert lib.adft_basis_nbf(None, ctypes.byref(n)) == adft.ADFT_ERR_ARG
    assert len(adft.last_error()) > 0
