"""The C-ABI library loads without a GPU, exports every entry point that
include/corr.h declares, and rejects bad arguments before touching a device."""

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(corr_\w+)\s*\(", src, flags=re.M))
    return names


@pytest.fixture(scope="module")
def built():
    from paper_1102_0148_gb300 import build
    return build.build()


def test_every_declared_symbol_is_exported(built):
    decl = _declared()
    assert {"corr_create", "corr_push", "corr_dump", "corr_destroy"} <= decl
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (corr_\w+)", out))
    missing = decl - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_binding_covers_declarations(built, lib):
    assert _declared() <= set(lib.EXPORTED)


def test_argument_validation_without_device(lib):
    for N, K, dt in [(0, 512, 0), (lib.CORR_MAX_N + 1, 512, 0), (44, 500, 0), (44, 8, 0),
                     (44, 8192, 0), (44, 512, 7), (44, 512, -1)]:
        with pytest.raises(lib.CorrError) as ei:
            lib.corr_create(N, K, dt)
        assert ei.value.code == lib.CORR_EINVAL
    assert "K=500" in _last_create_error(lib, 44, 500)


def _last_create_error(lib, N, K):
    try:
        lib.corr_create(N, K, 0)
    except lib.CorrError:
        pass
    return lib.corr_last_error(None)


def test_null_handle_is_rejected(lib):
    import ctypes
    L = lib._lib
    assert L.corr_push(None, None, 0) == lib.CORR_EINVAL
    assert L.corr_dump(None, None, None, 0) == lib.CORR_EINVAL
    assert L.corr_sync(None) == lib.CORR_EINVAL
    assert L.corr_set_chunk(None, 128) == lib.CORR_EINVAL
    assert L.corr_info(None, None, None, None, None, None) == lib.CORR_EINVAL
    L.corr_destroy(None)
    assert isinstance(L.corr_last_error(None), bytes)
    assert L.corr_profile_read(None, None, None, 0) == lib.CORR_EINVAL
    del ctypes
