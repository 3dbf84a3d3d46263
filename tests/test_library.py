"""Host-side checks of the C ABI library (no GPU needed): it builds for
sm_103a, loads, and exports every entry point that include/mkf.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mkf.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:mkf_status|void|const char\*)\s+(mkf_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2002_06295_gb300 import build_ext
    return build_ext.build()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("mkf_load_geometry", "mkf_bin_hits", "mkf_build_tracks", "mkf_fit_tracks", "mkf_fit_backward",
              "mkf_fit_tracks_adjoint", "mkf_dedup_tracks", "mkf_create", "mkf_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2002_06295_gb300 import _lib
    assert set(declared_symbols()) <= set(_lib.SIGNATURES)


def test_no_fallback_without_library(tmp_path, monkeypatch):
    """The binding raises when libmkf.so is absent; there is no CPU path."""
    from paper_2002_06295_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError):
        _lib.load()


def test_create_without_gpu_fails_cleanly(libpath):
    """On a machine without a GPU, mkf_create reports an error instead of crashing."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    lib = ctypes.CDLL(libpath)
    lib.mkf_create.restype = ctypes.c_int
    h = ctypes.c_void_p()
    rc = lib.mkf_create(ctypes.byref(h), 0)
    assert rc != 0 and not h.value
