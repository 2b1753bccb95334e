"""The C ABI library builds, loads and exports every entry point that
include/rgg.h declares (no GPU needed: only argument checks that fail before
any CUDA call are exercised)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rgg.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rgg_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_28674_gb300 import build
    from paper_2603_28674_gb300 import rgg
    build.build()
    return rgg._lib()


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for call in ("rgg_roadmap_create", "rgg_upload_edges", "rgg_update_obstacles",
                 "rgg_classify", "rgg_fetch_labels"):
        assert call in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2603_28674_gb300 import rgg
    names = declared_functions()
    assert names, "no declarations parsed"
    for n in names:
        assert hasattr(lib, n), f"{n} declared in rgg.h but not exported"
    assert sorted(rgg.EXPORTS) == names


def test_status_strings(lib):
    from paper_2603_28674_gb300 import rgg
    for code in (rgg.RGG_OK, rgg.RGG_ERR_INVALID, rgg.RGG_ERR_OOM, rgg.RGG_ERR_CUDA,
                 rgg.RGG_ERR_TIMEOUT, rgg.RGG_ERR_STATE, 12345):
        s = lib.rgg_status_string(code)
        assert isinstance(s, bytes) and s


def test_argument_checks_without_device(lib):
    from paper_2603_28674_gb300 import rgg
    h = ctypes.c_void_p()
    assert lib.rgg_roadmap_create(None, ctypes.byref(h)) == rgg.RGG_ERR_INVALID
    bad = rgg._Desc(0, 4, 16, 2e-5, 0)          # zero links
    assert lib.rgg_roadmap_create(ctypes.byref(bad), ctypes.byref(h)) == rgg.RGG_ERR_INVALID
    bad = rgg._Desc(3, 4, 16, -1.0, 0)          # negative margin
    assert lib.rgg_roadmap_create(ctypes.byref(bad), ctypes.byref(h)) == rgg.RGG_ERR_INVALID
    bad = rgg._Desc(3, 4, 1 << 20, 2e-5, 0)     # too many obstacles
    assert lib.rgg_roadmap_create(ctypes.byref(bad), ctypes.byref(h)) == rgg.RGG_ERR_INVALID
    for fn in ("rgg_classify", "rgg_check_status"):
        assert getattr(lib, fn)(None, None) == rgg.RGG_ERR_INVALID
    assert lib.rgg_roadmap_destroy(None) == rgg.RGG_OK
    assert lib.rgg_classify_many(None, 0, None) == rgg.RGG_OK


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2603_28674_gb300 import rgg
    monkeypatch.setattr(rgg, "_LIB", None)
    monkeypatch.setattr(rgg, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        rgg.Roadmap(3, 4, 16)
