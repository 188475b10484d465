"""Host-side checks of the C ABI that need no GPU: the library builds, loads and
exports every entry point include/ultraray.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ultraray.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(ur_\w+)\s*\(", src, flags=re.M))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("ur_create", "ur_destroy", "ur_scene_upload", "ur_set_array", "ur_set_plane_waves", "ur_trace",
              "ur_beamform", "ur_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_2501_05828_gb300 as ur
    from paper_2501_05828_gb300 import build as b
    b.build()
    L = ctypes.CDLL(b.LIB)
    for name in declared():
        assert hasattr(L, name), name
    assert set(ur.EXPORTS) == declared()


def test_null_context_is_rejected_without_a_gpu():
    import paper_2501_05828_gb300 as ur
    L = ur.lib()
    assert L.ur_last_error(None) == b"null context"
    assert L.ur_destroy(None) == 1
    assert L.ur_sync(None) == 1
    assert L.ur_set_array(None, None) == 1


def test_create_fails_cleanly_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2501_05828_gb300 as ur
    h = ctypes.c_void_p()
    code = ur.lib().ur_create(ctypes.byref(h), 0, None)
    assert code != 0 and not h.value


def test_binding_refuses_to_run_without_the_library(tmp_path, monkeypatch):
    import paper_2501_05828_gb300 as ur
    monkeypatch.setattr(ur, "_lib", None)
    monkeypatch.setattr(ur, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        ur.lib()
