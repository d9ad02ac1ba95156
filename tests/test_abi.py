"""CPU checks of the C ABI: libwp.so builds for sm_103a, loads without a GPU, and exports
every function include/wp.h declares; the Python binding wraps each of them under the
same name.  No compute call is made here (no GPU on this side)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "wp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wp_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2201_06914_gb300 import build as B
    return ctypes.CDLL(B.build())


def test_header_declares_the_path_entry_points():
    names = _declared()
    for must in ("wp_model", "wp_probe_forward", "wp_adjoint_image", "wp_exact_gradient",
                 "wp_workspace_bytes", "wp_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol(lib):
    from paper_2201_06914_gb300 import wp
    assert set(_declared()) <= set(wp.EXPORTS)
    for n in _declared():
        assert callable(getattr(wp, n)), n


def test_last_error_is_empty_string_initially(lib):
    """The message is thread-local: a thread that made no call sees "" (a fresh thread, so
    failures exercised earlier in the same process do not leak in)."""
    import threading
    lib.wp_last_error.restype = ctypes.c_char_p
    seen = []
    th = threading.Thread(target=lambda: seen.append(lib.wp_last_error()))
    th.start()
    th.join()
    assert seen == [b""]


def test_workspace_bytes_rejects_null_model(lib):
    lib.wp_workspace_bytes.restype = ctypes.c_size_t
    assert lib.wp_workspace_bytes(None, None, 8, 32, 0) == 0
