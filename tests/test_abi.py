"""The C-ABI library loads and exports every function declared in include/hgl.h
(no GPU needed: nothing here launches a kernel)."""
import ctypes

import pytest

from paper_1908_08281_gb300 import build as _build
from paper_1908_08281_gb300 import hgl


@pytest.fixture(scope="module")
def libhgl():
    _build.build()
    return hgl.lib()


def test_every_declared_function_is_exported(libhgl):
    names = hgl.header_functions()
    assert len(names) >= 17
    for name in names:
        assert hasattr(libhgl, name), name
        assert name in hgl._SIGNATURES, f"binding lacks {name}"


def test_status_strings_and_version(libhgl):
    assert libhgl.hgl_version() >= 100
    for code, name in hgl.STATUS.items():
        assert libhgl.hgl_status_string(code).decode() == name
    assert libhgl.hgl_status_string(12345).decode() == "HGL_ERR_UNKNOWN"


def test_argument_errors_need_no_device(libhgl):
    out = ctypes.c_void_p()
    # invalid sizes are rejected before any CUDA call
    assert libhgl.hgl_build_incidence(0, 1, None, None, 0, None, ctypes.byref(out)) == -1
    assert out.value is None
    assert libhgl.hgl_apply_theta(None, None, 0.0, 1.0, None, 0, None, 0, 1, 0, None) == -1
    assert "NULL" in libhgl.hgl_last_error().decode()
    assert libhgl.hgl_graph_info(None, None, None, None) == -1
    libhgl.hgl_graph_destroy(None)
