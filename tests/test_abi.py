"""Host-side checks of the C ABI library: it builds for sm_103a, loads, exports
every function include/jdec.h declares, and behaves without a GPU."""
import ctypes
import os
import re

import pytest

from paper_1311_5304_gb300 import build as jbuild
from paper_1311_5304_gb300 import jdec

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"JDEC_API\s+[\w\s\*]+?\b(jdec_\w+)\s*\(", txt)
    return names


def test_library_builds_and_exports_every_declared_function():
    path = jbuild.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 7
    for n in names:
        assert hasattr(lib, n), n
    assert set(jdec.exported_symbols()) <= set(names)


def test_status_strings():
    assert jdec.status_str(jdec.OK) == "ok"
    assert "invalid" in jdec.status_str(jdec.EINVAL)
    assert "timed out" in jdec.status_str(jdec.ETIMEOUT)
    assert jdec.status_str(12345) == "unknown status"


def test_null_arguments_are_rejected_without_a_device():
    lib = jdec.load()
    assert lib.jdec_create(None, None) == jdec.EINVAL
    assert lib.jdec_decode_coeffs(None, None, None) == jdec.EINVAL
    assert lib.jdec_decode_batch(None, None, 0, None) == jdec.EINVAL
    assert lib.jdec_decode_host(None, None, None) == jdec.EINVAL
    assert lib.jdec_decode_host_batch(None, None, 1, None) == jdec.EINVAL
    assert lib.jdec_decode_jpeg(None, None, 0, None, 0, 0, 1, None) == jdec.EINVAL
    assert lib.jdec_sync_status(None, None) == jdec.EINVAL
    assert lib.jdec_destroy(None) == jdec.EINVAL


def test_create_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(jdec.JdecError):
        jdec.Context()


def test_kernels_are_built_for_sm103a_only():
    # the build passes exactly one -gencode, for sm_103a
    assert jbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
