"""The C ABI library loads (no GPU needed) and exports every function include/stretto.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "stretto.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(st_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libst():
    from paper_2602_04430_b300 import build
    build.build()
    from paper_2602_04430_b300 import stretto
    return stretto.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("st_create", "st_kv_build", "st_kv_retain", "st_op_eval", "st_kv_view",
                     "st_run_host", "st_last_error", "st_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(libst):
    missing = [n for n in declared_functions() if not hasattr(libst, n)]
    assert not missing, missing


def test_version_and_error_without_gpu(libst):
    from paper_2602_04430_b300 import stretto
    assert "sm_103a" in stretto.version()
    # argument validation runs on the host: a NULL config is rejected without touching a device
    out = ctypes.c_void_p()
    rc = libst.st_create(None, None, None, ctypes.byref(out))
    assert rc == stretto.ST_EINVAL
    assert b"NULL" in libst.st_last_error(None)


def test_library_is_sm103a_only():
    from paper_2602_04430_b300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_binding_covers_every_declared_function(libst):
    """The Python binding declares a ctypes signature for every entry point of
    the header, under the same name, and for nothing else."""
    from paper_2602_04430_b300 import stretto
    src = open(stretto.__file__).read()
    bound = set(re.findall(r'"(st_[a-z0-9_]+)":\s*\(', src))
    assert bound == set(declared_functions())
    for name in bound:
        assert getattr(libst, name).argtypes is not None


def test_checked_build_exports_every_declared_symbol():
    """The checked build (-DST_CHECK: index and offset checks that record
    ST_ECHECK) is the same library with the same exports."""
    from paper_2602_04430_b300 import build
    path = build.build(check=True)
    assert os.path.basename(path) == "libstretto_check.so"
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = ctypes.c_void_p()
    assert lib.st_create(None, None, None, ctypes.byref(out)) == 1   # ST_EINVAL on the host
