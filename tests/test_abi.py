"""The C-ABI library builds (cross-compiled for sm_103a), loads without a GPU,
and exports every entry point that include/gwfish.h declares; host-side
argument checks that never reach the GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(gw_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2207_06910_gb300 import build
    build.build()
    import paper_2207_06910_gb300 as gw
    return gw.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    import paper_2207_06910_gb300 as gw
    assert set(gw.EXPORTS) <= set(names)


def test_abi_version_and_null_context(lib):
    assert lib.gw_abi_version() == 7
    assert b"null" in lib.gw_last_error(None)
    assert lib.gw_fisher(None, None, None, 0, 11, None, None, None, None, None, None) == 1  # EINVAL
    assert lib.gw_destroy(None) == 0


def test_kernels_are_sm103a(lib):
    """Every object is built for sm_103a (the build flags say so; the library
    has no PTX fallback for other architectures)."""
    from paper_2207_06910_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.getsize(build.LIB) > 100_000
