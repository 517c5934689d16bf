"""The C ABI library loads and exports every entry point include/mge.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mge.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:mge_status|const char\*)\s+(mge_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2112_07862_gb300 import build, mge
    if not os.path.exists(mge.LIB_PATH):
        build.build()
    return mge.load()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ["mge_create", "mge_build_graph_ops", "mge_embed", "mge_submit", "mge_poll", "mge_release",
              "mge_ops_export", "mge_strerror"]:
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s
    from paper_2112_07862_gb300 import mge
    assert sorted(mge.EXPORTS) == declared_symbols()


def test_strerror_is_total(lib):
    from paper_2112_07862_gb300 import mge
    for s in range(0, 13):
        assert mge.mge_strerror(s) not in ("", "unknown status")
    assert mge.mge_strerror(999) == "unknown status"


def test_create_fails_loudly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2112_07862_gb300 import mge
    with pytest.raises(mge.MgeError):
        mge.mge_create(0)


def test_null_arguments_are_rejected(lib):
    lib.mge_destroy.argtypes = [ctypes.c_void_p]
    assert lib.mge_destroy(None) == 1          # MGE_EINVAL
    assert lib.mge_ops_destroy(None) == 1


def test_package_has_no_cpu_fallback():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2112_07862_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
