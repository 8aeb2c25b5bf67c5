"""The C ABI library builds, loads without a GPU and exports every function
declared in include/*.h; argument errors are reported without touching the
device."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(cg_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1508_06329_gb300 import build, binding
    build.build()
    return binding.load()


def test_header_declares_entry_points():
    names = declared_functions()
    for want in ("cg_context_create", "cg_chordal_test_dense", "cg_lexbfs_order_dense", "cg_peo_check_dense",
                 "cg_chordal_test_batch", "cg_chordal_test_dense_host"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1508_06329_gb300 import binding
    missing = [n for n in declared_functions() if n not in binding.SIGNATURES or not hasattr(binding, n)]
    assert not missing, missing


def test_version_and_null_checks(lib):
    from paper_1508_06329_gb300 import binding as B
    assert b"sm_103a" in B.cg_version()
    # a null context is rejected before any CUDA call
    assert B.cg_chordal_test_dense(None, None, None, None, None) == B.CG_EINVAL
    assert b"context" in B.cg_last_error_string()
    assert B.cg_context_create(None, None) == B.CG_EINVAL
    assert B.cg_step_floor(None, 1024, 16, 1 << 20, 16, None, None) == B.CG_EINVAL
