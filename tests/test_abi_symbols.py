"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function include/plhr.h declares; the Python binding declares a signature for
each of them (no compute call is made here)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "plhr.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)     # comments
    names = set(re.findall(r"\b(plhr_[a-z0-9_]+)\s*\(", text))
    # typedef'd struct/enum names are not followed by "(", so names holds the
    # functions; drop anything that is only a type name
    types = set(re.findall(r"\}\s*(plhr_[a-z0-9_]+)\s*;", text))
    return sorted(names - types)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("plhr_solve", "plhr_op_stencil", "plhr_prec_avmg", "plhr_prec_apply", "plhr_prec_apply_f32",
                 "plhr_tharm_extract", "plhr_tharm_extract_noalloc", "plhr_status_string"):
        assert must in names


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1408_0042_gb300 import build
    path = build.build()
    try:
        return ctypes.CDLL(path)
    except OSError as e:          # CUDA runtime library missing on this host
        pytest.skip("cannot load libplhr.so here: %s" % e)


def test_library_exports_every_declared_function(lib):
    missing = [nm for nm in _declared_functions() if not hasattr(lib, nm)]
    assert not missing, missing


def test_binding_has_a_signature_for_every_declared_function():
    import paper_1408_0042_gb300 as p
    missing = [nm for nm in _declared_functions() if nm not in p._SIGS]
    assert not missing, missing
