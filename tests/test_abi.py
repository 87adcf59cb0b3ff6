"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function include/he_gb300.h declares (no compute calls)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "he_gb300.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(he_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("he_ctx_create", "he_encode_encrypt", "he_encrypt_poly", "he_add",
                     "he_mul_relin_rescale", "he_rotate", "he_decrypt_decode",
                     "he_lr_gradient_step", "he_refresh", "he_ct_export", "he_ct_import"):
        assert required in names


def test_library_exports_every_declared_symbol():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2006_10091_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
