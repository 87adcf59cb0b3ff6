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


def test_batch_lengths_checked_before_the_library():
    """The binding refuses batches of different lengths (the C entry points
    take one count for all their arrays) and an import source smaller than
    the ciphertexts, before any call into the library."""
    import types

    import numpy as np

    import paper_2006_10091_gb300 as he
    two, one = [object(), object()], [object()]
    with pytest.raises(ValueError):
        he.he_mul_relin_rescale_batch(None, two, two, one)
    with pytest.raises(ValueError):
        he.he_mul_relin_rescale_batch(None, two, one, two)
    with pytest.raises(ValueError):
        he.he_rotate_batch(None, two, 1, one)
    with pytest.raises(ValueError):
        he.he_rotate_sum_batch(None, one, [1, 2], two)
    ctx = types.SimpleNamespace(n=16)
    with pytest.raises(ValueError):
        he.he_ct_import_batch(ctx, np.zeros((2, 2, 3, 16), dtype=np.uint64)[:1], 3, 1.0, two)
    z, w = np.zeros((4, 2, 6, 16), dtype=np.uint64), np.zeros((2, 6, 16), dtype=np.uint64)
    with pytest.raises(ValueError):  # data ciphertexts claimed at 7 limbs, stored at 6
        he.he_lr_gradient_step_host(ctx, z, 7, 1.0, w, 6, 1.0, None, np.zeros(64, dtype=np.uint64))
    with pytest.raises(ValueError):
        he.he_lr_gradient_step_host(ctx, z, 6, 1.0, w[:1], 6, 1.0, None, np.zeros(64, dtype=np.uint64))
