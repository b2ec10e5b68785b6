"""The C ABI library loads and exports every entry point include/cacl.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "cacl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cacl_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("cacl_create", "cacl_set_geometry", "cacl_set_contact_angle",
              "cacl_step", "cacl_get_fields", "cacl_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2607_25444_b300 import build as B
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_the_same_symbols():
    from paper_2607_25444_b300 import cacl
    assert sorted(cacl.EXPORTS) == declared()


def test_binding_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2607_25444_b300 import cacl
    from paper_2607_25444_b300 import inputs as I
    with pytest.raises(RuntimeError):
        cacl.Solver(I.base_params(8, 8, 8))
