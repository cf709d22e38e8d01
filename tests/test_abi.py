"""The C-ABI library builds, loads and exports every entry point include/tmbir.h declares.

No compute call here: these run without a GPU.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "tmbir.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tmbir_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import paper_2603_28756_gb300 as tm

    return tm.load()


def test_every_declared_symbol_is_exported(lib):
    names = header_functions()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), f"{n} declared in tmbir.h but not exported"


def test_binding_covers_the_header():
    import paper_2603_28756_gb300 as tm

    assert sorted(tm.SYMBOLS) == header_functions()


def test_null_arguments_are_rejected(lib):
    assert lib.tmbir_set_geometry(None, 1, None) == -1
    assert b"NULL" in lib.tmbir_last_error()
    assert lib.tmbir_workspace_size(None, None) == -1
    assert lib.tmbir_sync(None) == -1
    assert lib.tmbir_destroy(None) == 0


def test_create_without_device_fails_loudly(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.tmbir_create(ctypes.byref(h), None) == -4
    assert b"no CUDA device" in lib.tmbir_last_error()


def test_product_path_does_not_import_the_oracle():
    # the package must not reference the CPU oracle in any form
    pkg = os.path.join(ROOT, "paper_2603_28756_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "orc_" not in src, f
