"""The C-ABI library builds, loads without a GPU and exports every symbol include/v3dg.h declares."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "v3dg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(v3dg_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def native():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2505_06523_gb300 import _native
    return _native


def test_every_declared_symbol_is_exported(native):
    lib = native.lib()
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(native):
    assert set(_declared()) == set(native.SIGNATURES)


def test_struct_sizes_match_the_header(native):
    import ctypes
    # v3dg_camera: 12 doubles + 4 floats + 2 int32 + float (+ padding to 8)
    assert ctypes.sizeof(native.v3dg_camera) == 96 + 16 + 8 + 4 + 4
    assert ctypes.sizeof(native.v3dg_stats) == 5 * 8 + 2 * 4 + 2 * 8


def test_no_gpu_means_an_error_not_a_fallback(native):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(native.V3dgError) as e:
        native.v3dg_create(0)
    assert e.value.status == native.V3DG_ECUDA
    from paper_2505_06523_gb300 import Context
    with pytest.raises(RuntimeError):
        Context(0)
