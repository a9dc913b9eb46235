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


def test_struct_sizes_match_the_header(native, tmp_path):
    """The ctypes structures have the sizes and field offsets that a C compiler gives the header's
    structures (compiled here with the host C compiler)."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = {"v3dg_camera": native.v3dg_camera, "v3dg_stats": native.v3dg_stats,
               "v3dg_hierarchy_desc": native.v3dg_hierarchy_desc, "v3dg_request": native.v3dg_request,
               "v3dg_result": native.v3dg_result, "v3dg_allocator": native.v3dg_allocator}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "v3dg.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    for line in filter(None, out):
        name, field, value = line.split()
        cls = structs[name]
        got = ctypes.sizeof(cls) if field == "size" else getattr(cls, field).offset
        assert got == int(value), (name, field, got, value)


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
