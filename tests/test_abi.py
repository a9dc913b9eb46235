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


def _header_enum(prefix):
    """name -> value of the header's enumerators that start with `prefix` (explicit values, or the
    previous value + 1)."""
    text = open(os.path.join(ROOT, "include", "v3dg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for body in re.findall(r"enum\s*(?:\w+\s*)?\{(.*?)\}", text, flags=re.S):
        value = -1
        for item in body.split(","):
            item = item.strip()
            if not item:
                continue
            m = re.match(r"(\w+)\s*(?:=\s*(-?\w+))?$", item)
            assert m, item
            value = int(m.group(2), 0) if m.group(2) else value + 1
            if m.group(1).startswith(prefix):
                out[m.group(1)] = value
    return out


def test_option_and_status_constants_match_the_header(native):
    """Every option and status value of the header has a binding constant with the same value."""
    for prefix in ("V3DG_OPT_", "V3DG_OK", "V3DG_E"):
        want = _header_enum(prefix)
        assert want, prefix
        for name, value in want.items():
            assert getattr(native, name) == value, name
    status = {**_header_enum("V3DG_OK"), **_header_enum("V3DG_E")}
    assert native.STATUS_NAMES == [n for n, _ in sorted(status.items(), key=lambda kv: kv[1])]


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
