"""The C-ABI library builds, loads and exports every symbol that
include/rg.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

import paper_2001_09792_gb300 as rg
from paper_2001_09792_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "rg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rg_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def librg():
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["rg_scene_create", "rg_blas_build", "rg_tlas_build", "rg_tlas_refit", "rg_trace_rays", "rg_render"]:
        assert name in syms
    assert sorted(rg.SYMBOLS) == syms


def test_library_exports_every_declared_symbol(librg):
    for name in declared_symbols():
        assert hasattr(librg, name), name


def test_binding_loads_library():
    L = rg.lib()
    assert L.rg_last_error() == b""


def test_struct_sizes_match_header():
    assert ctypes.sizeof(rg.rg_camera) == 40
    assert ctypes.sizeof(rg.rg_material) == 32
    assert ctypes.sizeof(rg.rg_light) == 24
    assert ctypes.sizeof(rg.rg_scene_desc) == 20
    inst = rg.pack_instances([[[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]]], [3], [5])
    assert inst.shape == (1, 16) and inst.view("uint32")[0, 12] == 3 and inst.view("uint32")[0, 13] == 5


def test_null_scene_is_rejected_without_gpu():
    # argument checks run on the host before any CUDA call
    L = rg.lib()
    assert L.rg_sync(None) == rg.RG_ERR_INVALID_ARG
    assert b"NULL" in L.rg_last_error()


STRUCTS = ["rg_camera", "rg_material", "rg_light", "rg_scene_desc", "rg_stats", "rg_server_desc", "rg_request",
           "rg_completion", "rg_server_stats", "rg_trace_shape"]


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """Every ctypes mirror has the size and field offsets gcc gives the
    header's struct."""
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "rg.h"', "int main(void) {"]
    for name in STRUCTS:
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in getattr(rg, name)._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n") if l)
    for name in STRUCTS:
        cls = getattr(rg, name)
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, f"{name}.{f}"


def test_null_server_is_rejected_without_gpu():
    L = rg.lib()
    assert L.rg_server_step(None, None) == rg.RG_ERR_INVALID_ARG
    assert L.rg_server_destroy(None) == rg.RG_OK
    assert L.rg_server_create(None, None) == rg.RG_ERR_INVALID_ARG
