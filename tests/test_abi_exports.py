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


def header_signatures():
    """name -> list of parameter declarations, from include/rg.h."""
    txt = open(os.path.join(ROOT, "include", "rg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(?:rg_status|const char\*)\s+(rg_[a-z_0-9]+)\s*\(([^)]*)\)\s*;", txt):
        params = [p.strip() for p in m.group(2).replace("\n", " ").split(",") if p.strip() and p.strip() != "void"]
        out[m.group(1)] = params
    return out


def test_binding_argument_types_match_the_header():
    """Every function the binding declares takes as many arguments as the
    header says, pointers where the header has pointers and 32-bit integers
    where it has 32-bit integers."""
    sigs = header_signatures()
    L = rg.lib()
    assert set(sigs) == set(declared_symbols())
    ptr_types = (ctypes.c_void_p, ctypes.c_char_p)
    for name, params in sigs.items():
        if name == "rg_last_error":
            assert params == [] and L.rg_last_error.argtypes == []
            continue
        args = getattr(L, name).argtypes
        assert args is not None and len(args) == len(params), (name, params, args)
        for decl, t in zip(params, args):
            is_ptr = "*" in decl or "[" in decl  # an array parameter is a pointer
            binding_ptr = t in ptr_types or (isinstance(t, type) and issubclass(t, ctypes._Pointer))
            assert is_ptr == binding_ptr, (name, decl, t)
            if not is_ptr:
                assert t in (ctypes.c_uint32, ctypes.c_int32), (name, decl, t)
                assert ("uint32_t" in decl) == (t is ctypes.c_uint32), (name, decl, t)


def test_product_path_has_no_cpu_fallback():
    """The package never imports the oracle, and without a usable GPU the
    library's own calls fail with a CUDA status instead of computing on the
    host."""
    import subprocess
    import sys
    code = ("import sys, paper_2001_09792_gb300 as rg\n"
            "assert not [m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')]\n")
    subprocess.run([sys.executable, "-c", code], check=True, cwd=ROOT)
    pkg = os.path.join(ROOT, "paper_2001_09792_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, flags=re.M), f
                assert "oracle.cpp" not in txt and "liboracle" not in txt, f
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the failure path is not reachable")
    with pytest.raises(rg.RgError) as e:
        rg.rg_scene_create()
    assert e.value.status == rg.RG_ERR_CUDA


def test_binding_checks_tensor_devices_against_the_scene():
    """The binding knows the device of each scene it made and refuses tensors
    on another device (their addresses would reach the scene's kernels);
    scenes it did not make are not checked.  A stand-in object carries the
    only attribute the check reads."""
    import types

    def on(idx):
        return types.SimpleNamespace(device=types.SimpleNamespace(index=idx))

    rg._same_device(None, rays=on(1))
    rg._same_device(0, rays=on(0), hits=None)
    with pytest.raises(ValueError, match="rays is on cuda:1, the scene on cuda:0"):
        rg._same_device(0, rays=on(1))
    h = ctypes.c_void_p(0x1234560)
    assert rg._scene_dev(h) is None
    rg._SCENE_DEVICE[h.value] = 2
    try:
        assert rg._scene_dev(h) == 2 and rg._scene_dev(h.value) == 2
    finally:
        del rg._SCENE_DEVICE[h.value]
