"""Python face of the CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU baseline
may import this package.  It compiles ``oracle.cpp`` with the host compiler
(float64, no FMA contraction, dynamic rounding honoured) into
``oracle/_build/liboracle.so`` and wraps its C functions with ctypes.  It
never imports, loads or calls the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

CXXFLAGS = ["-O2", "-std=c++17", "-ffp-contract=off", "-frounding-math", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle shared library if missing or older than its source."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["g++", *CXXFLAGS, "-o", tmp, _SRC, "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # RG_ORACLE_LIB: a copy of the oracle built elsewhere (the planted-slip
            # check, plant_slips.py, points it at a copy with one change)
            L = ctypes.CDLL(os.environ.get("RG_ORACLE_LIB") or build())
            P = ctypes.c_void_p
            u32, i64, i32, f64, f32 = ctypes.c_uint32, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_float
            L.orc_tri_bounds.argtypes = [P, u32, P, u32, P]
            L.orc_morton.argtypes = [P, u32, i32, P, P]
            L.orc_stable_sort.argtypes = [P, u32, P]
            L.orc_karras.argtypes = [P, u32, P, P, P]
            L.orc_range_boxes.argtypes = [P, u32, P, P, P]
            L.orc_sah_build.argtypes = [P, u32, P, P, P, P]
            L.orc_instance_prep.argtypes = [P, u32, P, P, P, P]
            L.orc_bound_r2.argtypes = [P, u32, P]
            L.orc_bound_r2.restype = ctypes.c_float
            L.orc_scene_new.restype = P
            L.orc_scene_new.argtypes = []
            L.orc_scene_free.argtypes = [P]
            L.orc_scene_free.restype = None
            L.orc_scene_add_mesh.argtypes = [P, P, u32, P, u32]
            L.orc_scene_set_instances.argtypes = [P, P, P, P, u32]
            L.orc_scene_set_shading.argtypes = [P, P, P, P, u32, P, P, u32, P, f32]
            L.orc_trace.argtypes = [P, P, i64, i32, i32, f64, f64, i32, P, P, P, P, P, P, P, P]
            L.orc_camera_rays.argtypes = [P, u32, u32, P, i64, P]
            L.orc_render.argtypes = [P, P, u32, u32, u32, P, i64, f64, f64, i32, P, P, P]
            L.orc_reflect.argtypes = [P, P, P]
            L.orc_refract.argtypes = [P, P, i32, f64, P, P]
            L.orc_fxaa.argtypes = [P, i32, i32, P, i32]
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# ---------------------------------------------------------------- LBVH steps

def tri_bounds(vtx, idx):
    vtx, idx = _c(vtx, np.float32), _c(idx, np.uint32)
    nt = idx.shape[0]
    out = np.empty((nt, 6), np.float32)
    rc = lib().orc_tri_bounds(_p(vtx), vtx.shape[0], _p(idx), nt, _p(out))
    if rc:
        raise ValueError("index out of range")
    return out


def morton(lohi, bits):
    """Morton codes (uint64) of the box centroids and the centroid bounds."""
    lohi = _c(lohi, np.float32)
    n = lohi.shape[0]
    codes = np.empty(n, np.uint64)
    cb = np.empty(6, np.float32)
    lib().orc_morton(_p(lohi), n, bits, _p(codes), _p(cb))
    return codes, cb


def stable_sort(keys):
    keys = _c(keys, np.uint64)
    perm = np.empty(keys.shape[0], np.uint32)
    lib().orc_stable_sort(_p(keys), keys.shape[0], _p(perm))
    return perm


def karras(sorted_keys):
    """(first, last, split) int32 arrays of the n-1 internal nodes."""
    k = _c(sorted_keys, np.uint64)
    n = k.shape[0]
    m = max(n - 1, 0)
    first, last, split = (np.full(m, -1, np.int32) for _ in range(3))
    lib().orc_karras(_p(k), n, _p(first), _p(last), _p(split))
    return first, last, split


def range_boxes(lohi_sorted, first, last):
    lohi_sorted = _c(lohi_sorted, np.float32)
    n = lohi_sorted.shape[0]
    out = np.empty((max(n - 1, 0), 6), np.float32)
    lib().orc_range_boxes(_p(lohi_sorted), n, _p(_c(first, np.int32)), _p(_c(last, np.int32)), _p(out))
    return out


def bound_r2(vtx, obj_box):
    """Upward-rounded bound on the squared distance of the vertices from the
    centre of the object box (float32)."""
    vtx = _c(vtx, np.float32).reshape(-1, 3)
    obj_box = _c(obj_box, np.float32).reshape(6)
    return np.float32(lib().orc_bound_r2(_p(vtx), vtx.shape[0], _p(obj_box)))


def instance_prep(M, obj_box, obj_r2=None):
    """(Minv float64 (n,3,4), world box float32 (n,6), rc).  World box: Arvo's
    box of the object box, intersected with the transformed bounding sphere's
    box when obj_r2 (per instance) is given."""
    M = _c(M, np.float32).reshape(-1, 12)
    obj_box = _c(obj_box, np.float32).reshape(-1, 6)
    n = M.shape[0]
    r2 = None if obj_r2 is None else _c(obj_r2, np.float32).reshape(n)
    Minv = np.empty((n, 12), np.float64)
    wbox = np.empty((n, 6), np.float32)
    rc = lib().orc_instance_prep(_p(M), n, _p(obj_box), None if r2 is None else _p(r2), _p(Minv), _p(wbox))
    return Minv.reshape(n, 3, 4), wbox, rc


def lbvh_reference(vtx, idx, bits=10):
    """All reference build steps for one mesh, as a dict of numpy arrays."""
    lohi = tri_bounds(vtx, idx)
    codes, cb = morton(lohi, bits)
    perm = stable_sort(codes)
    sk = codes[perm]
    first, last, split = karras(sk)
    boxes = range_boxes(lohi[perm], first, last)
    return dict(lohi=lohi, codes=codes, cbounds=cb, perm=perm, sorted_codes=sk, first=first, last=last,
                split=split, boxes=boxes)


def sah_reference(vtx, idx, bits=10):
    """The binned-SAH hierarchy of one mesh (the trace-speed BLAS build, see
    orc_sah_build): dict with the triangle of each leaf (perm), the children of
    each internal node (child, (n-1, 2) uint32, bit 31 a leaf) and the
    triangle boxes (lohi, in triangle order)."""
    return sah_boxes(tri_bounds(vtx, idx), bits)


def sah_boxes(lohi, bits=10):
    """The binned-SAH hierarchy over boxes (lo xyz, hi xyz per row; triangles
    or a TLAS's instance world boxes), as sah_reference."""
    lohi = _c(lohi, np.float32).reshape(-1, 6)
    codes, _ = morton(lohi, bits)
    perm = stable_sort(codes)
    sk = _c(codes[perm], np.uint64)
    n = lohi.shape[0]
    perm_out = np.empty(n, np.uint32)
    child = np.zeros((max(n - 1, 0), 2), np.uint32)
    lib().orc_sah_build(_p(lohi), n, _p(sk), _p(_c(perm, np.uint32)), _p(perm_out), _p(child))
    return dict(perm=perm_out, child=child, lohi=lohi)


# ---------------------------------------------------------------- float64 scene

class OracleScene:
    """A scene held by the oracle: meshes, instances, materials and lights."""

    def __init__(self, scene=None):
        self._L = lib()
        self.h = self._L.orc_scene_new()
        self._keep = []
        if scene is not None:
            for v, i in scene.meshes:
                self.add_mesh(v, i)
            self.set_instances(scene.M, scene.mesh_id, scene.material_id)
            self.set_shading(scene.mat_type, scene.mat_albedo, scene.mat_ior, scene.light_pos, scene.light_I,
                             scene.background, scene.ambient)

    def __del__(self):
        try:
            if self.h:
                self._L.orc_scene_free(self.h)
                self.h = None
        except Exception:
            pass

    def add_mesh(self, vtx, idx):
        vtx, idx = _c(vtx, np.float32), _c(idx, np.uint32)
        rc = self._L.orc_scene_add_mesh(self.h, _p(vtx), vtx.shape[0], _p(idx), idx.shape[0])
        if rc < 0:
            raise ValueError("bad mesh")
        return rc

    def set_instances(self, M, mesh_id, material_id=None):
        M = _c(M, np.float32).reshape(-1, 12)
        mesh_id = _c(mesh_id, np.uint32)
        mat = None if material_id is None else _c(material_id, np.uint32)
        rc = self._L.orc_scene_set_instances(self.h, _p(M), _p(mesh_id), _p(mat), M.shape[0])
        if rc:
            raise ValueError(f"bad instances ({rc})")

    def set_shading(self, mat_type, albedo, ior, light_pos, light_I, background=(0.2, 0.3, 0.5), ambient=0.1):
        mt, al, io = _c(mat_type, np.uint32), _c(albedo, np.float32), _c(ior, np.float32)
        lp, li = _c(light_pos, np.float32).reshape(-1, 3), _c(light_I, np.float32).reshape(-1, 3)
        bg = _c(background, np.float32)
        rc = self._L.orc_scene_set_shading(self.h, _p(mt), _p(al), _p(io), mt.shape[0], _p(lp), _p(li), lp.shape[0],
                                           _p(bg), float(ambient))
        if rc:
            raise ValueError("bad materials")

    def trace(self, rays, any_hit=False, brute=False, kappa=16.0, rel_t=1e-5, threads=0):
        rays = _c(rays, np.float32).reshape(-1, 8)
        n = rays.shape[0]
        out = dict(inst=np.empty(n, np.uint32), prim=np.empty(n, np.uint32), t=np.empty(n), u=np.empty(n),
                   v=np.empty(n), ambiguous=np.empty(n, np.uint8), tol_t=np.empty(n), tol_b=np.empty(n))
        self._L.orc_trace(self.h, _p(rays), n, 1 if any_hit else 0, 1 if brute else 0, kappa, rel_t, threads,
                          _p(out["inst"]), _p(out["prim"]), _p(out["t"]), _p(out["u"]), _p(out["v"]),
                          _p(out["ambiguous"]), _p(out["tol_t"]), _p(out["tol_b"]))
        out["ambiguous"] = out["ambiguous"].astype(bool)
        if any_hit:
            out = dict(occluded=out["inst"] == 0, ambiguous=out["ambiguous"])
        return out

    def render(self, camera, width, height, max_depth, pixels=None, kappa=16.0, rel_t=1e-5, threads=0):
        cam = _camera_array(camera)
        if pixels is None:
            pixels = np.arange(width * height, dtype=np.uint32)
        pixels = _c(pixels, np.uint32)
        n = pixels.shape[0]
        rgba = np.empty((n, 4))
        amb = np.empty(n, np.uint8)
        counts = np.zeros(2, np.uint64)
        self._L.orc_render(self.h, _p(cam), width, height, max_depth, _p(pixels), n, kappa, rel_t, threads,
                           _p(rgba), _p(amb), _p(counts))
        return dict(rgba=rgba, ambiguous=amb.astype(bool), closest_rays=int(counts[0]), shadow_rays=int(counts[1]))


def _camera_array(camera):
    return np.array([*camera["eye"], *camera["target"], *camera.get("up", (0, 1, 0)), camera["vfov"]], np.float32)


def camera_dirs(camera, width, height, pixels):
    cam = _camera_array(camera)
    pixels = _c(pixels, np.uint32)
    out = np.empty((pixels.shape[0], 3))
    lib().orc_camera_rays(_p(cam), width, height, _p(pixels), pixels.shape[0], _p(out))
    return out


def reflect(d, nf):
    d, nf = _c(d, np.float64), _c(nf, np.float64)
    r = np.empty(3)
    lib().orc_reflect(_p(d), _p(nf), _p(r))
    return r


def refract(d, nf, entering, ior):
    """(T, R) or None on total internal reflection."""
    d, nf = _c(d, np.float64), _c(nf, np.float64)
    T = np.empty(3)
    R = np.empty(1)
    ok = lib().orc_refract(_p(d), _p(nf), 1 if entering else 0, float(ior), _p(T), _p(R))
    return (T, float(R[0])) if ok else None


def fxaa(rgba, threads=0):
    """FXAA of an (h, w, 4) float32 image (the oracle's float32 restatement)."""
    img = np.ascontiguousarray(rgba, np.float32)
    h, w = img.shape[0], img.shape[1]
    out = np.empty_like(img)
    lib().orc_fxaa(_p(img), w, h, _p(out), int(threads))
    return out
