"""Python binding of librg, the GB300 ray tracer (see include/rg.h).

Argument marshalling only: every step of the hot path runs in the CUDA
kernels of librg.so.  PyTorch provides device memory and streams.  There is
no CPU fallback: if librg.so is missing or the device is not a CUDA GPU the
calls raise.

Functions carry the C names (rg_scene_create, rg_blas_build, rg_tlas_build,
rg_tlas_refit, rg_trace_rays, rg_render, ...).  Device buffers are torch
tensors on the current CUDA device; uint32 data travels in int32 tensors and
uint64 keys in int64 tensors (bit patterns unchanged).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librg.so")

RG_OK = 0
RG_ERR_INVALID_ARG, RG_ERR_OOM, RG_ERR_CUDA, RG_ERR_NOT_BUILT, RG_ERR_STACK, RG_ERR_TIMEOUT, RG_ERR_SINGULAR = range(1, 8)
RG_MORTON30, RG_MORTON63 = 0, 1
RG_CLOSEST, RG_ANY, RG_TRACE_BRUTE, RG_TRACE_STATS, RG_TRACE_PLAIN = 0, 1, 2, 4, 8
RG_SCENE_TIMING = 1
RG_SCENE_COUNT = 2
RG_SCENE_COMPRESSED = 4
RG_SCENE_NO_PAIR = 8
RG_SCENE_FRUGAL = 16
RG_SCENE_SAH_TLAS = 32
RG_COMPRESSED = 2
RG_BLAS_SAH = 4
RG_TLAS_ID = 0xFFFFFFFF
RG_MAT_DIFFUSE, RG_MAT_MIRROR, RG_MAT_GLASS = 0, 1, 2
MISS = 0xFFFFFFFF

# exported symbols, in include/rg.h order
SYMBOLS = ["rg_scene_create", "rg_scene_create_shared", "rg_scene_destroy", "rg_blas_build", "rg_tlas_build", "rg_tlas_refit",
           "rg_scene_set_materials", "rg_scene_set_lights", "rg_trace_rays", "rg_render", "rg_sync", "rg_get_stats",
           "rg_reset_stats", "rg_last_error", "rg_tri_bounds", "rg_morton_codes", "rg_radix_sort_pairs", "rg_karras",
           "rg_blas_export", "rg_tlas_export", "rg_wide_export", "rg_radix_sort_pairs_noalloc",
           "rg_server_create", "rg_server_destroy", "rg_server_add_scene", "rg_server_submit", "rg_server_step",
           "rg_server_drain", "rg_server_poll", "rg_server_get_stats", "rg_server_set_shape", "rg_server_get_shape",
           "rg_server_autotune", "rg_fxaa"]
RG_NOALLOC_SORT_MAX_PAIRS = 262144
RG_SERVER_MAX_SLOTS = 32
RG_SERVER_MAX_PIXELS = 1 << 23
RG_SERVER_MAX_DEPTH = 15
RG_SERVER_NO_GRAPH = 1
RG_SERVER_NO_PAIR = 2
RG_TUNE_FORCE = 1

f32x3 = ctypes.c_float * 3


class rg_camera(ctypes.Structure):
    _fields_ = [("eye", f32x3), ("target", f32x3), ("up", f32x3), ("vfov_deg", ctypes.c_float)]


class rg_material(ctypes.Structure):
    _fields_ = [("type", ctypes.c_uint32), ("albedo", f32x3), ("ior", ctypes.c_float), ("pad", f32x3)]


class rg_light(ctypes.Structure):
    _fields_ = [("pos", f32x3), ("intensity", f32x3)]


class rg_scene_desc(ctypes.Structure):
    _fields_ = [("background", f32x3), ("ambient", ctypes.c_float), ("flags", ctypes.c_uint32)]


class rg_stats(ctypes.Structure):
    _fields_ = [("closest_rays", ctypes.c_uint64), ("shadow_rays", ctypes.c_uint64),
                ("trace_launches", ctypes.c_uint64), ("trace_ms", ctypes.c_double),
                ("any_launches", ctypes.c_uint64), ("any_ms", ctypes.c_double),
                ("node_visits", ctypes.c_uint64), ("tri_tests", ctypes.c_uint64), ("inst_entries", ctypes.c_uint64),
                ("any_node_visits", ctypes.c_uint64), ("any_tri_tests", ctypes.c_uint64),
                ("any_inst_entries", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64),
                ("pair_launches", ctypes.c_uint64), ("pair_ms", ctypes.c_double),
                ("refine_launches", ctypes.c_uint64), ("refine_ms", ctypes.c_double)]


class rg_server_desc(ctypes.Structure):
    _fields_ = [("ring_log2", ctypes.c_uint32), ("batch_rays", ctypes.c_uint32), ("max_lights", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("admit_rays", ctypes.c_uint32), ("lanes", ctypes.c_uint32)]


class rg_request(ctypes.Structure):
    _fields_ = [("scene", ctypes.c_uint32), ("camera", rg_camera), ("width", ctypes.c_uint32),
                ("height", ctypes.c_uint32), ("max_depth", ctypes.c_uint32), ("h_transforms", ctypes.c_void_p),
                ("d_rgba", ctypes.c_void_p), ("tag", ctypes.c_uint64)]


class rg_completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("tag", ctypes.c_uint64), ("admitted_step", ctypes.c_uint32),
                ("completed_step", ctypes.c_uint32)]


class rg_server_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_uint64), ("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64),
                ("completed", ctypes.c_uint64), ("closest_rays", ctypes.c_uint64), ("shadow_rays", ctypes.c_uint64),
                ("pending", ctypes.c_uint32), ("active", ctypes.c_uint32), ("ring_rays", ctypes.c_uint32),
                ("ring_peak", ctypes.c_uint32), ("graph_launches", ctypes.c_uint64),
                ("graph_captures", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64),
                ("newest_first_steps", ctypes.c_uint64), ("lane_steps", ctypes.c_uint64)]


class rg_trace_shape(ctypes.Structure):
    _fields_ = [("block", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32), ("refill", ctypes.c_uint32),
                ("stack", ctypes.c_uint32), ("ms", ctypes.c_float)]


class RgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"rg status {status}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load librg.so (build it with __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build(); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        P, u32, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int32
        sig = {
            "rg_scene_create": [ctypes.POINTER(P), P],
            "rg_scene_create_shared": [ctypes.POINTER(P), P],
            "rg_scene_destroy": [P],
            "rg_blas_build": [P, P, u32, P, u32, u32, ctypes.POINTER(u32), P],
            "rg_tlas_build": [P, P, u32, P],
            "rg_tlas_refit": [P, P, u32, P],
            "rg_scene_set_materials": [P, P, u32],
            "rg_scene_set_lights": [P, P, u32],
            "rg_trace_rays": [P, P, u32, u32, P, P],
            "rg_render": [P, P, u32, u32, u32, P, P],
            "rg_sync": [P],
            "rg_get_stats": [P, P],
            "rg_reset_stats": [P],
            "rg_tri_bounds": [P, u32, P, u32, P, P],
            "rg_morton_codes": [P, u32, u32, P, P, P],
            "rg_radix_sort_pairs": [P, P, u32, u32, P, P, P],
            "rg_karras": [P, u32, u32, P, P, P],
            "rg_blas_export": [P, u32, P, P, ctypes.POINTER(u32)],
            "rg_tlas_export": [P, P, P, P, P, ctypes.POINTER(u32)],
            "rg_radix_sort_pairs_noalloc": [P, P, u32, u32, P, P, P],
            "rg_wide_export": [P, u32, P, P, P, P],
            "rg_server_create": [ctypes.POINTER(P), P],
            "rg_server_destroy": [P],
            "rg_server_add_scene": [P, P, ctypes.POINTER(u32)],
            "rg_server_submit": [P, P, ctypes.POINTER(ctypes.c_uint64)],
            "rg_server_step": [P, ctypes.POINTER(u32)],
            "rg_server_drain": [P],
            "rg_server_poll": [P, P, u32, ctypes.POINTER(u32)],
            "rg_server_get_stats": [P, P],
            "rg_server_set_shape": [P, u32, P],
            "rg_server_get_shape": [P, u32, P],
            "rg_server_autotune": [P, P, ctypes.c_char_p, u32, P],
            "rg_fxaa": [P, u32, u32, P, P],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = i32
        L.rg_last_error.argtypes = []
        L.rg_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(status):
    if status != RG_OK:
        raise RgError(status, lib().rg_last_error().decode())


def _torch():
    import torch
    return torch


def _stream(stream, device=None):
    """The stream argument: `stream`, or the current stream of `device` (an
    index; None: the current device)."""
    torch = _torch()
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dev(t, dtype, shape_tail=None, name="tensor"):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape_tail is not None and tuple(t.shape[1:]) != tuple(shape_tail):
        raise ValueError(f"{name} must have shape (n, {', '.join(map(str, shape_tail))})")
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------- scene

# CUDA device index of each scene made here (a scene lives on the device that
# was current when it was created, and its calls run there)
_SCENE_DEVICE = {}


def _scene_dev(scene):
    """Device index of a scene made through this binding (None otherwise)."""
    return _SCENE_DEVICE.get(scene.value if isinstance(scene, ctypes.c_void_p) else scene)


def _same_device(dev, **tensors):
    """Raise unless every given tensor is on CUDA device `dev` (None: no check):
    the library would hand another GPU's addresses to the scene's kernels."""
    if dev is None:
        return
    for name, t in tensors.items():
        if t is not None and t.device.index != dev:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the scene on cuda:{dev}")


def rg_scene_create(background=(0.2, 0.3, 0.5), ambient=0.1, flags=0):
    d = rg_scene_desc(f32x3(*background), float(ambient), int(flags))
    h = ctypes.c_void_p()
    _check(lib().rg_scene_create(ctypes.byref(h), ctypes.byref(d)))
    _SCENE_DEVICE[h.value] = _torch().cuda.current_device()
    return h


def rg_scene_create_shared(src):
    """A scene sharing src's BLAS, with copies of its materials and lights."""
    h = ctypes.c_void_p()
    _check(lib().rg_scene_create_shared(ctypes.byref(h), src))
    dev = _scene_dev(src)
    if dev is not None:
        _SCENE_DEVICE[h.value] = dev
    return h


def rg_scene_destroy(scene):
    _check(lib().rg_scene_destroy(scene))
    _SCENE_DEVICE.pop(scene.value if isinstance(scene, ctypes.c_void_p) else scene, None)


def rg_blas_build(scene, vtx, idx, flags=RG_MORTON30, stream=None):
    """vtx: (nv,3) float32, idx: (nt,3) int32 (uint32 indices); returns the BLAS id."""
    torch = _torch()
    pv = _dev(vtx, torch.float32, (3,), "vtx")
    pi = _dev(idx, torch.int32, (3,), "idx")
    dev = _scene_dev(scene)
    _same_device(dev, vtx=vtx, idx=idx)
    out = ctypes.c_uint32()
    _check(lib().rg_blas_build(scene, pv, vtx.shape[0], pi, idx.shape[0], flags, ctypes.byref(out),
                               _stream(stream, dev)))
    return out.value


def pack_instances(M, blas_ids, material_ids=None):
    """rg_instance array as a (n,16) float32 numpy array (ids as uint32 bit patterns)."""
    M = np.ascontiguousarray(M, np.float32).reshape(-1, 12)
    n = M.shape[0]
    out = np.zeros((n, 16), np.float32)
    out[:, :12] = M
    ids = out.view(np.uint32)
    ids[:, 12] = np.asarray(blas_ids, np.uint32)
    ids[:, 13] = 0 if material_ids is None else np.asarray(material_ids, np.uint32)
    ids[:, 14] = 0xFF
    return out


def rg_tlas_build(scene, inst, stream=None):
    """inst: (n,16) float32 CUDA tensor of rg_instance records (see pack_instances)."""
    torch = _torch()
    p = _dev(inst, torch.float32, (16,), "inst")
    dev = _scene_dev(scene)
    _same_device(dev, inst=inst)
    _check(lib().rg_tlas_build(scene, p, inst.shape[0], _stream(stream, dev)))


def rg_tlas_refit(scene, inst, stream=None):
    torch = _torch()
    p = _dev(inst, torch.float32, (16,), "inst")
    dev = _scene_dev(scene)
    _same_device(dev, inst=inst)
    _check(lib().rg_tlas_refit(scene, p, inst.shape[0], _stream(stream, dev)))


def rg_scene_set_materials(scene, types, albedo, ior):
    types = np.asarray(types, np.uint32)
    albedo = np.asarray(albedo, np.float32).reshape(-1, 3)
    ior = np.asarray(ior, np.float32)
    arr = (rg_material * len(types))()
    for k in range(len(types)):
        arr[k] = rg_material(int(types[k]), f32x3(*albedo[k]), float(ior[k]), f32x3(0, 0, 0))
    _check(lib().rg_scene_set_materials(scene, arr, len(types)))


def rg_scene_set_lights(scene, pos, intensity):
    pos = np.asarray(pos, np.float32).reshape(-1, 3)
    intensity = np.asarray(intensity, np.float32).reshape(-1, 3)
    arr = (rg_light * max(len(pos), 1))()
    for k in range(len(pos)):
        arr[k] = rg_light(f32x3(*pos[k]), f32x3(*intensity[k]))
    _check(lib().rg_scene_set_lights(scene, arr, len(pos)))


# ---------------------------------------------------------------- dispatch

def rg_trace_rays(scene, rays, flags=RG_CLOSEST, hits=None, stream=None):
    """rays: (n,8) float32 CUDA tensor {o, tmin, d, tmax}; returns hits (n,5) int32
    {instance, prim, t, u, v} (t/u/v as float32 bit patterns; see split_hits)."""
    torch = _torch()
    pr = _dev(rays, torch.float32, (8,), "rays")
    n = rays.shape[0]
    if hits is None:
        hits = torch.empty((n, 5), dtype=torch.int32, device=rays.device)
    ph = _dev(hits, torch.int32, (5,), "hits")
    if hits.shape[0] < n:
        raise ValueError("hits buffer too small")
    dev = _scene_dev(scene)
    _same_device(dev, rays=rays, hits=hits)
    _check(lib().rg_trace_rays(scene, pr, n, flags, ph, _stream(stream, dev)))
    return hits


def split_hits(hits):
    """Host view of a hit tensor: dict of numpy arrays instance/prim (uint32), t/u/v (float32)."""
    h = hits.cpu().numpy() if hasattr(hits, "cpu") else np.asarray(hits)
    h = np.ascontiguousarray(h)
    return dict(inst=h[:, 0].view(np.uint32), prim=h[:, 1].view(np.uint32), t=h[:, 2].view(np.float32),
                u=h[:, 3].view(np.float32), v=h[:, 4].view(np.float32))


def make_camera(camera):
    return rg_camera(f32x3(*camera["eye"]), f32x3(*camera["target"]), f32x3(*camera.get("up", (0, 1, 0))),
                     float(camera["vfov"]))


def rg_render(scene, camera, width, height, max_depth, out=None, stream=None):
    """Render into a (h, w, 4) float32 CUDA tensor (allocated if out is None)."""
    torch = _torch()
    dev = _scene_dev(scene)
    if out is None:
        out = torch.empty((height, width, 4), dtype=torch.float32,
                          device="cuda" if dev is None else torch.device("cuda", dev))
    if out.numel() != width * height * 4 or out.dtype != torch.float32 or not out.is_cuda or not out.is_contiguous():
        raise ValueError("out must be a contiguous float32 CUDA tensor of w*h*4 elements")
    _same_device(dev, out=out)
    cam = camera if isinstance(camera, rg_camera) else make_camera(camera)
    _check(lib().rg_render(scene, ctypes.byref(cam), width, height, max_depth, ctypes.c_void_p(out.data_ptr()),
                           _stream(stream, dev)))
    return out


def rg_fxaa(image, out=None, stream=None):
    """FXAA of an (h, w, 4) float32 CUDA image into `out` (allocated if None)."""
    torch = _torch()
    if image.dim() != 3 or image.shape[2] != 4 or image.dtype != torch.float32 or not image.is_cuda \
            or not image.is_contiguous():
        raise ValueError("image must be a contiguous (h, w, 4) float32 CUDA tensor")
    if out is None:
        out = torch.empty_like(image)
    if out.shape != image.shape or out.dtype != torch.float32 or not out.is_cuda or not out.is_contiguous() \
            or out.device != image.device:
        raise ValueError("out must match the image (shape, type, device)")
    h, w = image.shape[0], image.shape[1]
    with torch.cuda.device(image.device):
        _check(lib().rg_fxaa(ctypes.c_void_p(image.data_ptr()), w, h, ctypes.c_void_p(out.data_ptr()),
                             _stream(stream)))
    return out


def rg_sync(scene):
    _check(lib().rg_sync(scene))


def rg_get_stats(scene):
    st = rg_stats()
    _check(lib().rg_get_stats(scene, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in rg_stats._fields_}


def rg_reset_stats(scene):
    _check(lib().rg_reset_stats(scene))


# ---------------------------------------------------------------- build steps

def rg_tri_bounds(vtx, idx, stream=None):
    torch = _torch()
    out = torch.empty((idx.shape[0], 6), dtype=torch.float32, device=vtx.device)
    _check(lib().rg_tri_bounds(_dev(vtx, torch.float32, (3,), "vtx"), vtx.shape[0], _dev(idx, torch.int32, (3,), "idx"),
                               idx.shape[0], ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def rg_morton_codes(lohi, bits, stream=None):
    """Morton codes (int32 for bits=10, int64 for bits=21) and centroid bounds."""
    torch = _torch()
    n = lohi.shape[0]
    codes = torch.empty(n, dtype=torch.int32 if bits == 10 else torch.int64, device=lohi.device)
    cb = torch.empty(6, dtype=torch.float32, device=lohi.device)
    _check(lib().rg_morton_codes(_dev(lohi, torch.float32, (6,), "lohi"), n, bits, ctypes.c_void_p(codes.data_ptr()),
                                 ctypes.c_void_p(cb.data_ptr()), _stream(stream)))
    return codes, cb


def _sort_args(keys, vals, keys_out=None, vals_out=None):
    """Checks shared by the two sorts: n = len(keys) pairs; vals holds n
    values; outputs (when given) hold at least n elements of the right type;
    every tensor is on keys' device.  Returns (n, key_bits)."""
    torch = _torch()
    if keys.dim() != 1 or vals.dim() != 1:
        raise ValueError("keys and vals must be 1-D")
    n = keys.shape[0]
    if vals.numel() != n:
        raise ValueError(f"vals holds {vals.numel()} values for {n} keys")
    for name, t in (("vals", vals), ("keys_out", keys_out), ("vals_out", vals_out)):
        if t is not None and t.device != keys.device:
            raise ValueError(f"{name} is on {t.device}, keys on {keys.device}")
    for name, t in (("keys_out", keys_out), ("vals_out", vals_out)):
        if t is not None and t.numel() < n:
            raise ValueError(f"{name} holds {t.numel()} elements, fewer than n = {n}")
    return n, (64 if keys.dtype == torch.int64 else 32)


def rg_radix_sort_pairs(keys, vals, stream=None):
    """Stable sort of (keys int32/int64 as unsigned, vals int32); returns (keys, vals)."""
    torch = _torch()
    n, key_bits = _sort_args(keys, vals)
    with torch.cuda.device(keys.device):
        ko = torch.empty_like(keys)
        vo = torch.empty_like(vals)
        _check(lib().rg_radix_sort_pairs(_dev(keys, keys.dtype, None, "keys"), _dev(vals, torch.int32, None, "vals"),
                                         n, key_bits, ctypes.c_void_p(ko.data_ptr()),
                                         ctypes.c_void_p(vo.data_ptr()), _stream(stream)))
    return ko, vo


def rg_radix_sort_pairs_noalloc(keys, vals, keys_out=None, vals_out=None, stream=None):
    """rg_radix_sort_pairs through the entry point that allocates nothing on
    the device (its temporaries live in a fixed array inside librg.so; at
    most RG_NOALLOC_SORT_MAX_PAIRS pairs).  Outputs are caller buffers; they
    are allocated here only when not given."""
    torch = _torch()
    n, key_bits = _sort_args(keys, vals, keys_out, vals_out)
    with torch.cuda.device(keys.device):
        ko = torch.empty_like(keys) if keys_out is None else keys_out
        vo = torch.empty_like(vals) if vals_out is None else vals_out
        _check(lib().rg_radix_sort_pairs_noalloc(_dev(keys, keys.dtype, None, "keys"),
                                                 _dev(vals, torch.int32, None, "vals"), n, key_bits,
                                                 _dev(ko, keys.dtype, None, "keys_out"),
                                                 _dev(vo, torch.int32, None, "vals_out"), _stream(stream)))
    return ko, vo


def rg_karras(sorted_keys, stream=None):
    """(children (n-1,2) int32, parents (2n-1,) int32) of the radix tree."""
    torch = _torch()
    n = sorted_keys.shape[0]
    key_bits = 64 if sorted_keys.dtype == torch.int64 else 32
    ch = torch.empty((max(n - 1, 1), 2), dtype=torch.int32, device=sorted_keys.device)
    par = torch.empty(max(2 * n - 1, 1), dtype=torch.int32, device=sorted_keys.device)
    _check(lib().rg_karras(_dev(sorted_keys, sorted_keys.dtype, None, "keys"), n, key_bits,
                           ctypes.c_void_p(ch.data_ptr()), ctypes.c_void_p(par.data_ptr()), _stream(stream)))
    return ch, par


def rg_blas_export(scene, blas_id, nt):
    nodes = np.zeros((max(nt - 1, 1), 16), np.float32)
    tris = np.zeros((nt, 12), np.float32)
    root = ctypes.c_uint32()
    _check(lib().rg_blas_export(scene, blas_id, nodes.ctypes.data_as(ctypes.c_void_p),
                                tris.ctypes.data_as(ctypes.c_void_p), ctypes.byref(root)))
    return dict(nodes=nodes[: max(nt - 1, 0)], tris=tris, root=root.value)


def rg_wide_export(scene, blas_id, n_leaves):
    """Compressed 8-wide BVH of a BLAS (or RG_TLAS_ID): dict with the decoded
    nodes (p, e, imask, child_base, item_base, meta, qlo, qhi), slot sources
    and item sources (numpy arrays)."""
    cap = max(n_leaves - 1, 1)
    raw = np.zeros((cap, 20), np.uint32)
    src = np.zeros((cap, 8), np.uint32)
    item_src = np.zeros(max(n_leaves, 1), np.uint32)
    counts = np.zeros(2, np.uint32)
    v = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    _check(lib().rg_wide_export(scene, blas_id, v(raw), src.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                item_src.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                counts.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))))
    nn, ni = int(counts[0]), int(counts[1])
    raw = raw[:nn]
    b = raw.view(np.uint8).reshape(nn, 80)
    bits = raw[:, 3]
    e = np.stack([(bits >> (8 * k)) & 0xFF for k in range(3)], 1).astype(np.uint8).view(np.int8).astype(np.int32)
    return dict(p=raw[:, 0:3].view(np.float32), e=e, imask=(bits >> 24).astype(np.uint32), child_base=raw[:, 4],
                item_base=raw[:, 5], meta=b[:, 24:32], qlo=np.stack([b[:, 32:40], b[:, 40:48], b[:, 48:56]], 2),
                qhi=np.stack([b[:, 56:64], b[:, 64:72], b[:, 72:80]], 2), src=src[:nn], item_src=item_src[:ni],
                n_nodes=nn, n_items=ni)


def rg_tlas_export(scene, n):
    nodes = np.zeros((max(n - 1, 1), 16), np.float32)
    wbox = np.zeros((n, 6), np.float32)
    inv = np.zeros((n, 12), np.float32)
    order = np.zeros(n, np.uint32)
    root = ctypes.c_uint32()
    v = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    _check(lib().rg_tlas_export(scene, v(nodes), v(wbox), v(inv), v(order), ctypes.byref(root)))
    return dict(nodes=nodes[: max(n - 1, 0)], wbox=wbox, inv=inv.reshape(n, 3, 4), order=order, root=root.value)


# ---------------------------------------------------------------- render server

def rg_server_create(ring_log2=0, batch_rays=0, max_lights=0, flags=0, admit_rays=0, lanes=0):
    d = rg_server_desc(int(ring_log2), int(batch_rays), int(max_lights), int(flags), int(admit_rays), int(lanes))
    h = ctypes.c_void_p()
    _check(lib().rg_server_create(ctypes.byref(h), ctypes.byref(d)))
    return h


def rg_server_destroy(server):
    _check(lib().rg_server_destroy(server))


def rg_server_add_scene(server, scene):
    sid = ctypes.c_uint32()
    _check(lib().rg_server_add_scene(server, scene, ctypes.byref(sid)))
    return sid.value


def make_request(scene_id, camera, width, height, max_depth, image, transforms=None, tag=0):
    """An rg_request; `image` is a contiguous float32 CUDA tensor of w*h*4
    elements, `transforms` None or (n_inst, 3, 4) float32 (kept alive by the
    returned pair until submission copies it)."""
    torch = _torch()
    if image.numel() != width * height * 4 or image.dtype != torch.float32 or not image.is_cuda \
            or not image.is_contiguous():
        raise ValueError("image must be a contiguous float32 CUDA tensor of w*h*4 elements")
    cam = camera if isinstance(camera, rg_camera) else make_camera(camera)
    tr = None
    if transforms is not None:
        tr = np.ascontiguousarray(transforms, np.float32).reshape(-1, 12)
    q = rg_request(int(scene_id), cam, int(width), int(height), int(max_depth),
                   ctypes.c_void_p(tr.ctypes.data) if tr is not None else None, ctypes.c_void_p(image.data_ptr()),
                   int(tag))
    return q, tr


def rg_server_submit(server, scene_id, camera, width, height, max_depth, image, transforms=None, tag=0):
    q, _keep = make_request(scene_id, camera, width, height, max_depth, image, transforms, tag)
    rid = ctypes.c_uint64()
    _check(lib().rg_server_submit(server, ctypes.byref(q), ctypes.byref(rid)))
    return rid.value


def rg_server_step(server):
    n = ctypes.c_uint32()
    _check(lib().rg_server_step(server, ctypes.byref(n)))
    return n.value


def rg_server_drain(server):
    _check(lib().rg_server_drain(server))


def rg_server_poll(server, max_n=RG_SERVER_MAX_SLOTS * 4):
    buf = (rg_completion * max_n)()
    n = ctypes.c_uint32()
    _check(lib().rg_server_poll(server, buf, max_n, ctypes.byref(n)))
    return [dict(id=c.id, tag=c.tag, admitted_step=c.admitted_step, completed_step=c.completed_step)
            for c in buf[: n.value]]


def rg_server_get_stats(server):
    st = rg_server_stats()
    _check(lib().rg_server_get_stats(server, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in rg_server_stats._fields_}


def rg_server_set_shape(server, which, block, blocks_per_sm, refill, stack=0):
    sh = rg_trace_shape(int(block), int(blocks_per_sm), int(refill), int(stack), 0.0)
    _check(lib().rg_server_set_shape(server, int(which), ctypes.byref(sh)))


def rg_server_get_shape(server, which):
    sh = rg_trace_shape()
    _check(lib().rg_server_get_shape(server, int(which), ctypes.byref(sh)))
    return dict(block=sh.block, blocks_per_sm=sh.blocks_per_sm, refill=sh.refill, stack=sh.stack)


def rg_server_autotune(server, scene_id, camera, width, height, max_depth, image, cache_path=None, force=False):
    q, _keep = make_request(scene_id, camera, width, height, max_depth, image)
    out = (rg_trace_shape * 2)()
    path = cache_path.encode() if cache_path else None
    _check(lib().rg_server_autotune(server, ctypes.byref(q), path, RG_TUNE_FORCE if force else 0, out))
    return [dict(block=o.block, blocks_per_sm=o.blocks_per_sm, refill=o.refill, stack=o.stack, ms=o.ms) for o in out]


# ---------------------------------------------------------------- convenience

class GpuScene:
    """Owns one rg_scene built from a scenegen-style scene description
    (meshes, instance transforms, materials, lights)."""

    def __init__(self, scene, flags=0, morton_flags=RG_MORTON30, stream=None):
        torch = _torch()
        self.h = rg_scene_create(scene.background, scene.ambient, flags)
        self.n_inst = scene.n_instances
        self.nts = []
        try:
            self.blas = []
            for v, i in scene.meshes:
                tv = torch.from_numpy(np.ascontiguousarray(v, np.float32)).cuda()
                ti = torch.from_numpy(np.ascontiguousarray(i, np.uint32).view(np.int32)).cuda()
                self.blas.append(rg_blas_build(self.h, tv, ti, morton_flags, stream))
                self.nts.append(int(i.shape[0]))
            self.inst_host = pack_instances(scene.M, [self.blas[m] for m in scene.mesh_id], scene.material_id)
            self.inst = torch.from_numpy(self.inst_host).cuda()
            rg_tlas_build(self.h, self.inst, stream)
            rg_scene_set_materials(self.h, scene.mat_type, scene.mat_albedo, scene.mat_ior)
            rg_scene_set_lights(self.h, scene.light_pos, scene.light_I)
            rg_sync(self.h)
        except Exception:
            self.close()
            raise

    def shared(self, stream=None):
        """Another GpuScene over the same BLAS (rg_scene_create_shared) with
        this one's instances, materials and lights and a TLAS of its own."""
        torch = _torch()
        other = GpuScene.__new__(GpuScene)
        other.h = rg_scene_create_shared(self.h)
        try:
            other.n_inst, other.nts, other.blas = self.n_inst, list(self.nts), list(self.blas)
            other.inst_host = self.inst_host.copy()
            other.inst = torch.from_numpy(other.inst_host).cuda()
            rg_tlas_build(other.h, other.inst, stream)
            rg_sync(other.h)
        except Exception:
            other.close()
            raise
        return other

    def refit(self, M, stream=None):
        torch = _torch()
        host = self.inst_host.copy()
        host[:, :12] = np.ascontiguousarray(M, np.float32).reshape(-1, 12)
        self.inst = torch.from_numpy(host).cuda()
        rg_tlas_refit(self.h, self.inst, stream)

    def close(self):
        if getattr(self, "h", None):
            rg_scene_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
