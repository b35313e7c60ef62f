"""Compressed 8-wide BVH (8-bit child boxes against a float32 parent frame).

* Every dequantized child box contains the exact float32 box of the binary
  subtree it replaces (outward rounding), every item appears exactly once,
  and each wide node's slots reference the binary tree consistently.
* Hit records of the compressed path are bit-identical to the float32 binary
  path (closest-hit and any-hit), on the tiny, medium, random (with mirrored
  instances) and large scenes; renders agree to float-atomic ordering.
* The wide TLAS refit equals a fresh wide build."""
import numpy as np
import pytest
import torch

import oracle
import paper_2001_09792_gb300 as rg
import scenegen as g
from test_gpu_trace import _random_scene, camera_rays

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("librg")]
MISS = 0xFFFFFFFF
LEAF = 0x80000000


def dequant(w):
    scale = np.ldexp(1.0, w["e"]).astype(np.float64)                 # (nodes, 3)
    p = w["p"].astype(np.float64)
    lo = p[:, None, :] + w["qlo"].astype(np.float64) * scale[:, None, :]
    hi = p[:, None, :] + w["qhi"].astype(np.float64) * scale[:, None, :]
    return lo, hi                                                      # (nodes, 8, 3)


def binary_box(nodes2, ref, leaf_boxes):
    if ref & LEAF:
        return leaf_boxes[ref & 0x7FFFFFFF]
    f = nodes2[ref].reshape(16)
    return np.r_[np.minimum(f[0:3], f[6:9]), np.maximum(f[3:6], f[9:12])]


def check_wide(w, nodes2, leaf_boxes, n_items):
    lo, hi = dequant(w)
    assert np.all(np.abs(w["e"]) <= 127)
    assert np.array_equal(np.sort(w["item_src"]), np.arange(n_items))
    for k in range(w["n_nodes"]):
        imask = int(w["imask"][k])
        rank = 0
        for s in range(8):
            ref = int(w["src"][k, s])
            meta = int(w["meta"][k, s])
            if ref == MISS:
                assert meta == 0 and not (imask >> s) & 1
                continue
            b = binary_box(nodes2, ref, leaf_boxes).astype(np.float64)
            assert np.all(lo[k, s] <= b[:3]) and np.all(hi[k, s] >= b[3:]), (k, s)
            if (imask >> s) & 1:
                child = int(w["child_base"][k]) + rank
                rank += 1
                assert child < w["n_nodes"]
            else:
                cnt, off = meta >> 5, meta & 31
                assert 1 <= cnt <= 3
                items = w["item_src"][int(w["item_base"][k]) + off: int(w["item_base"][k]) + off + cnt]
                if ref & LEAF:
                    assert cnt == 1 and items[0] == ref & 0x7FFFFFFF
                else:
                    assert np.array_equal(items, np.sort(items)) and items[-1] - items[0] == cnt - 1


MESHES = {"cube": g.cube_mesh(0.5), "uv": g.make_mesh("uv", 16, 8), "ico4": g.make_mesh("ico", 4),
          "hf33": g.make_mesh("hf", 33, rng=np.random.default_rng(1)),
          "one": (np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32), np.array([[0, 1, 2]], np.uint32)),
          "two": (np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 1]], np.float32),
                  np.array([[0, 1, 2], [1, 2, 3]], np.uint32))}


@pytest.mark.parametrize("name", list(MESHES))
def test_wide_blas_is_conservative_and_complete(name):
    v, i = MESHES[name]
    h = rg.rg_scene_create(flags=rg.RG_SCENE_COMPRESSED)
    try:
        bid = rg.rg_blas_build(h, torch.from_numpy(v).cuda(), torch.from_numpy(i.astype(np.uint32).view(np.int32)).cuda())
        rg.rg_sync(h)
        nt = i.shape[0]
        ex = rg.rg_blas_export(h, bid, nt)
        w = rg.rg_wide_export(h, bid, nt)
    finally:
        rg.rg_scene_destroy(h)
    tris = ex["tris"].reshape(nt, 12)
    tv = np.stack([tris[:, 0:3], tris[:, 4:7], tris[:, 8:11]], 1)
    leaf_boxes = np.c_[tv.min(1), tv.max(1)]
    assert w["n_items"] == nt and 1 <= w["n_nodes"] <= max(nt - 1, 1)
    check_wide(w, ex["nodes"].reshape(-1, 16) if nt > 1 else None, leaf_boxes, nt)


@pytest.mark.parametrize("n_inst", [1, 2, 9, 300])
def test_wide_tlas_is_conservative_and_complete(n_inst):
    s = _random_scene(n_inst, n_inst)
    with rg.GpuScene(s, flags=rg.RG_SCENE_COMPRESSED) as gs:
        ex = rg.rg_tlas_export(gs.h, n_inst)
        w = rg.rg_wide_export(gs.h, rg.RG_TLAS_ID, n_inst)
    leaf_boxes = ex["wbox"][ex["order"]]
    check_wide(w, ex["nodes"].reshape(-1, 16) if n_inst > 1 else None, leaf_boxes, n_inst)


def trace(h, rays, flags):
    out = rg.rg_trace_rays(h, torch.from_numpy(np.ascontiguousarray(rays, np.float32)).cuda(), flags)
    rg.rg_sync(h)
    return out


def assert_same(a, b):
    assert torch.equal(a, b), f"{(a != b).any(1).sum().item()} hit records differ"


def compare_paths(s, rays, any_tmax=None):
    with rg.GpuScene(s, flags=rg.RG_SCENE_COMPRESSED) as gs:
        assert_same(trace(gs.h, rays, 0), trace(gs.h, rays, rg.RG_TRACE_PLAIN))
        r2 = rays.copy()
        if any_tmax is not None:
            r2[:, 7] = any_tmax
        a = trace(gs.h, r2, rg.RG_ANY)
        b = trace(gs.h, r2, rg.RG_ANY | rg.RG_TRACE_PLAIN)
        assert torch.equal(a[:, 0] == -1, b[:, 0] == -1)


def test_identical_hits_tiny():
    s = g.tiny_scene()
    rays = np.concatenate([camera_rays(s), g.random_rays(100_000, np.array([-6, -3, -6]), np.array([6, 5, 6]), seed=3)])
    compare_paths(s, rays, any_tmax=np.random.default_rng(0).uniform(0.5, 8, len(rays)))


def test_identical_hits_random_mirrored():
    s = _random_scene(41, 80)
    lo, hi = s.world_aabb()
    rays = g.random_rays(300_000, lo - 5, hi + 5, seed=42)
    compare_paths(s, rays, any_tmax=np.random.default_rng(1).uniform(1, 40, len(rays)))


def test_identical_hits_axis_aligned_and_edges():
    s = _random_scene(7, 20)
    lo, hi = s.world_aabb()
    rng = np.random.default_rng(3)
    n = 50_000
    o = rng.uniform(lo - 2, hi + 2, size=(n, 3)).astype(np.float32)
    d = np.zeros((n, 3), np.float32)
    d[np.arange(n), rng.integers(0, 3, n)] = rng.choice([-1.0, 1.0], n)
    rays = np.c_[o, np.zeros(n), d, np.full(n, np.inf)].astype(np.float32)
    compare_paths(s, rays)


def test_identical_hits_medium():
    s = g.medium_scene()
    lo, hi = s.world_aabb()
    rays = np.concatenate([camera_rays(s), g.random_rays(1_000_000, lo, hi, seed=5)])
    compare_paths(s, rays, any_tmax=np.random.default_rng(2).uniform(1, 50, len(rays)))


def test_identical_hits_large_full_launch():
    s = g.large_scene()
    closest, anyhit = g.large_rays(s, 1 << 24)
    with rg.GpuScene(s, flags=rg.RG_SCENE_COMPRESSED) as gs:
        d = torch.from_numpy(closest).cuda()
        a = rg.rg_trace_rays(gs.h, d, 0)
        b = rg.rg_trace_rays(gs.h, d, rg.RG_TRACE_PLAIN)
        rg.rg_sync(gs.h)
        assert_same(a, b)
        del d, a, b
        d = torch.from_numpy(anyhit).cuda()
        a = rg.rg_trace_rays(gs.h, d, rg.RG_ANY)
        b = rg.rg_trace_rays(gs.h, d, rg.RG_ANY | rg.RG_TRACE_PLAIN)
        rg.rg_sync(gs.h)
        assert torch.equal(a[:, 0] == -1, b[:, 0] == -1)


def test_compressed_render_matches_plain_render():
    s = g.medium_scene()
    with rg.GpuScene(s, flags=rg.RG_SCENE_COMPRESSED) as gw:
        a = rg.rg_render(gw.h, s.camera, s.width, s.height, s.max_depth)
        rg.rg_sync(gw.h)
        a = a.cpu().numpy()
    with rg.GpuScene(s) as gp:
        b = rg.rg_render(gp.h, s.camera, s.width, s.height, s.max_depth)
        rg.rg_sync(gp.h)
        b = b.cpu().numpy()
    np.testing.assert_allclose(a, b, atol=1e-5)


def test_wide_refit_equals_fresh_build():
    s = _random_scene(51, 64)
    M2 = g.motion(s.M, 7)
    lo, hi = s.world_aabb()
    rays = g.random_rays(200_000, lo - 5, hi + 5, seed=52)
    with rg.GpuScene(s, flags=rg.RG_SCENE_COMPRESSED) as gs:
        gs.refit(M2)
        a = trace(gs.h, rays, 0)
        p = trace(gs.h, rays, rg.RG_TRACE_PLAIN)
        w = rg.rg_wide_export(gs.h, rg.RG_TLAS_ID, 64)
        ex = rg.rg_tlas_export(gs.h, 64)
    assert_same(a, p)
    check_wide(w, ex["nodes"].reshape(-1, 16), ex["wbox"][ex["order"]], 64)
    s.M = M2
    with rg.GpuScene(s, flags=rg.RG_SCENE_COMPRESSED) as gs:
        b = trace(gs.h, rays, 0)
    assert_same(a, b)


def test_compressed_vs_oracle_tiny():
    s = g.tiny_scene()
    O = oracle.OracleScene(s)
    rays = np.concatenate([camera_rays(s), g.random_rays(20_000, np.array([-6, 0.55, -6]), np.array([6, 5, 6]), seed=9)])
    with rg.GpuScene(s, flags=rg.RG_SCENE_COMPRESSED) as gs:
        h = rg.split_hits(trace(gs.h, rays, 0))
    from test_gpu_trace import KAPPA, REL_T, compare_closest
    compare_closest(h, O.trace(rays, kappa=KAPPA, rel_t=REL_T), label="wide tiny")


def test_not_built_without_wide_blas():
    h = rg.rg_scene_create()
    try:
        v, i = g.cube_mesh(0.5)
        bid = rg.rg_blas_build(h, torch.from_numpy(v).cuda(), torch.from_numpy(i.view(np.int32)).cuda())
        with pytest.raises(rg.RgError) as e:
            rg.rg_wide_export(h, bid, 12)
        assert e.value.status == rg.RG_ERR_NOT_BUILT
    finally:
        rg.rg_scene_destroy(h)
