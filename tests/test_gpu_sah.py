"""The binned-SAH BLAS build (RG_BLAS_SAH).  Its hierarchy is a choice, not a
result of the method; the tests compare it with the oracle's restatement of
the same build (orc_sah_build) bit for bit, and pin what must hold for any
valid tree and what the heuristic promises: the leaves are the mesh's triangles, each once;
every internal node is reached once and every subtree's leaves are one range
of the leaf order; every child box is
the union of the oracle's triangle boxes below it, bit for bit; the tree's
surface-area cost is lower than the LBVH's; two builds are identical; and
every query answers exactly as on the LBVH build (closest-hit records bit
for bit, any-hit occlusion, rendered images to the rounding of their atomic
sums), which the oracle pins."""
import numpy as np
import pytest
import torch

import oracle
import paper_2001_09792_gb300 as rg
import scenegen as g
from test_gpu_build import LEAF, MESHES, cu, node_fields
from test_gpu_trace import KAPPA, MISS, REL_T, compare_closest, trace, _random_scene
from test_oracle_sah import boxes_mesh, chain_to_level_40, tree_ranges

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("librg")]


def build(v, i, flags):
    h = rg.rg_scene_create()
    try:
        bid = rg.rg_blas_build(h, cu(v, np.float32), cu(i.astype(np.uint32), np.int32), flags)
        rg.rg_sync(h)
        return rg.rg_blas_export(h, bid, i.shape[0])
    finally:
        rg.rg_scene_destroy(h)


def walk(ex, nt):
    _, _, _, _, ch = node_fields(ex["nodes"])
    first, last, _ = tree_ranges(ch, nt)
    return first, last


def sah_cost(ex):
    lo0, hi0, lo1, hi1, _ = node_fields(ex["nodes"])
    lo, hi = np.minimum(lo0, lo1).astype(np.float64), np.maximum(hi0, hi1).astype(np.float64)
    d = hi - lo
    area = d[:, 0] * d[:, 1] + d[:, 1] * d[:, 2] + d[:, 2] * d[:, 0]
    return area.sum() / area[0]


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("morton", [rg.RG_MORTON30, rg.RG_MORTON63])
def test_sah_tree_is_valid(name, morton):
    v, i = MESHES[name]
    nt = i.shape[0]
    ex = build(v, i, morton | rg.RG_BLAS_SAH)
    tris = ex["tris"].reshape(nt, 12)
    perm = tris[:, 3].view(np.uint32)
    assert np.array_equal(np.sort(perm), np.arange(nt, dtype=np.uint32))
    vv = v[i[perm]]
    assert np.array_equal(tris[:, 0:3], vv[:, 0]) and np.array_equal(tris[:, 8:11], vv[:, 2])
    if nt == 1:
        assert ex["root"] == LEAF
        return
    assert ex["root"] == 0
    first, last = walk(ex, nt)
    lohi = oracle.tri_bounds(v, i)[perm]
    lo0, hi0, lo1, hi1, ch = node_fields(ex["nodes"])
    for k in range(nt - 1):
        c0 = int(ch[k][0])
        split = (c0 & ~LEAF) if c0 & LEAF else last[c0]
        assert np.array_equal(np.r_[lo0[k], hi0[k]], np.r_[lohi[first[k]:split + 1, :3].min(0),
                                                           lohi[first[k]:split + 1, 3:].max(0)]), k
        assert np.array_equal(np.r_[lo1[k], hi1[k]], np.r_[lohi[split + 1:last[k] + 1, :3].min(0),
                                                           lohi[split + 1:last[k] + 1, 3:].max(0)]), k


def peeled_series(n=70):
    s = np.float32(1.8) ** np.arange(n, dtype=np.float32)
    lo = np.c_[s, np.zeros(n), np.zeros(n)].astype(np.float32)
    return boxes_mesh(lo, np.c_[s * np.float32(1.8), s, s].astype(np.float32))


# large3 (409,600 triangles) has levels of more than 65,536 segments, which
# the build runs in several slices; chain40 reaches the hand-over to the
# Karras hierarchy at level 40
SAH_MESHES = dict(MESHES, peeled=peeled_series(), chain40=chain_to_level_40(), large1=g.large_scene().meshes[1],
                  large3=g.large_scene().meshes[3])


@pytest.mark.parametrize("name", list(SAH_MESHES))
@pytest.mark.parametrize("morton", [rg.RG_MORTON30, rg.RG_MORTON63])
def test_sah_matches_oracle(name, morton):
    v, i = SAH_MESHES[name]
    nt = i.shape[0]
    ex = build(v, i, morton | rg.RG_BLAS_SAH)
    ref = oracle.sah_reference(v, i, 21 if morton else 10)
    assert np.array_equal(ex["tris"].reshape(nt, 12)[:, 3].view(np.uint32), ref["perm"])
    if nt > 1:
        assert np.array_equal(node_fields(ex["nodes"])[4], ref["child"])


@pytest.mark.parametrize("nt", [2, 15, 16, 17, 18, 33, 2049])
def test_sah_sizes_around_the_thresholds(nt):
    v, i = g.make_mesh("ico", 4)
    i = i[:nt]
    ex = build(v, i, rg.RG_BLAS_SAH)
    walk(ex, nt)
    assert np.array_equal(np.sort(ex["tris"].reshape(nt, 12)[:, 3].view(np.uint32)), np.arange(nt, dtype=np.uint32))


def test_sah_cost_below_lbvh_and_deterministic():
    s = g.large_scene()
    v, i = s.meshes[2]                       # 102,400 triangles
    a = build(v, i, rg.RG_BLAS_SAH)
    b = build(v, i, rg.RG_BLAS_SAH)
    lb = build(v, i, rg.RG_MORTON30)
    assert np.array_equal(a["nodes"].view(np.uint32), b["nodes"].view(np.uint32))
    assert np.array_equal(a["tris"].view(np.uint32), b["tris"].view(np.uint32))
    ca, cl = sah_cost(a), sah_cost(lb)
    print(f"surface-area cost: SAH {ca:.2f}, LBVH {cl:.2f} ({ca / cl:.3f})")
    assert ca < 0.95 * cl
    walk(a, i.shape[0])


def test_sah_scene_answers_like_lbvh_and_brute_force():
    s = _random_scene(41, 60)
    lo, hi = s.world_aabb()
    rays = g.random_rays(200_000, lo - 5, hi + 5, seed=42)
    with rg.GpuScene(s) as gl, rg.GpuScene(s, morton_flags=rg.RG_BLAS_SAH) as gs:
        a, b = trace(gl, rays), trace(gs, rays)
        c = trace(gs, rays[:50_000], rg.RG_TRACE_BRUTE)
        for k in ("inst", "prim"):
            assert np.array_equal(a[k], b[k]), k
            assert np.array_equal(b[k][:50_000], c[k]), k
        for k in ("t", "u", "v"):
            assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32)), k
            assert np.array_equal(b[k][:50_000].view(np.uint32), c[k].view(np.uint32)), k
        assert (b["inst"] != MISS).mean() > 0.1
        rays[:, 7] = np.random.default_rng(43).uniform(1, 40, len(rays))
        oa, ob = trace(gl, rays, rg.RG_ANY), trace(gs, rays, rg.RG_ANY)
        assert np.array_equal(oa["inst"] != MISS, ob["inst"] != MISS)


def test_sah_scene_vs_oracle():
    s = _random_scene(51, 60)
    lo, hi = s.world_aabb()
    rays = g.random_rays(200_000, lo - 5, hi + 5, seed=52)
    with rg.GpuScene(s, morton_flags=rg.RG_BLAS_SAH) as gs:
        h = trace(gs, rays)
    ref = oracle.OracleScene(s).trace(rays, kappa=KAPPA, rel_t=REL_T)
    compare_closest(h, ref, label="sah")


@pytest.mark.parametrize("scene", ["tiny", "medium"])
def test_sah_scene_renders_like_lbvh(scene):
    s = g.tiny_scene() if scene == "tiny" else g.medium_scene()
    imgs = []
    for flags in (rg.RG_MORTON30, rg.RG_BLAS_SAH):
        with rg.GpuScene(s, morton_flags=flags) as gs:
            img = rg.rg_render(gs.h, s.camera, s.width, s.height, s.max_depth)
            rg.rg_sync(gs.h)
            imgs.append(img.cpu().numpy())
    # hit records are the same; a pixel's contributions are summed by float
    # atomics in launch order, so the images agree to rounding, not bit for bit
    assert np.abs(imgs[0].astype(np.float64) - imgs[1]).max() <= 1e-5


def test_sah_compressed_matches_binary():
    s = _random_scene(61, 40)
    lo, hi = s.world_aabb()
    rays = g.random_rays(100_000, lo - 5, hi + 5, seed=62)
    with rg.GpuScene(s, morton_flags=rg.RG_BLAS_SAH) as gb, \
            rg.GpuScene(s, flags=rg.RG_SCENE_COMPRESSED, morton_flags=rg.RG_BLAS_SAH) as gw:
        a, b = trace(gb, rays), trace(gw, rays)
    for k in ("inst", "prim"):
        assert np.array_equal(a[k], b[k]), k
    for k in ("t", "u", "v"):
        assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32)), k


# ---------------------------------------------------------------- TLAS (one-block build)

@pytest.mark.parametrize("n_inst", [2, 3, 17, 65, 66, 300, 1024, 1025, 4096, 4099])
def test_sah_tlas_matches_oracle(n_inst):
    from test_gpu_build import small_instanced_scene
    check_sah_tlas(small_instanced_scene(n_inst, n_inst), n_inst)


@pytest.mark.parametrize("n_inst,dup", [(300, (100, 200)), (129, (0, 129)), (1000, (0, 1000)), (4096, (7, 3000))])
def test_sah_tlas_with_coincident_instances(n_inst, dup):
    """Instances with one transform and mesh share their centroid: segments of
    them are halved by position, and their nodes' boxes come from the refit."""
    from test_gpu_build import small_instanced_scene
    s = small_instanced_scene(n_inst + 5, n_inst)
    a, b = dup
    s.M[a:b] = s.M[a]
    s.mesh_id[a:b] = s.mesh_id[a]
    check_sah_tlas(s, n_inst)


def test_sah_tlas_hand_over_at_level_40():
    """Instances of a one-point mesh placed at the points of
    chain_to_level_40: their world boxes are those points, so the one-block
    TLAS build peels one instance per level and hands the 11 left at level
    40 to the Karras hierarchy, as the oracle does."""
    from test_oracle_sah import chain_to_level_40
    v, _ = chain_to_level_40()
    n = v.shape[0] // 3
    M = np.zeros((n, 3, 4), np.float32)
    M[:, 0, 0] = M[:, 1, 1] = M[:, 2, 2] = 1.0
    M[:, :, 3] = v[0::3]
    point = (np.zeros((3, 3), np.float32), np.array([[0, 1, 2]], np.uint32))
    s = g.Scene(meshes=[point], M=M, mesh_id=np.zeros(n, np.uint32), material_id=np.zeros(n, np.uint32),
                mat_type=np.zeros(1, np.uint32), mat_albedo=np.full((1, 3), 0.5, np.float32),
                mat_ior=np.ones(1, np.float32), light_pos=np.array([[0, 50, 0]], np.float32),
                light_I=np.ones((1, 3), np.float32))
    check_sah_tlas(s, n)


def check_sah_tlas(s, n_inst):
    """The SAH TLAS of scene s against the oracle: instance boxes, leaf order,
    children, and both child boxes of every node (unions of leaf boxes)."""
    from test_gpu_build import object_bounds
    with rg.GpuScene(s, flags=rg.RG_SCENE_SAH_TLAS) as gs:
        ex = rg.rg_tlas_export(gs.h, n_inst)
    obj_box, obj_r2 = object_bounds(s)
    _, wbox, rc = oracle.instance_prep(s.M, obj_box, obj_r2)
    assert rc == 0 and np.array_equal(ex["wbox"], wbox)
    _, _, _, _, ch = node_fields(ex["nodes"])
    if n_inst > 4096:     # beyond the one-block build: the LBVH
        codes, _ = oracle.morton(wbox, 10)
        assert np.array_equal(ex["order"], oracle.stable_sort(codes))
        return
    ref = oracle.sah_boxes(wbox)
    assert np.array_equal(ex["order"], ref["perm"])
    assert np.array_equal(ch, ref["child"])
    first, last, _ = tree_ranges(ch, n_inst)
    ws = wbox[ref["perm"]]
    lo0, hi0, lo1, hi1, _ = node_fields(ex["nodes"])
    for k in range(n_inst - 1):
        c0 = int(ch[k][0])
        split = (c0 & ~LEAF) if c0 & LEAF else last[c0]
        assert np.array_equal(np.r_[lo0[k], hi0[k]], np.r_[ws[first[k]:split + 1, :3].min(0),
                                                           ws[first[k]:split + 1, 3:].max(0)]), k
        assert np.array_equal(np.r_[lo1[k], hi1[k]], np.r_[ws[split + 1:last[k] + 1, :3].min(0),
                                                           ws[split + 1:last[k] + 1, 3:].max(0)]), k


def test_sah_tlas_answers_like_lbvh_and_refits():
    s = _random_scene(71, 1500)
    lo, hi = s.world_aabb()
    rays = g.random_rays(200_000, lo - 5, hi + 5, seed=72)
    with rg.GpuScene(s) as gl, rg.GpuScene(s, flags=rg.RG_SCENE_SAH_TLAS) as gs:
        a, b = trace(gl, rays), trace(gs, rays)
        for k in ("inst", "prim"):
            assert np.array_equal(a[k], b[k]), k
        for k in ("t", "u", "v"):
            assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32)), k
        assert (b["inst"] != MISS).mean() > 0.05
        # a refit keeps the SAH topology and answers like a fresh SAH build
        M2 = g.motion(s.M, 3)
        inst = torch.from_numpy(rg.pack_instances(M2, [gs.blas[m] for m in s.mesh_id], s.material_id)).cuda()
        rg.rg_tlas_refit(gs.h, inst)
        c = trace(gs, rays)
        rg.rg_tlas_build(gs.h, inst)
        d = trace(gs, rays)
        for k in ("inst", "prim", "t"):
            assert np.array_equal(c[k].view(np.uint32) if k == "t" else c[k], d[k].view(np.uint32) if k == "t" else d[k])
