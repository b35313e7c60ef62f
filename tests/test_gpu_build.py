"""GPU build steps vs the oracle, bit for bit: triangle boxes, Morton codes,
radix sort order, Karras topology, BLAS node boxes and triangle order, TLAS
instance boxes (directed rounding), inverses and topology."""
import numpy as np
import pytest
import torch

import oracle
import paper_2001_09792_gb300 as rg
import scenegen as g

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("librg")]
LEAF = 0x80000000


def cu(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a).view(dt) if np.asarray(a).dtype.itemsize == np.dtype(dt).itemsize
                            else np.ascontiguousarray(a, dt)).cuda()


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def meshes():
    rng = np.random.default_rng(7)
    pts = rng.normal(size=(5000, 3)).astype(np.float32)
    out = {
        "cube": g.cube_mesh(0.5),
        "uv16x8": g.make_mesh("uv", 16, 8),
        "hf45": g.make_mesh("hf", 45, rng=rng),            # 4050 tris: two sort tiles and a ragged tail
        "ico4": g.make_mesh("ico", 4),                       # 5120 tris
        "soup": (pts, rng.integers(0, 5000, size=(7001, 3)).astype(np.uint32)),
        "flat": (np.c_[rng.random((300, 2)), np.zeros(300)].astype(np.float32),
                 rng.integers(0, 300, size=(513, 3)).astype(np.uint32)),   # degenerate z axis
        "dup": (np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32), np.zeros((37, 3), np.uint32) + [0, 1, 2]),
        "one": (np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32), np.array([[0, 1, 2]], np.uint32)),
    }
    return out


MESHES = meshes()


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("bits", [10, 21])
def test_tri_bounds_and_morton_bit_exact(name, bits):
    v, i = MESHES[name]
    lohi = rg.rg_tri_bounds(cu(v, np.float32), cu(i.astype(np.uint32), np.int32))
    ref = oracle.tri_bounds(v, i)
    assert np.array_equal(lohi.cpu().numpy(), ref)
    codes, cb = rg.rg_morton_codes(lohi, bits)
    rc, rcb = oracle.morton(ref, bits)
    got = codes.cpu().numpy().view(np.uint32 if bits == 10 else np.uint64).astype(np.uint64)
    assert np.array_equal(got, rc)
    assert np.array_equal(cb.cpu().numpy(), rcb)


@pytest.mark.parametrize("n", [1, 2, 2047, 2048, 2049, 3 * 2048 + 517, 100_003])
@pytest.mark.parametrize("key_bits", [32, 64])
@pytest.mark.parametrize("spread", ["dups", "full"])
def test_radix_sort_stable(n, key_bits, spread):
    rng = np.random.default_rng(n + key_bits)
    if key_bits == 32:
        hi = 97 if spread == "dups" else 2 ** 32
        keys = rng.integers(0, hi, size=n, dtype=np.uint64).astype(np.uint32)
        kt = torch.from_numpy(keys.view(np.int32)).cuda()
    else:
        hi = 97 if spread == "dups" else 2 ** 63
        keys = rng.integers(0, hi, size=n, dtype=np.uint64)
        if spread == "full":
            keys |= (rng.integers(0, 2, size=n, dtype=np.uint64) << np.uint64(63))
        kt = torch.from_numpy(keys.view(np.int64)).cuda()
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    ko, vo = rg.rg_radix_sort_pairs(kt, vals)
    perm = oracle.stable_sort(keys.astype(np.uint64))
    assert np.array_equal(vo.cpu().numpy().view(np.uint32), perm)
    assert np.array_equal(ko.cpu().numpy().view(keys.dtype), keys[perm])
    # inputs untouched
    assert np.array_equal(kt.cpu().numpy().view(keys.dtype), keys)


def check_children(children, first, last, split):
    ch = children.view(np.uint32) if children.dtype != np.uint32 else children
    left_leaf = split == first
    right_leaf = split + 1 == last
    want_l = np.where(left_leaf, LEAF | split.astype(np.uint32), split.astype(np.uint32))
    want_r = np.where(right_leaf, LEAF | (split + 1).astype(np.uint32), (split + 1).astype(np.uint32))
    assert np.array_equal(ch[:, 0], want_l)
    assert np.array_equal(ch[:, 1], want_r)


@pytest.mark.parametrize("n,hi", [(2, 4), (3, 1), (17, 1), (1000, 8), (4097, 1 << 30), (50_000, 1 << 30), (9999, 64)])
@pytest.mark.parametrize("key_bits", [32, 64])
def test_karras_topology(n, hi, key_bits):
    rng = np.random.default_rng(n)
    keys = np.sort(rng.integers(0, hi, size=n, dtype=np.uint64))
    if key_bits == 32:
        kt = torch.from_numpy(keys.astype(np.uint32).view(np.int32)).cuda()
    else:
        kt = torch.from_numpy((keys << np.uint64(20)).view(np.int64)).cuda()
        keys = keys << np.uint64(20)
    ch, par = rg.rg_karras(kt)
    first, last, split = oracle.karras(keys)
    chn = ch.cpu().numpy().view(np.uint32)
    check_children(chn, first, last, split)
    parents = par.cpu().numpy().view(np.uint32)
    assert parents[0] == 0xFFFFFFFF
    for k in range(n - 1):
        for c in chn[k]:
            idx = (n - 1 + (int(c) & 0x7FFFFFFF)) if int(c) & LEAF else int(c)
            assert parents[idx] == k


def node_fields(nodes):
    f = nodes.reshape(-1, 16)
    return f[:, 0:3], f[:, 3:6], f[:, 6:9], f[:, 9:12], f[:, 12:14].view(np.uint32)


def range_union(lohi_sorted, a, b):
    return np.r_[lohi_sorted[a:b + 1, :3].min(0), lohi_sorted[a:b + 1, 3:].max(0)]


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("flags", [rg.RG_MORTON30, rg.RG_MORTON63])
def test_blas_matches_reference(name, flags):
    v, i = MESHES[name]
    h = rg.rg_scene_create()
    try:
        bid = rg.rg_blas_build(h, cu(v, np.float32), cu(i.astype(np.uint32), np.int32), flags)
        rg.rg_sync(h)
        nt = i.shape[0]
        ex = rg.rg_blas_export(h, bid, nt)
    finally:
        rg.rg_scene_destroy(h)
    ref = oracle.lbvh_reference(v, i, 21 if flags else 10)
    perm = ref["perm"]
    tris = ex["tris"].reshape(nt, 12)
    assert np.array_equal(tris[:, 3].view(np.uint32), perm)
    vv = v[i[perm]]
    assert np.array_equal(tris[:, 0:3], vv[:, 0]) and np.array_equal(tris[:, 4:7], vv[:, 1])
    assert np.array_equal(tris[:, 8:11], vv[:, 2])
    if nt == 1:
        assert ex["root"] == LEAF
        return
    assert ex["root"] == 0
    lo0, hi0, lo1, hi1, ch = node_fields(ex["nodes"])
    check_children(ch, ref["first"], ref["last"], ref["split"])
    lohi_s = ref["lohi"][perm]
    for k in range(nt - 1):
        f, l, s = ref["first"][k], ref["last"][k], ref["split"][k]
        assert np.array_equal(np.r_[lo0[k], hi0[k]], range_union(lohi_s, f, s)), k
        assert np.array_equal(np.r_[lo1[k], hi1[k]], range_union(lohi_s, s + 1, l)), k


def small_instanced_scene(seed, n_inst):
    rng = np.random.default_rng(seed)
    meshes = [g.make_mesh("ico", 2), g.make_mesh("uv", 12, 6), g.cube_mesh(1.0), g.make_mesh("hf", 9, rng=rng),
              (np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32), np.array([[0, 1, 2]], np.uint32))]
    M = np.stack([g.affine(g.random_rotation(rng), rng.uniform(-30, 30, 3), rng.uniform(0.5, 2)) for _ in range(n_inst)])
    mid = rng.integers(0, len(meshes), n_inst).astype(np.uint32)
    mt = np.zeros(n_inst, np.uint32)
    return g.Scene(meshes=meshes, M=M, mesh_id=mid, material_id=np.arange(n_inst, dtype=np.uint32),
                   mat_type=mt, mat_albedo=np.full((n_inst, 3), 0.5, np.float32), mat_ior=np.ones(n_inst, np.float32),
                   light_pos=np.array([[0, 50, 0]], np.float32), light_I=np.ones((1, 3), np.float32))


def blas_root_box(v, i):
    lohi = oracle.tri_bounds(v, i)
    return np.r_[lohi[:, :3].min(0), lohi[:, 3:].max(0)].astype(np.float32)


def object_bounds(s):
    """Per instance: its mesh's root box and bounding-sphere bound r2."""
    boxes = [blas_root_box(*m) for m in s.meshes]
    r2 = [oracle.bound_r2(m[0], b) for m, b in zip(s.meshes, boxes)]
    return np.stack([boxes[m] for m in s.mesh_id]), np.array([r2[m] for m in s.mesh_id], np.float32)


@pytest.mark.parametrize("n_inst", [1, 2, 3, 300, 4099])
def test_tlas_matches_reference(n_inst):
    s = small_instanced_scene(n_inst, n_inst)
    with rg.GpuScene(s) as gs:
        ex = rg.rg_tlas_export(gs.h, n_inst)
    obj_box, obj_r2 = object_bounds(s)
    Minv, wbox, rc = oracle.instance_prep(s.M, obj_box, obj_r2)
    assert rc == 0
    assert np.array_equal(ex["wbox"], wbox)
    # float32 inverse = float32 rounding of the float64 inverse (within one ulp)
    want = Minv.astype(np.float32)
    ulp = np.spacing(np.abs(want)).astype(np.float64)
    assert np.all(np.abs(ex["inv"].astype(np.float64) - want.astype(np.float64)) <= ulp)
    if n_inst == 1:
        assert ex["root"] == LEAF and ex["order"][0] == 0
        return
    codes, _ = oracle.morton(wbox, 10)
    perm = oracle.stable_sort(codes)
    assert np.array_equal(ex["order"], perm)
    first, last, split = oracle.karras(codes[perm])
    lo0, hi0, lo1, hi1, ch = node_fields(ex["nodes"])
    check_children(ch, first, last, split)
    ws = wbox[perm]
    for k in range(n_inst - 1):
        assert np.array_equal(np.r_[lo0[k], hi0[k]], range_union(ws, first[k], split[k]))
        assert np.array_equal(np.r_[lo1[k], hi1[k]], range_union(ws, split[k] + 1, last[k]))


def test_tlas_refit_boxes_match_reference():
    s = small_instanced_scene(5, 257)
    with rg.GpuScene(s) as gs:
        order0 = rg.rg_tlas_export(gs.h, 257)["order"]
        M2 = g.motion(s.M, 1)
        gs.refit(M2)
        rg.rg_sync(gs.h)
        ex = rg.rg_tlas_export(gs.h, 257)
    assert np.array_equal(ex["order"], order0)            # topology unchanged
    obj_box, obj_r2 = object_bounds(s)
    _, wbox, _ = oracle.instance_prep(M2, obj_box, obj_r2)
    assert np.array_equal(ex["wbox"], wbox)
    codes, _ = oracle.morton(oracle.instance_prep(s.M, obj_box, obj_r2)[1], 10)
    first, last, split = oracle.karras(codes[order0])
    lo0, hi0, lo1, hi1, ch = node_fields(ex["nodes"])
    ws = wbox[order0]
    for k in range(256):
        assert np.array_equal(np.r_[lo0[k], hi0[k]], range_union(ws, first[k], split[k]))
        assert np.array_equal(np.r_[lo1[k], hi1[k]], range_union(ws, split[k] + 1, last[k]))


def test_build_errors_reported():
    h = rg.rg_scene_create()
    try:
        v, i = g.cube_mesh(0.5)
        # index out of range: detected on the device, reported at rg_sync
        bad = i.copy()
        bad[3, 1] = 99
        rg.rg_blas_build(h, cu(v, np.float32), cu(bad, np.int32))
        with pytest.raises(rg.RgError) as e:
            rg.rg_sync(h)
        assert e.value.status == rg.RG_ERR_INVALID_ARG
        rg.rg_sync(h)  # cleared
        with pytest.raises(rg.RgError) as e:
            rg.rg_blas_build(h, cu(v, np.float32), cu(i[:0], np.int32))
        assert e.value.status == rg.RG_ERR_INVALID_ARG
        with pytest.raises(rg.RgError) as e:
            rg.rg_blas_build(h, cu(v, np.float32), cu(i, np.int32), flags=8)
        assert e.value.status == rg.RG_ERR_INVALID_ARG
        bid = rg.rg_blas_build(h, cu(v, np.float32), cu(i, np.int32))
        # singular transform
        inst = torch.from_numpy(rg.pack_instances(np.zeros((1, 3, 4), np.float32), [bid])).cuda()
        rg.rg_tlas_build(h, inst)
        with pytest.raises(rg.RgError) as e:
            rg.rg_sync(h)
        assert e.value.status == rg.RG_ERR_SINGULAR
        # refit with another instance count / another BLAS id
        inst = torch.from_numpy(rg.pack_instances(np.stack([g.affine(np.eye(3), [0, 0, 0])] * 2), [bid, bid])).cuda()
        rg.rg_tlas_build(h, inst)
        rg.rg_sync(h)
        with pytest.raises(rg.RgError) as e:
            rg.rg_tlas_refit(h, inst[:1])
        assert e.value.status == rg.RG_ERR_INVALID_ARG
        bid2 = rg.rg_blas_build(h, cu(v, np.float32), cu(i, np.int32))
        inst2 = torch.from_numpy(rg.pack_instances(np.stack([g.affine(np.eye(3), [0, 0, 0])] * 2), [bid, bid2])).cuda()
        rg.rg_tlas_refit(h, inst2)
        with pytest.raises(rg.RgError) as e:
            rg.rg_sync(h)
        assert e.value.status == rg.RG_ERR_INVALID_ARG
    finally:
        rg.rg_scene_destroy(h)


def test_not_built_errors():
    h = rg.rg_scene_create()
    try:
        rays = torch.zeros((4, 8), dtype=torch.float32, device="cuda")
        with pytest.raises(rg.RgError) as e:
            rg.rg_trace_rays(h, rays)
        assert e.value.status == rg.RG_ERR_NOT_BUILT
        with pytest.raises(rg.RgError) as e:
            rg.rg_render(h, dict(eye=(0, 0, 5), target=(0, 0, 0), vfov=60), 8, 8, 1)
        assert e.value.status == rg.RG_ERR_NOT_BUILT
        inst = torch.zeros((1, 16), dtype=torch.float32, device="cuda")
        with pytest.raises(rg.RgError) as e:
            rg.rg_tlas_build(h, inst)
        assert e.value.status == rg.RG_ERR_NOT_BUILT
    finally:
        rg.rg_scene_destroy(h)
