"""Closest-hit / any-hit / miss on the GPU vs the FP64 oracle.

Tolerances are the plain ones of the method's statement:
  * t within 1e-5 relative: |t - t_ref| <= 1e-5 t_ref;
  * barycentrics within 1e-5 relative: |u - u_ref| <= 1e-5 max(|u_ref|, 1e-3),
    the same for v (a floor of 1e-3 keeps the bound finite at an edge);
  * hit ids equal.
A ray that fails any of these "differs".  Every differing ray must be one the
oracle flags as ambiguous (its exact winner lies within the float32 error band
of an edge, another candidate lies within that band of its distance, or it
grazes), and the differing rays number at most 1e-4 of the set.  The float32
error band (eta / |cos|, from the magnitudes that enter the object-space ray)
only decides which rays are flagged; it widens no comparison.
BVH traversal must equal brute force bit for bit.
"""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
import paper_2001_09792_gb300 as rg
import scenegen as g

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("librg")]
MISS = 0xFFFFFFFF
KAPPA = 16.0
REL_T = 1e-5       # t within 1e-5 relative
REL_B = 1e-5       # barycentrics within 1e-5 relative ...
B_FLOOR = 1e-3     # ... to max(|u|, 1e-3)
MAX_EXEMPT = 1e-4  # differing (flagged) rays, at most this fraction of a set


def trace(gs, rays, flags=0):
    hits = rg.rg_trace_rays(gs.h, torch.from_numpy(np.ascontiguousarray(rays, np.float32)).cuda(), flags)
    rg.rg_sync(gs.h)
    return rg.split_hits(hits)


def plain_differ(h, ref):
    """Per ray: True where the GPU record differs from the oracle's under the
    plain tolerances (ids, t, u, v; a miss must be the exact miss record)."""
    id_diff = (h["inst"] != ref["inst"]) | (h["prim"] != ref["prim"])
    hit = ~id_diff & (ref["inst"] != MISS)
    t_ref = ref["t"]
    with np.errstate(invalid="ignore"):   # inf - inf where both records are misses; those rays are checked below
        dt = np.abs(h["t"].astype(np.float64) - t_ref)
        du = np.abs(h["u"].astype(np.float64) - ref["u"])
        dv = np.abs(h["v"].astype(np.float64) - ref["v"])
        bad_t = hit & ~(dt <= REL_T * np.abs(t_ref))
        bad_u = hit & ~(du <= REL_B * np.maximum(np.abs(ref["u"]), B_FLOOR))
        bad_v = hit & ~(dv <= REL_B * np.maximum(np.abs(ref["v"]), B_FLOOR))
    miss = ~id_diff & (ref["inst"] == MISS)
    bad_miss = miss & ~(np.isinf(h["t"]) & (h["u"] == 0) & (h["v"] == 0))
    return id_diff | bad_t | bad_u | bad_v | bad_miss


def compare_closest(h, ref, max_exempt=MAX_EXEMPT, label=""):
    """Every ray that differs under the plain tolerances must be flagged
    ambiguous by the oracle, and at most max_exempt of the rays may differ.
    Prints the counts and the worst errors of the agreeing hits; returns the
    differing fraction."""
    amb = ref["ambiguous"]
    differ = plain_differ(h, ref)
    unflagged = differ & ~amb
    assert not unflagged.any(), (
        f"{label}: {unflagged.sum()} differing rays are not flagged, e.g. ray {np.nonzero(unflagged)[0][:5]}")
    n = len(differ)
    allowed = int(np.floor(max_exempt * n))
    assert differ.sum() <= allowed, f"{label}: {differ.sum()} rays differ (flagged), more than {allowed} of {n}"
    agree = ~differ & (ref["inst"] != MISS)
    rt = (np.abs(h["t"][agree] - ref["t"][agree]) / np.abs(ref["t"][agree])).max(initial=0.0)
    ru = (np.abs(h["u"][agree] - ref["u"][agree]) / np.maximum(np.abs(ref["u"][agree]), B_FLOOR)).max(initial=0.0)
    rv = (np.abs(h["v"][agree] - ref["v"][agree]) / np.maximum(np.abs(ref["v"][agree]), B_FLOOR)).max(initial=0.0)
    print(f"{label}: {differ.sum()} of {n} rays differ (all flagged; allowed {allowed}), {amb.sum()} flagged; "
          f"worst relative error t {rt:.2e}, u {ru:.2e}, v {rv:.2e}")
    return differ.mean()


def camera_rays(scene, pixels=None):
    w, h = scene.width, scene.height
    if pixels is None:
        pixels = np.arange(w * h, dtype=np.uint32)
    d = oracle.camera_dirs(scene.camera, w, h, pixels)
    r = np.zeros((len(pixels), 8), np.float32)
    r[:, 0:3] = scene.camera["eye"]
    r[:, 4:7] = d
    r[:, 7] = np.inf
    return r


@pytest.fixture(scope="module")
def tiny():
    s = g.tiny_scene()
    gs = rg.GpuScene(s)
    yield s, gs, oracle.OracleScene(s)
    gs.close()


@pytest.fixture(scope="module")
def medium():
    s = g.medium_scene()
    gs = rg.GpuScene(s)
    yield s, gs, oracle.OracleScene(s)
    gs.close()


def test_tiny_camera_and_random_rays(tiny):
    s, gs, O = tiny
    # origins above the cubes (which rest on the ground, bottom faces coplanar
    # with it: that contact is covered by the next test)
    rays = np.concatenate([camera_rays(s), g.random_rays(50_000, np.array([-6, 0.55, -6]), np.array([6, 5, 6]), seed=3)])
    h = trace(gs, rays)
    ref = O.trace(rays, kappa=KAPPA, rel_t=REL_T)
    compare_closest(h, ref, label="tiny")
    assert (ref["inst"] != MISS).mean() > 0.2


def test_tiny_coplanar_contact_from_below(tiny):
    """The cubes rest on the ground: their bottom faces are coplanar with it,
    so rays from below meet both surfaces at exactly the same t.  Both sides
    decide that tie on the exact distance rounded to float32, then by the
    smaller instance (the ground), so the contact is bounded like any other
    ray set."""
    s, gs, O = tiny
    rays = g.random_rays(50_000, np.array([-6, -3, -6]), np.array([6, -0.5, 6]), seed=13)
    h = trace(gs, rays)
    ref = O.trace(rays, kappa=KAPPA, rel_t=REL_T)
    # rays that meet a cube's bottom face inside the ground's footprint: exact ties
    ties = (ref["inst"] == 0) & ref["ambiguous"]
    assert ties.sum() > 100
    compare_closest(h, ref, label="tiny-below")


def test_tiny_rays_from_all_directions(tiny):
    """The tiny scene from every direction: origins uniform in a box around it
    (above, beside and below the ground), directions uniform on the sphere;
    the coplanar contact of the cubes and the ground is met from below."""
    s, gs, O = tiny
    rng = np.random.default_rng(17)
    n = 200_000
    o = rng.uniform([-7, -4, -7], [7, 6, 7], (n, 3))
    d = rng.normal(size=(n, 3))
    rays = np.c_[o, np.zeros(n), d / np.linalg.norm(d, axis=1, keepdims=True), np.full(n, np.inf)].astype(np.float32)
    h = trace(gs, rays)
    ref = O.trace(rays, kappa=KAPPA, rel_t=REL_T)
    assert (ref["inst"] != MISS).mean() > 0.1
    compare_closest(h, ref, label="tiny all directions")


def test_tiny_any_hit(tiny):
    s, gs, O = tiny
    rays = g.random_rays(50_000, np.array([-6, -1, -6]), np.array([6, 5, 6]), seed=4, tmax_range=(0.5, 8))
    h = trace(gs, rays, rg.RG_ANY)
    ref = O.trace(rays, any_hit=True, kappa=KAPPA, rel_t=REL_T)
    ok = ~ref["ambiguous"]
    occ = h["inst"] != MISS
    assert np.array_equal(occ[ok], ref["occluded"][ok])
    assert ref["ambiguous"].mean() <= MAX_EXEMPT
    # a reported hit is a real hit inside [tmin, tmax]
    assert np.all((h["t"][occ] >= rays[occ, 3]) & (h["t"][occ] <= rays[occ, 7]))
    # any-hit <=> closest hit within tmax (same rays, closest query)
    c = trace(gs, rays)
    assert np.array_equal(occ, c["inst"] != MISS)


@pytest.mark.parametrize("blas", ["lbvh", "sah"])
def test_medium_rays_at_full_launch(medium, blas):
    """Camera rays of the 1920x1080 view plus random rays in the scene box, all
    traced in one launch, on LBVH and on binned-SAH BLAS (the benchmark's
    build); the oracle checks a seeded sample."""
    s, gs, O = medium
    if blas == "sah":
        gs = rg.GpuScene(s, morton_flags=rg.RG_BLAS_SAH)
    all_cam = camera_rays(s)
    lo, hi = s.world_aabb()
    rnd = g.random_rays(1_000_000, lo, hi, seed=5)
    rays = np.concatenate([all_cam, rnd])
    h = trace(gs, rays)
    idx = np.random.default_rng(0).choice(len(rays), 100_000, replace=False)
    ref = O.trace(rays[idx], kappa=KAPPA, rel_t=REL_T)
    frac = compare_closest({k: v[idx] for k, v in h.items()}, ref, label="medium")
    if blas == "sah":
        gs.close()
    print(f"medium ({blas}): differing (exempt) fraction {frac:.2e}, ambiguous {ref['ambiguous'].mean():.2e}")


def test_bvh_equals_brute_force_bit_exact():
    s = _random_scene(11, 40)
    with rg.GpuScene(s) as gs:
        lo, hi = s.world_aabb()
        rays = g.random_rays(100_000, lo - 5, hi + 5, seed=12)
        a = trace(gs, rays)
        b = trace(gs, rays, rg.RG_TRACE_BRUTE)
        for k in ("inst", "prim"):
            assert np.array_equal(a[k], b[k]), k
        for k in ("t", "u", "v"):
            assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32)), k
        assert (a["inst"] != MISS).mean() > 0.1
        rays[:, 7] = np.random.default_rng(1).uniform(1, 40, len(rays))
        a = trace(gs, rays, rg.RG_ANY)
        b = trace(gs, rays, rg.RG_ANY | rg.RG_TRACE_BRUTE)
        assert np.array_equal(a["inst"] != MISS, b["inst"] != MISS)


def _random_scene(seed, n_inst):
    rng = np.random.default_rng(seed)
    meshes = [g.make_mesh("ico", 2), g.make_mesh("uv", 12, 6), g.cube_mesh(1.0), g.make_mesh("hf", 8, rng=rng),
              (np.array([[0, 0, 0], [2, 0, 0], [0, 2, 0]], np.float32), np.array([[0, 1, 2]], np.uint32))]
    M = []
    for k in range(n_inst):
        R = g.random_rotation(rng)
        if k % 7 == 3:
            R = R @ np.diag([1, 1, -1])   # mirrored instance: negative determinant
        M.append(g.affine(R, rng.uniform(-25, 25, 3), rng.uniform(0.5, 2)))
    M = np.stack(M)
    mid = rng.integers(0, len(meshes), n_inst).astype(np.uint32)
    return g.Scene(meshes=meshes, M=M, mesh_id=mid, material_id=np.zeros(n_inst, np.uint32),
                   mat_type=np.zeros(1, np.uint32), mat_albedo=np.full((1, 3), 0.5, np.float32),
                   mat_ior=np.ones(1, np.float32), light_pos=np.zeros((0, 3), np.float32),
                   light_I=np.zeros((0, 3), np.float32))


def test_random_scene_vs_oracle_with_mirrored_instances():
    s = _random_scene(21, 60)
    with rg.GpuScene(s) as gs:
        lo, hi = s.world_aabb()
        rays = g.random_rays(200_000, lo - 5, hi + 5, seed=22)
        h = trace(gs, rays)
    O = oracle.OracleScene(s)
    ref = O.trace(rays, kappa=KAPPA, rel_t=REL_T)
    compare_closest(h, ref, label="random")


def test_edge_cases():
    cube = g.cube_mesh(0.5)
    tri = (np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32), np.array([[0, 1, 2]], np.uint32))
    s = g.Scene(meshes=[cube, tri], M=np.stack([g.affine(np.eye(3), [0, 0, 0]), g.affine(np.eye(3), [5, 0, 0])]),
                mesh_id=np.array([0, 1], np.uint32), material_id=np.zeros(2, np.uint32),
                mat_type=np.zeros(1, np.uint32), mat_albedo=np.full((1, 3), 0.5, np.float32),
                mat_ior=np.ones(1, np.float32), light_pos=np.zeros((0, 3), np.float32),
                light_I=np.zeros((0, 3), np.float32))
    inf = np.inf
    rays = np.array([
        [0.1, -0.2, 3, 0, 0, 0, -1, inf],       # axis ray onto the +z face: t = 2.5
        [3, 0.1, -0.2, 0, -1, 0, 0, inf],       # onto the +x face
        [0.1, 0.2, 0.0, 0, 0, 1, 0, inf],       # from inside the cube: hits the +y face at t = 0.3
        [0.1, -0.2, 3, 0, 0, 0, 1, inf],        # pointing away: miss
        [0.1, -0.2, 3, 3, 0, 0, -1, 2],         # tmin > tmax: miss
        [0.1, -0.2, 3, 0, 0, 0, -1, 2.5],       # tmax exactly at the hit: hit (closed interval)
        [0.1, -0.2, 3, 0, 0, 0, -1, 2.4999998], # tmax just short: miss
        [5.2, 0.2, 4, 0, 0, 0, -2, inf],        # single-triangle BLAS, unnormalised direction: t = 2
        [0.5, 0.5, 3, 0, 0, 0, -1, inf],        # exactly through a cube edge: some face is hit
    ], np.float32)
    with rg.GpuScene(s) as gs:
        h = trace(gs, rays)
        empty = rg.rg_trace_rays(gs.h, torch.zeros((0, 8), dtype=torch.float32, device="cuda"))
        assert empty.shape == (0, 5)
    # instance 0 is the cube, instance 1 the single triangle
    assert h["inst"][0] == 0 and h["t"][0] == 2.5
    assert h["inst"][1] == 0 and h["t"][1] == 2.5
    assert h["inst"][2] == 0 and abs(h["t"][2] - 0.3) < 1e-7
    assert h["inst"][3] == MISS and h["inst"][4] == MISS
    assert h["inst"][5] == 0 and h["t"][5] == 2.5
    assert h["inst"][6] == MISS
    assert h["inst"][7] == 1 and h["prim"][7] == 0 and h["t"][7] == 2.0
    assert abs(h["u"][7] - 0.2) < 1e-6 and abs(h["v"][7] - 0.2) < 1e-6
    assert h["inst"][8] == 0


def test_stats_mode_same_hits_and_counts(medium):
    s, gs, O = medium
    rays = camera_rays(s, np.arange(0, s.width * s.height, 7, dtype=np.uint32))
    a = trace(gs, rays)
    rg.rg_reset_stats(gs.h)
    b = trace(gs, rays, rg.RG_TRACE_STATS)
    st = rg.rg_get_stats(gs.h)
    for k in a:
        assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32))
    assert st["node_visits"] > len(rays) and st["tri_tests"] > 0 and st["inst_entries"] > 0


def test_refit_equals_fresh_build():
    s = _random_scene(31, 50)
    M2 = g.motion(s.M, 4)
    lo, hi = s.world_aabb()
    rays = g.random_rays(100_000, lo - 5, hi + 5, seed=32)
    with rg.GpuScene(s) as gs:
        gs.refit(M2)
        a = trace(gs, rays)
    s2 = _random_scene(31, 50)
    s2.M = M2
    with rg.GpuScene(s2) as gs:
        b = trace(gs, rays)
    for k in a:
        assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32)), k


def test_injected_allocation_failure_is_reported():
    """RG_FAULT=alloc:N makes the N-th library allocation fail (host side);
    the call returns RG_ERR_OOM and the library stays usable."""
    code = r"""
import numpy as np, torch, paper_2001_09792_gb300 as rg, scenegen as g
v, i = g.cube_mesh(0.5)
h = rg.rg_scene_create()
tv = torch.from_numpy(v).cuda(); ti = torch.from_numpy(i.view(np.int32)).cuda()
try:
    rg.rg_blas_build(h, tv, ti)
    print("NOFAIL")
except rg.RgError as e:
    print("STATUS", e.status)
b = rg.rg_blas_build(h, tv, ti)
rg.rg_sync(h)
print("AFTER", b)
rg.rg_scene_destroy(h)
"""
    env = dict(os.environ, RG_FAULT="alloc:4")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    p = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    assert f"STATUS {rg.RG_ERR_OOM}" in p.stdout and "AFTER 0" in p.stdout, p.stdout


@pytest.mark.parametrize("env,status", [("RG_TEST_STACK=1", "RG_ERR_STACK"), ("RG_TEST_ITER_CAP=3", "RG_ERR_TIMEOUT")])
def test_traversal_limits_report_errors(env, status):
    """A traversal stack of one entry, or an iteration cap of three steps (test
    limits set from the environment; the stack limit applies to the counting
    traversals, which the test uses), is exceeded by most rays of the medium
    scene: the rays come back as misses, the next rg_sync returns the error
    (for rg_trace_rays and rg_render alike), and the scene stays usable.  No
    GPU fault is involved: the kernels record the error and end the ray."""
    code = r"""
import numpy as np, torch, paper_2001_09792_gb300 as rg, scenegen as g
s = g.medium_scene(width=160, height=90, max_depth=2)
with rg.GpuScene(s, flags=rg.RG_SCENE_COUNT) as gs:
    lo, hi = s.world_aabb()
    rays = torch.from_numpy(g.random_rays(20000, lo - 5, hi + 5, seed=9)).cuda()
    hits = rg.split_hits(rg.rg_trace_rays(gs.h, rays, rg.RG_TRACE_STATS))
    try:
        rg.rg_sync(gs.h)
        print("NOERROR")
    except rg.RgError as e:
        print("TRACE", e.status)
    print("MISSES", float((hits["inst"] == 0xFFFFFFFF).mean()))
    rg.rg_render(gs.h, s.camera, s.width, s.height, s.max_depth)
    try:
        rg.rg_sync(gs.h)
        print("NOERROR")
    except rg.RgError as e:
        print("RENDER", e.status)
    rg.rg_sync(gs.h)
    print("USABLE")
"""
    k, v = env.split("=")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    p = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, **{k: v}), cwd=root, capture_output=True,
                       text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    want = getattr(rg, status)
    assert f"TRACE {want}" in p.stdout and f"RENDER {want}" in p.stdout and "USABLE" in p.stdout, p.stdout
    misses = float(p.stdout.split("MISSES")[1].split()[0])
    assert misses > 0.5, p.stdout
