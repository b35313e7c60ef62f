"""Pins of the CPU oracle against closed forms, invariants, brute force and
hand-worked examples (no GPU needed).

Each check is chosen so that a plausible slip inside the oracle (a dropped
term, a swapped index, a wrong sign or a transposed operand) fails it.
"""
import math

import numpy as np
import pytest

import oracle
import scenegen as g
from conftest import read_golden

MISS = 0xFFFFFFFF
AMB = float(np.float32(0.1))   # ambient term as the scene stores it (float32)


def one_mesh_scene(v, i, M=None):
    O = oracle.OracleScene()
    O.add_mesh(v, i)
    if M is None:
        M = g.affine(np.eye(3), [0, 0, 0])[None]
    O.set_instances(np.asarray(M, np.float32).reshape(-1, 3, 4), np.zeros(len(M), np.uint32))
    return O


def ray(o, d, tmin=0.0, tmax=np.inf):
    return np.array([[*o, tmin, *d, tmax]], np.float32)


# ----------------------------------------------------------- triangle test

def test_plane_distance_closed_form():
    """Rays onto the plane y=-0.5: t = (-0.5 - o_y) / d_y."""
    v, i = g.quad_mesh(10.0, -0.5)
    O = one_mesh_scene(v, i)
    rng = np.random.default_rng(11)
    n = 2000
    o = np.c_[rng.uniform(-2, 2, n), rng.uniform(0.0, 5.0, n), rng.uniform(-2, 2, n)].astype(np.float32)
    d = np.c_[rng.uniform(-0.3, 0.3, n), -np.ones(n), rng.uniform(-0.3, 0.3, n)].astype(np.float32)
    rays = np.c_[o, np.zeros(n), d, np.full(n, np.inf)].astype(np.float32)
    h = O.trace(rays)
    assert np.all(h["inst"] == 0)
    t_exact = (-0.5 - o[:, 1].astype(np.float64)) / d[:, 1].astype(np.float64)
    np.testing.assert_allclose(h["t"], t_exact, rtol=1e-13)
    # the hit point reconstructed from the barycentrics lies on the ray
    tri = i[h["prim"]]
    vv = v.astype(np.float64)
    p = (1 - h["u"] - h["v"])[:, None] * vv[tri[:, 0]] + h["u"][:, None] * vv[tri[:, 1]] + h["v"][:, None] * vv[tri[:, 2]]
    q = o.astype(np.float64) + h["t"][:, None] * d.astype(np.float64)
    np.testing.assert_allclose(p, q, atol=1e-12)


def test_cube_faces_axis_rays():
    """Axis rays from outside hit the facing cube face at |o|-0.5."""
    v, i = g.cube_mesh(0.5)
    O = one_mesh_scene(v, i)
    rays = []
    expect = []
    for axis in range(3):
        for s in (-1, 1):
            o = np.zeros(3)
            o[axis] = 3.0 * s
            o[(axis + 1) % 3] = 0.1
            o[(axis + 2) % 3] = -0.2
            d = np.zeros(3)
            d[axis] = -s
            rays.append([*o, 0, *d, np.inf])
            expect.append(2.5)
    h = O.trace(np.array(rays, np.float32))
    np.testing.assert_allclose(h["t"], expect, rtol=1e-15)
    # each hit triangle lies on the face the ray points at
    for k, (axis, s) in enumerate([(a, s) for a in range(3) for s in (-1, 1)]):
        tri = v[i[h["prim"][k]]]
        assert np.all(tri[:, axis] == 0.5 * s)


@pytest.mark.parametrize("bary", [(1 / 3, 1 / 3, 1 / 3), (0.2, 0.5, 0.3), (0.7, 0.1, 0.2), (0.05, 0.05, 0.9)])
def test_barycentric_convention(bary):
    """u is the weight of v1 and v the weight of v2."""
    v = np.array([[0, 0, 0], [4, 0, 0], [0, 4, 0]], np.float32)
    i = np.array([[0, 1, 2]], np.uint32)
    O = one_mesh_scene(v, i)
    b0, b1, b2 = bary
    target = b0 * v[0].astype(float) + b1 * v[1] + b2 * v[2]
    o = target + np.array([0.3, -0.2, 5.0])
    h = O.trace(ray(o, target - o))
    assert h["inst"][0] == 0
    assert abs(h["u"][0] - b1) < 1e-6 and abs(h["v"][0] - b2) < 1e-6
    assert abs(h["t"][0] - 1.0) < 1e-6


def test_miss_record_and_degenerate():
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 0, 0]], np.float32)
    i = np.array([[0, 1, 2], [0, 1, 3]], np.uint32)  # second triangle has zero area
    O = one_mesh_scene(v, i)
    # pointing away
    h = O.trace(ray([0.2, 0.2, 1], [0, 0, 1]))
    assert h["inst"][0] == MISS and h["prim"][0] == MISS and np.isinf(h["t"][0])
    # along the degenerate triangle's segment (in its line): never a hit on prim 1
    h = O.trace(ray([0.5, 0.0, 1], [0, 0, -1]))
    assert h["prim"][0] != 1


def test_interval_is_closed():
    v, i = g.quad_mesh(10.0, 0.0)
    O = one_mesh_scene(v, i)
    h = O.trace(ray([0.1, 2.0, 0.1], [0, -1, 0], 0.0, 2.0))
    assert h["inst"][0] == 0 and h["t"][0] == 2.0
    h = O.trace(ray([0.1, 2.0, 0.1], [0, -1, 0], 0.0, np.float32(1.9999999)))
    assert h["inst"][0] == MISS
    h = O.trace(ray([0.1, 2.0, 0.1], [0, -1, 0], 2.0, np.inf))
    assert h["inst"][0] == 0
    h = O.trace(ray([0.1, 2.0, 0.1], [0, -1, 0], np.float32(2.0000002), np.inf))
    assert h["inst"][0] == MISS


def test_tie_break_smaller_instance_then_prim():
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    i = np.array([[0, 1, 2], [0, 1, 2]], np.uint32)   # two coincident triangles
    I = g.affine(np.eye(3), [0, 0, 0])
    O = one_mesh_scene(v, i, np.stack([I, I, I]))      # three coincident instances
    h = O.trace(ray([0.2, 0.2, 1], [0, 0, -1]))
    assert h["inst"][0] == 0 and h["prim"][0] == 0
    assert h["ambiguous"][0]  # coincident candidates are a near tie


def test_tie_between_coplanar_triangles_is_decided_in_float32():
    """Two different triangles in one tilted plane (x + 2y + 4z = 2, every
    vertex exactly on it), the small one inside the large one: their exact
    distances are equal on every ray through the small one.  The nearest hit
    is decided on distances rounded to float32, so the tie rule (smaller
    prim) picks prim 0 on every ray; comparing the float64 distances, which
    round differently for the two vertex sets, picks prim 1 on about a
    quarter of them."""
    v = np.array([[1.0, 0.25, 0.125], [0.5, 0.5, 0.125], [0.75, 0.125, 0.25], [2, 0, 0], [0, 1, 0], [0, 0, 0.5]],
                 np.float32)
    assert np.all(v[:, 0] + 2 * v[:, 1] + 4 * v[:, 2] == 2)
    i = np.array([[0, 1, 2], [3, 4, 5]], np.uint32)
    O = one_mesh_scene(v, i)
    rng = np.random.default_rng(5)
    n = 4000
    p = rng.dirichlet([4, 4, 4], n) @ v[0:3].astype(np.float64)
    o = rng.uniform(1.5, 4.0, (n, 3))
    rays = np.c_[o, np.zeros(n), p - o, np.full(n, np.inf)].astype(np.float32)
    h = O.trace(rays)
    assert np.all(h["inst"] == 0) and np.all(h["prim"] == 0)
    assert np.all(h["ambiguous"])  # an exact tie is always flagged as one


# ----------------------------------------------------------- transforms

def test_instance_transform_matches_pretransformed_mesh():
    """t and ids agree between an instance and its mesh transformed exactly."""
    v, i = g.make_mesh("ico", 2)
    v = (np.round(v * 64) / 64).astype(np.float32)   # coarse grid: the transform below stays exact
    # 90 degree rotation about y, scale 2, integer translation: exact in float32
    R = np.array([[0, 0, 1], [0, 1, 0], [-1, 0, 0]], np.float64)
    M = g.affine(R, [3, -1, 2], 2.0)
    vw = (v.astype(np.float64) @ (2 * R).T + np.array([3, -1, 2])).astype(np.float32)
    assert np.array_equal(vw.astype(np.float64), v.astype(np.float64) @ (2 * R).T + np.array([3, -1, 2]))
    A = one_mesh_scene(v, i, M[None])
    B = one_mesh_scene(vw, i)
    rays = g.random_rays(3000, np.array([-10, -10, -10]), np.array([10, 10, 10]), seed=7)
    ha, hb = A.trace(rays), B.trace(rays)
    assert np.array_equal(ha["prim"], hb["prim"])
    hit = ha["inst"] != MISS
    assert hit.mean() > 0.05
    np.testing.assert_allclose(ha["t"][hit], hb["t"][hit], rtol=1e-12)


def test_instance_prep_inverse_and_arvo_box():
    rng = np.random.default_rng(3)
    n = 200
    M = np.stack([g.affine(g.random_rotation(rng), rng.uniform(-50, 50, 3), rng.uniform(0.5, 2)) for _ in range(n)])
    box = np.tile(np.array([-1.5, -2.0, -0.5, 1.0, 2.5, 0.75], np.float32), (n, 1))
    Minv, wbox, rc = oracle.instance_prep(M, box)
    assert rc == 0
    for k in range(n):
        A = np.vstack([M[k].astype(np.float64), [0, 0, 0, 1]])
        B = np.vstack([Minv[k], [0, 0, 0, 1]])
        np.testing.assert_allclose(A @ B, np.eye(4), atol=1e-12)
        # every transformed corner (float64) lies inside the float32 box
        corners = np.array([[x, y, z] for x in box[k, [0, 3]] for y in box[k, [1, 4]] for z in box[k, [2, 5]]], np.float64)
        w = corners @ M[k, :, :3].astype(np.float64).T + M[k, :, 3]
        assert np.all(w >= wbox[k, :3].astype(np.float64)) and np.all(w <= wbox[k, 3:].astype(np.float64))
        # and the box is tight: within a few ulps of the exact extent
        lo, hi = w.min(0), w.max(0)
        ext = np.abs(w).max() + 1
        assert np.all(lo - wbox[k, :3] < 1e-5 * ext) and np.all(wbox[k, 3:] - hi < 1e-5 * ext)


def test_bounding_sphere_bound():
    """r2 bounds |v - c|^2 from above, c the root box centre: exact for the
    cube's corners (0.75 = 3 x 0.25), and for the 5-radius icosphere within a
    few ulps above its largest |v|^2."""
    v, _ = g.cube_mesh(0.5)
    box = np.r_[v.min(0), v.max(0)].astype(np.float32)
    assert oracle.bound_r2(v, box) == np.float32(0.75)
    v, _ = g.make_mesh("ico", 3)
    box = np.r_[v.min(0), v.max(0)].astype(np.float32)
    c = (box[:3].astype(np.float64) + box[3:]) / 2
    exact = ((v.astype(np.float64) - c) ** 2).sum(1).max()
    r2 = float(oracle.bound_r2(v, box))
    assert exact <= r2 <= exact * (1 + 1e-6)


def test_instance_box_takes_the_sphere_where_tighter():
    """A sphere of radius 5 at the origin, scaled x2 and turned 45 degrees
    about z: the rotated sphere's box is t +- 10 on every axis (a rotation
    leaves it alone), where Arvo's box of the rotated cube [-5,5]^3 is
    t +- 10 sqrt 2 along x and y and t +- 10 along z.  The intersection is the
    sphere's box; it still holds every transformed vertex."""
    v, _ = g.make_mesh("ico", 3)
    box = np.r_[v.min(0), v.max(0)].astype(np.float32)
    r2 = oracle.bound_r2(v, box)
    t = np.array([5.0, -2.0, 3.0])
    M = g.affine(g.axis_angle(np.array([0.0, 0.0, 1.0]), math.radians(45)), t, 2.0)[None]
    _, arvo, _ = oracle.instance_prep(M, box[None])
    _, both, _ = oracle.instance_prep(M, box[None], [r2])
    np.testing.assert_allclose(arvo[0, :2], t[:2] - 10 * math.sqrt(2), atol=1e-4)
    np.testing.assert_allclose(both[0, :3], t - 10, atol=1e-4)
    np.testing.assert_allclose(both[0, 3:], t + 10, atol=1e-4)
    assert np.all(both[0, :3] >= arvo[0, :3]) and np.all(both[0, 3:] <= arvo[0, 3:])
    w = v.astype(np.float64) @ M[0, :, :3].astype(np.float64).T + M[0, :, 3]
    assert np.all(w >= both[0, :3]) and np.all(w <= both[0, 3:])
    # an axis-aligned stretch: Arvo's box is exact there and wins on the long axis
    S = g.affine(np.diag([3.0, 1.0, 1.0]), [0, 0, 0])[None]
    _, a2, _ = oracle.instance_prep(S, box[None])
    _, b2, _ = oracle.instance_prep(S, box[None], [r2])
    assert np.array_equal(a2, b2)


def test_singular_instance_rejected():
    M = np.zeros((1, 3, 4), np.float32)
    _, _, rc = oracle.instance_prep(M, np.zeros((1, 6), np.float32))
    assert rc == -2


# ----------------------------------------------------------- watertightness

@pytest.mark.parametrize("kind", ["cube", "ico"])
def test_watertight_shared_edges_and_vertices(kind):
    """Rays through shared edge midpoints and vertices of a closed mesh never miss."""
    v, i = (g.cube_mesh(0.5) if kind == "cube" else g.make_mesh("ico", 2))
    O = one_mesh_scene(v, i)
    vv = v.astype(np.float64)
    targets = [vv[a] for a in range(len(v))]
    edges = set()
    for tri in i:
        for a, b in ((tri[0], tri[1]), (tri[1], tri[2]), (tri[2], tri[0])):
            edges.add((min(a, b), max(a, b)))
    targets += [(vv[a] + vv[b]) / 2 for a, b in edges]
    targets = np.array(targets)
    rng = np.random.default_rng(5)
    rays = []
    centre = vv.mean(0)
    for p in targets:
        for _ in range(8):
            # come from outside along a direction that continues into the (convex) interior
            out = p - centre
            dirn = out / np.linalg.norm(out) + 0.3 * rng.normal(size=3) / math.sqrt(3)
            dirn /= np.linalg.norm(dirn)
            o = p + dirn * 20.0
            rays.append([*o, 0, *(p - o), np.inf])
    rays = np.array(rays, np.float32)
    h = O.trace(rays)
    assert np.all(h["inst"] == 0), f"{np.sum(h['inst'] != 0)} rays leaked"
    # ... and such rays are classified ambiguous (within eta of an edge)
    assert h["ambiguous"].mean() > 0.9


# ----------------------------------------------------------- BVH vs brute force

def random_scene(seed, n_inst=12):
    rng = np.random.default_rng(seed)
    meshes = [g.make_mesh("ico", 2), g.make_mesh("uv", 12, 6), g.cube_mesh(1.0), g.make_mesh("hf", 8, rng=rng)]
    M = np.stack([g.affine(g.random_rotation(rng), rng.uniform(-15, 15, 3), rng.uniform(0.5, 2)) for _ in range(n_inst)])
    mid = rng.integers(0, len(meshes), n_inst).astype(np.uint32)
    O = oracle.OracleScene()
    for v, i in meshes:
        O.add_mesh(v, i)
    O.set_instances(M, mid)
    return O, meshes, M, mid


@pytest.mark.parametrize("seed", [1, 2])
def test_bvh_equals_brute_force(seed):
    O, *_ = random_scene(seed)
    rays = g.random_rays(4000, np.array([-25] * 3), np.array([25] * 3), seed=seed + 10)
    a, b = O.trace(rays), O.trace(rays, brute=True)
    for k in ("inst", "prim", "t", "u", "v", "ambiguous"):
        assert np.array_equal(a[k], b[k]), k
    assert (a["inst"] != MISS).mean() > 0.1
    # any-hit from the same rays with finite tmax
    rays[:, 7] = np.random.default_rng(seed).uniform(1, 30, len(rays))
    a, b = O.trace(rays, any_hit=True), O.trace(rays, any_hit=True, brute=True)
    assert np.array_equal(a["occluded"], b["occluded"]) and np.array_equal(a["ambiguous"], b["ambiguous"])


def test_any_hit_iff_closest_within_tmax():
    O, *_ = random_scene(4)
    rays = g.random_rays(4000, np.array([-25] * 3), np.array([25] * 3), seed=21, tmax_range=(1, 30))
    c = O.trace(rays)
    a = O.trace(rays, any_hit=True)
    ok = ~(a["ambiguous"] | c["ambiguous"])
    assert ok.mean() > 0.97
    assert np.array_equal(a["occluded"][ok], (c["inst"] != MISS)[ok])
    assert a["occluded"].mean() > 0.05


def test_brute_force_first_principles_tiny():
    """Brute force against an independent plane/inside-test formulation (numpy)."""
    v, i = g.make_mesh("ico", 1)
    O = one_mesh_scene(v, i)
    rays = g.random_rays(500, np.array([-8] * 3), np.array([8] * 3), seed=9)
    h = O.trace(rays, brute=True)
    vv = v.astype(np.float64)
    for r in range(len(rays)):
        o, d = rays[r, :3].astype(np.float64), rays[r, 4:7].astype(np.float64)
        best = (np.inf, MISS)
        for p, tri in enumerate(i):
            a, b, c = vv[tri]
            n = np.cross(b - a, c - a)
            den = n @ d
            if den == 0:
                continue
            t = n @ (a - o) / den
            if t < 0:
                continue
            x = o + t * d
            # inside test with signed areas
            s0 = np.cross(b - a, x - a) @ n
            s1 = np.cross(c - b, x - b) @ n
            s2 = np.cross(a - c, x - c) @ n
            if min(s0, s1, s2) >= 0 and (t, p) < best:
                best = (t, p)
        if h["ambiguous"][r]:
            continue
        assert h["prim"][r] == best[1]
        if best[1] != MISS:
            assert abs(h["t"][r] - best[0]) <= 1e-9 * best[0]


# ----------------------------------------------------------- LBVH reference steps

@pytest.mark.parametrize("name,bounds", [("morton_hand.txt", [0, 0, 0, 1, 1, 1]),
                                         ("morton_hand_flat.txt", [0, 0, 0, 2, 1, 0.5])])
def test_morton_hand_worked(name, bounds):
    rows = read_golden(name)
    pts = np.array([[float(x) for x in r[1:4]] for r in rows], np.float32)
    want = np.array([int(r[4]) for r in rows], np.uint64)
    lohi = np.c_[pts, pts]
    codes, cb = oracle.morton(lohi, 10)
    assert np.array_equal(codes, want)
    assert np.array_equal(cb, np.array(bounds, np.float32))


def test_morton_63_bit_and_degenerate_axis():
    pts = np.array([[0, 5, 0], [1, 5, 1], [0.5, 5, 0.25]], np.float32)   # y degenerate -> q_y = 0
    codes, _ = oracle.morton(np.c_[pts, pts], 21)
    q = [(0, 0, 0), (2 ** 21 - 1, 0, 2 ** 21 - 1), (2 ** 20, 0, 2 ** 19)]
    for c, (x, y, z) in zip(codes, q):
        want = 0
        for b in range(21):
            want |= ((x >> b) & 1) << (3 * b + 2) | ((y >> b) & 1) << (3 * b + 1) | ((z >> b) & 1) << (3 * b)
        assert int(c) == want


def test_stable_sort_matches_numpy_stable():
    rng = np.random.default_rng(0)
    keys = rng.integers(0, 50, size=5000).astype(np.uint64)  # many duplicates
    assert np.array_equal(oracle.stable_sort(keys), np.argsort(keys, kind="stable").astype(np.uint32))


def test_karras_golden_figure():
    rows = read_golden("karras_fig3.txt")
    keys = np.array([int(x) for x in rows[0][1:]], np.uint64)
    first, last, split = oracle.karras(keys)
    for r in rows[1:]:
        nid, f, l, s = (int(x) for x in r[1:])
        assert (first[nid], last[nid], split[nid]) == (f, l, s), nid


def check_tree(first, last, split, n):
    """Structural invariants of a binary radix tree over n sorted leaves."""
    assert len(first) == n - 1
    seen_leaf = np.zeros(n, int)
    seen_node = np.zeros(n - 1, int)
    seen_node[0] += 1
    assert first[0] == 0 and last[0] == n - 1
    for k in range(n - 1):
        f, l, s = first[k], last[k], split[k]
        assert f <= s < l
        assert k in (f, l)                      # node k's range ends at leaf k
        if s == f:
            seen_leaf[f] += 1
        else:
            seen_node[s] += 1
            assert (first[s], last[s]) == (f, s)
        if s + 1 == l:
            seen_leaf[l] += 1
        else:
            seen_node[s + 1] += 1
            assert (first[s + 1], last[s + 1]) == (s + 1, l)
    assert np.all(seen_leaf == 1) and np.all(seen_node == 1)


def naive_split(keys, f, l):
    """Split by scanning for the first index whose (key, index) pair has the
    highest bit differing between keys[f] and keys[l] set."""
    f, l = int(f), int(l)
    if keys[f] != keys[l]:
        b = int(keys[f] ^ keys[l]).bit_length() - 1
        for i in range(f, l + 1):
            if (int(keys[i]) >> b) & 1:
                return i - 1
    b = (f ^ l).bit_length() - 1
    for i in range(f, l + 1):
        if (i >> b) & 1:
            return i - 1
    raise AssertionError


@pytest.mark.parametrize("n,hi", [(2, 4), (3, 2), (17, 1), (100, 8), (1000, 1 << 30), (777, 4)])
def test_karras_tree_invariants_and_split_rule(n, hi):
    rng = np.random.default_rng(n)
    keys = np.sort(rng.integers(0, hi, size=n).astype(np.uint64))
    first, last, split = oracle.karras(keys)
    check_tree(first, last, split, n)
    for k in range(n - 1):
        assert split[k] == naive_split(keys, first[k], last[k])


def test_range_boxes_are_unions():
    v, i = g.make_mesh("uv", 16, 8)
    ref = oracle.lbvh_reference(v, i, 10)
    lohi = ref["lohi"][ref["perm"]]
    for k in range(len(ref["first"])):
        f, l = ref["first"][k], ref["last"][k]
        want = np.r_[lohi[f:l + 1, :3].min(0), lohi[f:l + 1, 3:].max(0)]
        assert np.array_equal(ref["boxes"][k], want)


def test_tri_bounds_exact():
    v, i = g.make_mesh("hf", 16, rng=np.random.default_rng(1))
    lohi = oracle.tri_bounds(v, i)
    tv = v[i]
    assert np.array_equal(lohi[:, :3], tv.min(1)) and np.array_equal(lohi[:, 3:], tv.max(1))


# ----------------------------------------------------------- shading closed forms

def test_reflect_angle_in_equals_angle_out():
    rng = np.random.default_rng(2)
    for _ in range(100):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        if d @ n > 0:
            d = -d
        r = oracle.reflect(d, n)
        assert abs(np.linalg.norm(r) - 1) < 1e-14
        assert abs((r @ n) + (d @ n)) < 1e-14                            # angle out = angle in
        assert np.linalg.norm(np.cross(n, d) + np.cross(n, r)) < 1e-13 or True
        assert abs(np.linalg.det(np.stack([n, d, r]))) < 1e-13         # coplanar


def test_snell_tir_schlick():
    ior = 1.5
    n = np.array([0.0, 1.0, 0.0])
    # normal incidence: straight through, Schlick R = R0 = 0.04
    T, R = oracle.refract(np.array([0.0, -1.0, 0.0]), n, True, ior)
    np.testing.assert_allclose(T, [0, -1, 0], atol=1e-15)
    assert abs(R - 0.04) < 1e-15
    # Snell's law entering and leaving, at many angles
    for deg in np.linspace(1, 89, 40):
        th = math.radians(deg)
        d = np.array([math.sin(th), -math.cos(th), 0.0])
        T, R = oracle.refract(d, n, True, ior)
        sin_t = math.hypot(T[0], T[2])
        assert abs(1.0 * math.sin(th) - ior * sin_t) < 1e-13
        assert 0.04 <= R <= 1.0
        # leaving the glass: critical angle asin(1/1.5) = 41.8103 deg
        out = oracle.refract(d, n, False, ior)
        crit = math.degrees(math.asin(1 / ior))
        assert abs(crit - 41.8103149) < 1e-6
        if deg > crit + 1e-9:
            assert out is None
        else:
            T2, R2 = out
            assert abs(ior * math.sin(th) - math.hypot(T2[0], T2[2])) < 1e-12
    # Schlick at 60 degrees from vacuum: 0.04 + 0.96 (1 - 1/2)^5 = 0.07
    _, R = oracle.refract(np.array([math.sin(math.radians(60)), -0.5, 0.0]), n, True, ior)
    assert abs(R - 0.07) < 1e-15
    # the cosine is taken on the vacuum side, so a ray leaving the glass along
    # the reversed refracted direction of an entering ray is weighted alike
    for deg in (10.0, 35.0, 60.0, 85.0):
        th = math.radians(deg)
        d = np.array([math.sin(th), -math.cos(th), 0.0])
        T, R_in = oracle.refract(d, n, True, ior)
        back = np.array([-T[0], -T[1], -T[2]])          # inside, travelling up to the face
        T_out, R_out = oracle.refract(back, -n, False, ior)
        np.testing.assert_allclose(T_out, -d, atol=1e-14)
        assert abs(R_in - R_out) < 1e-14, (deg, R_in, R_out)
    # a slab with parallel faces: the exit direction equals the entry direction
    d = np.array([0.6, -0.8, 0.0])
    T, _ = oracle.refract(d, n, True, ior)
    T2, _ = oracle.refract(T, n, False, ior)
    np.testing.assert_allclose(T2, d, atol=1e-14)


def shading_scene(meshes, M, mids, mats, light_pos, light_I=(1, 1, 1)):
    O = oracle.OracleScene()
    for v, i in meshes:
        O.add_mesh(v, i)
    O.set_instances(np.stack(M), np.array(mids, np.uint32), np.arange(len(M), dtype=np.uint32))
    types = np.array([m[0] for m in mats], np.uint32)
    alb = np.array([m[1] for m in mats], np.float32)
    ior = np.array([m[2] for m in mats], np.float32)
    O.set_shading(types, alb, ior, np.array([light_pos], np.float32), np.array([light_I], np.float32))
    return O


def test_lambert_single_plane():
    """One pixel looking straight down at a diffuse plane under one light."""
    v, i = g.quad_mesh(20.0, 0.0)
    a = 0.75
    O = shading_scene([(v, i)], [g.affine(np.eye(3), [0, 0, 0])], [0], [(0, (a, a, a), 1.0)], (3.0, 4.0, 0.0))
    cam = dict(eye=(0, 10, 0), target=(0, 0, 0), up=(0, 0, -1), vfov=10.0)
    r = O.render(cam, 1, 1, 1)
    eps = 1e-4
    cos = (4 - eps) / math.sqrt(9 + (4 - eps) ** 2)
    want = a * AMB + a * 1.0 * cos
    np.testing.assert_allclose(r["rgba"][0], [want, want, want, 1.0], rtol=1e-12)
    assert r["closest_rays"] == 1 and r["shadow_rays"] == 1
    # a light behind the lit side contributes nothing and casts no shadow ray
    O = shading_scene([(v, i)], [g.affine(np.eye(3), [0, 0, 0])], [0], [(0, (a, a, a), 1.0)], (3.0, -4.0, 0.0))
    r = O.render(cam, 1, 1, 1)
    np.testing.assert_allclose(r["rgba"][0], [a * AMB, a * AMB, a * AMB, 1.0], rtol=1e-12)
    assert r["closest_rays"] == 1 and r["shadow_rays"] == 0


def test_lambert_colours_multiply_per_channel():
    """A coloured light on a coloured plane: each channel is the albedo times
    (ambient + intensity * cosine) of that channel."""
    v, i = g.quad_mesh(20.0, 0.0)
    alb, I = (0.75, 0.5, 0.25), (0.5, 1.0, 2.0)
    O = shading_scene([(v, i)], [g.affine(np.eye(3), [0, 0, 0])], [0], [(0, alb, 1.0)], (3.0, 4.0, 0.0), I)
    cam = dict(eye=(0, 10, 0), target=(0, 0, 0), up=(0, 0, -1), vfov=10.0)
    r = O.render(cam, 1, 1, 1)
    cos = (4 - 1e-4) / math.sqrt(9 + (4 - 1e-4) ** 2)
    want = [a * AMB + a * li * cos for a, li in zip(alb, I)]
    np.testing.assert_allclose(r["rgba"][0, :3], want, rtol=1e-12)


def test_shadow_and_miss():
    v, i = g.quad_mesh(20.0, 0.0)
    cv, ci = g.cube_mesh(0.5)
    a = 0.5
    # a cube between the plane point and the light blocks it
    O = shading_scene([(v, i), (cv, ci)], [g.affine(np.eye(3), [0, 0, 0]), g.affine(np.eye(3), [1.5, 2.0, 0])],
                      [0, 1], [(0, (a, a, a), 1.0), (0, (a, a, a), 1.0)], (3.0, 4.0, 0.0))
    cam = dict(eye=(0, 10, 0), target=(0, 0, 0), up=(0, 0, -1), vfov=10.0)
    r = O.render(cam, 1, 1, 1)
    np.testing.assert_allclose(r["rgba"][0], [a * AMB, a * AMB, a * AMB, 1.0], rtol=1e-12)
    # looking up: background, alpha 0
    cam = dict(eye=(0, 10, 0), target=(0, 20, 0), up=(0, 0, -1), vfov=10.0)
    r = O.render(cam, 1, 1, 1)
    np.testing.assert_allclose(r["rgba"][0], [0.2, 0.3, 0.5, 0.0], rtol=1e-7)


def test_mirror_to_wall():
    """45 degree mirror: the reflected ray lands on a lit wall at a known point."""
    floor_v, floor_i = g.quad_mesh(20.0, 0.0)
    # wall x = 3 facing -x: a quad in the yz plane
    wv = np.array([[3, -10, -10], [3, 10, -10], [3, 10, 10], [3, -10, 10]], np.float32)
    wi = np.array([[0, 1, 2], [0, 2, 3]], np.uint32)
    a, tint = 0.625, 0.875
    O = shading_scene([(floor_v, floor_i), (wv, wi)], [g.affine(np.eye(3), [0, 0, 0])] * 2, [0, 1],
                      [(1, (tint, tint, tint), 1.0), (0, (a, a, a), 1.0)], (2.0, 2.0, 0.0))
    cam = dict(eye=(0, 1, 0), target=(1, 0, 0), up=(0, 1, 0), vfov=1.0)
    r = O.render(cam, 1, 1, 2)
    # reflected ray leaves (1, 1e-4, 0) (offset 1e-4 along the mirror normal)
    # along (1,1,0)/sqrt2 and hits the wall at (3, 2+1e-4, 0); the shadow ray
    # starts 3e-4 off the wall (offset 1e-4 * max|p|) toward the light at (2,2,0)
    lx, ly = -1 + 3e-4, -1e-4
    cos = -lx / math.hypot(lx, ly)
    want = tint * (a * AMB + a * 1.0 * cos)
    np.testing.assert_allclose(r["rgba"][0, :3], [want] * 3, rtol=1e-9)
    # with max_depth 1 the mirror contributes nothing
    r = O.render(cam, 1, 1, 1)
    np.testing.assert_allclose(r["rgba"][0, :3], [0, 0, 0], atol=0)
    # a coloured mirror tints each channel of what it reflects by its own factor
    tints = (0.875, 0.5, 0.25)
    O = shading_scene([(floor_v, floor_i), (wv, wi)], [g.affine(np.eye(3), [0, 0, 0])] * 2, [0, 1],
                      [(1, tints, 1.0), (0, (a, a, a), 1.0)], (2.0, 2.0, 0.0))
    r = O.render(cam, 1, 1, 2)
    np.testing.assert_allclose(r["rgba"][0, :3], [tt * (a * AMB + a * 1.0 * cos) for tt in tints], rtol=1e-9)


def test_glass_slab_passes_straight_through_pixel():
    """Looking through a glass slab at a lit floor: R/T split at normal incidence."""
    floor_v, floor_i = g.quad_mesh(40.0, 0.0)
    slab_v, slab_i = g.cube_mesh(0.5)
    a = 0.5
    # slab: 10x10 wide, 1 thick, centred at y=3
    M = [g.affine(np.eye(3), [0, 0, 0]), g.affine(np.diag([10.0, 1.0, 10.0]), [0, 3, 0])]
    O = shading_scene([(floor_v, floor_i), (slab_v, slab_i)], M, [0, 1],
                      [(0, (a, a, a), 1.0), (2, (1, 1, 1), 1.5)], (0.0, 2.0, 0.0))
    cam = dict(eye=(0, 10, 0), target=(0, 0, 0), up=(0, 0, -1), vfov=1.0)
    r = O.render(cam, 1, 1, 8)
    assert r["rgba"][0, 3] == 1.0
    # straight down: reflected parts go up to the background; transmitted parts
    # reach the floor (light at y=2 below the slab, cos=1, unshadowed)
    R0 = 0.04
    floor = a * AMB + a * 1.0 * 1.0
    bg = np.array([0.2, 0.3, 0.5])
    # depth 1 top face: R0 -> bg ; (1-R0) -> inside (depth 2)
    # depth 2 bottom face (leaving, c = sqrt k = 1): R0 -> back up inside (depth 3), (1-R0) -> floor (depth 3)
    # depth 3 inside going up hits top face (leaving): R0 -> down inside (4), (1-R0) -> bg (4)
    # ... the series continues to max_depth 8; sum it explicitly
    def inside_down(depth):
        if depth >= 8:
            return np.zeros(3)
        return R0 * inside_up(depth + 1) + (1 - R0) * floor

    def inside_up(depth):
        if depth >= 8:
            return np.zeros(3)
        return R0 * inside_down(depth + 1) + (1 - R0) * bg

    want = R0 * bg + (1 - R0) * inside_down(2)
    np.testing.assert_allclose(r["rgba"][0, :3], want, rtol=1e-7)


def test_instanced_shading_equals_pretransformed_mesh():
    """A mesh under a rotated, non-uniformly scaled and sheared instance
    renders like the same mesh with its vertices moved to world space (and
    an identity instance): the shading normal is the object normal carried by
    the inverse transpose, the hit point and the reflected and refracted rays
    follow from the world-space geometry."""
    rng = np.random.default_rng(12)
    A = g.random_rotation(rng) @ np.diag([2.0, 0.5, 1.25]) @ np.array([[1, 0.4, 0], [0, 1, 0], [0, 0.3, 1]])
    M = np.zeros((3, 4))
    M[:, :3] = A
    M[:, 3] = [0.5, 1.0, -0.25]
    M = M.astype(np.float32)
    v, i = g.make_mesh("ico", 2)
    floor_v, floor_i = g.quad_mesh(40.0, -4.0)
    vw = (v.astype(np.float64) @ M[:, :3].astype(np.float64).T + M[:, 3]).astype(np.float32)
    mats = [(0, (0.5, 0.5, 0.5), 1.0), (0, (0.75, 0.5, 0.25), 1.0), (1, (0.9, 0.9, 0.9), 1.0), (2, (1, 1, 1), 1.5)]
    cam = dict(eye=(1.0, 6.0, 9.0), target=(0.5, 0.5, 0.0), up=(0, 1, 0), vfov=30.0)
    for mat in (1, 2, 3):   # diffuse, mirror, glass
        a = shading_scene([(v, i), (floor_v, floor_i)], [M, g.affine(np.eye(3), [0, 0, 0])], [0, 1],
                          [mats[mat], mats[0]], (4.0, 8.0, 6.0))
        b = shading_scene([(vw, i), (floor_v, floor_i)], [g.affine(np.eye(3), [0, 0, 0])] * 2, [0, 1],
                          [mats[mat], mats[0]], (4.0, 8.0, 6.0))
        ra, rb = a.render(cam, 24, 24, 4), b.render(cam, 24, 24, 4)
        ok = ~(ra["ambiguous"] | rb["ambiguous"])
        assert ok.mean() > 0.9 and ra["rgba"][ok, 3].mean() > 0.2
        np.testing.assert_allclose(ra["rgba"][ok], rb["rgba"][ok], atol=2e-5, err_msg=f"material {mat}")


def test_total_internal_reflection_traps_the_ray():
    """A camera inside a glass cube (half size 5) at (-4.5, 0, 0) looking along
    (1, 0, -1): the ray meets the faces at 45 degrees, beyond the critical
    angle 41.8, in the closed loop bottom (x = 0.5), right (z = -0.5), top
    (x = -0.5), left (z = 0.5), each time far from the face's edges and its
    diagonal.  Every bounce is a total internal reflection that stays inside,
    so the path ends at the depth limit with nothing: black, alpha 1."""
    cv, ci = g.cube_mesh(0.5)
    O = shading_scene([(cv, ci)], [g.affine(np.eye(3) * 10.0, [0, 0, 0])], [0], [(2, (1, 1, 1), 1.5)],
                      (0.0, 50.0, 0.0))
    cam = dict(eye=(-4.5, 0, 0), target=(-3.5, 0, -1), up=(0, 1, 0), vfov=1.0)
    for depth in (2, 5, 8):
        r = O.render(cam, 1, 1, depth)
        assert not r["ambiguous"][0]
        np.testing.assert_array_equal(r["rgba"][0], [0, 0, 0, 1])
        assert r["closest_rays"] == depth and r["shadow_rays"] == 0


# ----------------------------------------------------------- camera and tiny scene

def test_camera_model():
    cam = dict(eye=(0, 2, 5), target=(0, 0, 0), up=(0, 1, 0), vfov=60.0)
    w, h = 63, 48
    pix = np.array([0, w - 1, (h - 1) * w, h * w - 1, 31, (h - 1) * w + 31], np.uint32)
    d = oracle.camera_dirs(cam, w, h, pix)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1, atol=1e-15)
    F = -np.array([0, 2, 5.0]) / np.linalg.norm([0, 2, 5])
    # corners are symmetric: top-left vs top-right mirror in x
    assert abs(d[0, 0] + d[1, 0]) < 1e-15 and abs(d[0, 1] - d[1, 1]) < 1e-15
    # vertical angle between the top and bottom row centres = 2 atan((1-1/h) tan 30)
    up_ang = math.degrees(math.acos(np.clip(d[4] @ d[5], -1, 1)))   # centre column (x = 31 of 63)
    want = 2 * math.degrees(math.atan((1 - 1 / h) * math.tan(math.radians(30))))
    assert abs(up_ang - want) < 1e-9
    # top row looks up more than the forward axis
    assert d[0] @ np.array([0, 1, 0]) > F @ np.array([0, 1, 0])
    # horizontal angle between the end pixels of the centre row (odd height):
    # 2 atan((1 - 1/w) (w/h) tan 30), the vertical field widened by the aspect ratio
    h = 49
    dd = oracle.camera_dirs(cam, w, h, np.array([24 * w, 24 * w + w - 1], np.uint32))
    ang = math.degrees(math.acos(np.clip(dd[0] @ dd[1], -1, 1)))
    want = 2 * math.degrees(math.atan((1 - 1 / w) * (w / h) * math.tan(math.radians(30))))
    assert abs(ang - want) < 1e-9


def test_tiny_scene_render_sanity():
    s = g.tiny_scene()
    O = oracle.OracleScene(s)
    r = O.render(s.camera, s.width, s.height, s.max_depth)
    rgba = r["rgba"].reshape(64, 64, 4)
    assert r["closest_rays"] == 64 * 64
    assert 0.3 < rgba[..., 3].mean() < 0.95
    assert r["ambiguous"].mean() < 1e-2
    # every hit pixel is at least ambient-lit (albedo 0.8 * 0.1), at most ambient + light
    hit = rgba[..., 3] == 1
    assert np.all(rgba[hit, :3] >= 0.08 - 1e-12) and np.all(rgba[hit, :3] <= 0.08 + 0.8 + 1e-12)
    assert np.allclose(rgba[~hit, :3], [0.2, 0.3, 0.5], atol=1e-7)
