"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module only *produces inputs*: procedural triangle meshes, instance
transforms, materials, lights, cameras and ray buffers, all as float32/uint32
numpy arrays.  It holds none of the ray tracer's arithmetic (no BVH, no
intersection, no shading, no camera-ray generation): both sides consume the
identical arrays it returns.

The paper drives its renderer with game scenes loaded from COLLADA files
(Sec. 2.2); none are available, so seeded procedural scenes stand in for them.
Recipe (sizes and distributions):

* tiny    : unit cube [-0.5,0.5]^3 (12 tris) on a 10x10 ground quad at y=-0.5
            (2 tris); instances = ground (identity), cube (identity),
            cube (T(2,0,-1) R_y(30 deg)); camera (0,2,5) -> origin, vfov 60;
            one light (2,4,3) intensity 1; all diffuse albedo 0.8; 64x64.
* medium  : 4 meshes (UV sphere 80x40 = 6,400 tris, icosphere subdiv 5 =
            20,480, cube = 12, 256x256-cell value-noise heightfield =
            131,072), each centred, normalised to bounding radius 1 and scaled
            x10 (so that about half the primary rays hit); 64 instances with mesh uniform, scale U(0.5,2), rotation
            uniform on SO(3) (Shoemake), translation U[-50,50]^3; materials
            60% diffuse (albedo U[0.2,0.9]^3) / 20% mirror (tint 0.9) / 20%
            glass (IOR 1.5); 4 lights in [-50,50]x[40,60]x[-50,50] at 0.25;
            camera (0,0,100) -> origin, vfov 60; 1920x1080, max depth 4.
* large   : 16 meshes (UV spheres, icospheres, heightfields, tori; 1,938,944
            unique tris, scaled x5), 4,096 instances with per-mesh counts proportional
            to tris^-0.77 (largest remainder), transforms as medium in a
            [-200,200]^3 box; 16M closest-hit rays with origins uniform in the
            scene AABB and directions uniform on the sphere, 16M any-hit rays
            of length U(1,50); per-frame seeded motion.

Seeds: scene 1, rays 2, motion 3, serving arrivals 4.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_SCENE = 1
SEED_RAYS = 2
SEED_MOTION = 3
SEED_SERVE = 4

MAT_DIFFUSE = 0
MAT_MIRROR = 1
MAT_GLASS = 2


# --------------------------------------------------------------------------
# meshes (float64 while generating, float32 on output; CCW = outward normal)
# --------------------------------------------------------------------------

def _f32(v, i):
    return np.ascontiguousarray(v, dtype=np.float32), np.ascontiguousarray(i, dtype=np.uint32)


def cube_mesh(half=0.5):
    """Axis-aligned cube [-half, half]^3, 8 vertices, 12 triangles."""
    h = half
    v = np.array([[x, y, z] for x in (-h, h) for y in (-h, h) for z in (-h, h)], dtype=np.float64)

    def vid(x, y, z):
        return (x > 0) * 4 + (y > 0) * 2 + (z > 0) * 1

    faces = []
    # each face as a quad (a, b, c, d) counter-clockwise seen from outside
    for axis in range(3):
        for sgn in (-1, 1):
            # corners on the face, in CCW order around the outward normal
            u_ax, w_ax = (axis + 1) % 3, (axis + 2) % 3
            quad = []
            for (su, sw) in ((-1, -1), (1, -1), (1, 1), (-1, 1)):
                p = [0, 0, 0]
                p[axis] = sgn
                p[u_ax] = su
                p[w_ax] = sw
                quad.append(vid(*p))
            if sgn < 0:
                quad = quad[::-1]
            a, b, c, d = quad
            faces += [(a, b, c), (a, c, d)]
    return _f32(v, np.array(faces))


def quad_mesh(size=10.0, y=-0.5):
    """Horizontal square of side `size` at height y, normal +y (2 triangles)."""
    s = size / 2
    v = np.array([[-s, y, -s], [s, y, -s], [s, y, s], [-s, y, s]], dtype=np.float64)
    # +y normal: (p0, p3, p2), (p0, p2, p1)
    i = np.array([[0, 3, 2], [0, 2, 1]])
    return _f32(v, i)


def uv_sphere(nu, nv):
    """Latitude/longitude sphere with nu segments around and nv rings.

    Pole quads are kept whole, so 2*nu of the 2*nu*nv triangles are degenerate
    (two coincident pole vertices)."""
    j = np.arange(nv + 1)[:, None]
    i = np.arange(nu)[None, :]
    th = math.pi * j / nv
    ph = 2 * math.pi * i / nu
    v = np.stack([np.sin(th) * np.cos(ph), np.cos(th) * np.ones_like(ph), np.sin(th) * np.sin(ph)], -1)
    v[0] = (0.0, 1.0, 0.0)     # exact poles: the pole triangles are exactly degenerate
    v[nv] = (0.0, -1.0, 0.0)
    v = v.reshape(-1, 3)
    jj, ii = np.meshgrid(np.arange(nv), np.arange(nu), indexing="ij")
    p00 = jj * nu + ii
    p10 = jj * nu + (ii + 1) % nu
    p01 = (jj + 1) * nu + ii
    p11 = (jj + 1) * nu + (ii + 1) % nu
    t1 = np.stack([p00, p10, p11], -1).reshape(-1, 3)
    t2 = np.stack([p00, p11, p01], -1).reshape(-1, 3)
    idx = np.stack([t1, t2], 1).reshape(-1, 3)
    return v, idx


def icosphere(subdiv):
    """Icosahedron subdivided `subdiv` times, vertices on the unit sphere."""
    t = (1 + math.sqrt(5)) / 2
    v = [[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0], [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
         [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]]
    f = [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11], [1, 5, 9], [5, 11, 4], [11, 10, 2],
         [10, 7, 6], [7, 1, 8], [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9], [4, 9, 5],
         [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = f
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        faces = nf
    return np.array(verts), np.array(faces)


def _value_noise(n_pts, rng, octaves=4, base_cells=4):
    """Seeded 2D value noise on an n_pts x n_pts grid over [0,1]^2 in [0,1]."""
    x = np.linspace(0.0, 1.0, n_pts)
    total = np.zeros((n_pts, n_pts))
    amp_sum = 0.0
    for k in range(octaves):
        cells = base_cells * (2 ** k)
        lat = rng.random((cells + 1, cells + 1))
        g = x * cells
        i0 = np.minimum(np.floor(g).astype(int), cells - 1)
        fr = g - i0
        s = fr * fr * (3 - 2 * fr)  # smoothstep
        a = lat[i0[:, None], i0[None, :]]
        b = lat[i0[:, None] + 1, i0[None, :]]
        c = lat[i0[:, None], i0[None, :] + 1]
        d = lat[i0[:, None] + 1, i0[None, :] + 1]
        sx, sz = s[:, None], s[None, :]
        val = (a * (1 - sx) + b * sx) * (1 - sz) + (c * (1 - sx) + d * sx) * sz
        amp = 0.5 ** k
        total += amp * val
        amp_sum += amp
    return total / amp_sum


def heightfield(n, rng, max_height=0.25):
    """n x n-cell heightfield over [-1,1]^2 (xz), y = value noise in [0, max_height]."""
    h = _value_noise(n + 1, rng) * max_height
    g = np.linspace(-1.0, 1.0, n + 1)
    X, Z = np.meshgrid(g, g, indexing="ij")
    v = np.stack([X, h, Z], -1).reshape(-1, 3)
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    p00 = ii * (n + 1) + jj
    p10 = (ii + 1) * (n + 1) + jj
    p01 = ii * (n + 1) + jj + 1
    p11 = (ii + 1) * (n + 1) + jj + 1
    t1 = np.stack([p00, p01, p11], -1).reshape(-1, 3)
    t2 = np.stack([p00, p11, p10], -1).reshape(-1, 3)
    idx = np.stack([t1, t2], 1).reshape(-1, 3)
    return v, idx


def torus(nu, nv, R=1.0, r=0.35):
    """Torus around the y axis, nu segments around the ring, nv around the tube."""
    u = 2 * math.pi * np.arange(nu) / nu
    w = 2 * math.pi * np.arange(nv) / nv
    U, W = np.meshgrid(u, w, indexing="ij")
    v = np.stack([(R + r * np.cos(W)) * np.cos(U), r * np.sin(W), (R + r * np.cos(W)) * np.sin(U)], -1).reshape(-1, 3)
    ii, jj = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    p00 = ii * nv + jj
    p10 = ((ii + 1) % nu) * nv + jj
    p01 = ii * nv + (jj + 1) % nv
    p11 = ((ii + 1) % nu) * nv + (jj + 1) % nv
    t1 = np.stack([p00, p01, p11], -1).reshape(-1, 3)
    t2 = np.stack([p00, p11, p10], -1).reshape(-1, 3)
    idx = np.stack([t1, t2], 1).reshape(-1, 3)
    return v, idx


def _orient_outward(v, idx, centre_fn):
    """Flip the winding globally if the majority of faces point inward."""
    a, b, c = v[idx[:, 0]], v[idx[:, 1]], v[idx[:, 2]]
    n = np.cross(b - a, c - a)
    cen = (a + b + c) / 3
    s = np.einsum("ij,ij->i", n, cen - centre_fn(cen))
    if np.sum(s < 0) > np.sum(s > 0):
        idx = idx[:, [0, 2, 1]]
    return idx


def normalise(v, radius=1.0, scale=5.0):
    """Centre on the bounding-box centre, scale to bounding radius `radius`, then x`scale`."""
    v = np.asarray(v, dtype=np.float64)
    c = (v.min(0) + v.max(0)) / 2
    v = v - c
    v = v / np.max(np.linalg.norm(v, axis=1)) * radius * scale
    return v


def make_mesh(kind, *args, rng=None, scale=5.0):
    """Procedural mesh by name, centred, normalised to radius 1 and scaled x`scale`."""
    if kind == "uv":
        v, i = uv_sphere(*args)
        i = _orient_outward(v, i, lambda c: 0 * c)
    elif kind == "ico":
        v, i = icosphere(*args)
        i = _orient_outward(v, i, lambda c: 0 * c)
    elif kind == "cube":
        v, i = cube_mesh(0.5)
        v = v.astype(np.float64)
    elif kind == "hf":
        v, i = heightfield(args[0], rng)
    elif kind == "torus":
        v, i = torus(*args)

        def ring(c):
            p = c.copy()
            p[:, 1] = 0
            nrm = np.linalg.norm(p, axis=1, keepdims=True)
            return p / np.maximum(nrm, 1e-12)
        i = _orient_outward(v, i, ring)
    else:
        raise ValueError(kind)
    return _f32(normalise(v, scale=scale), i)


# --------------------------------------------------------------------------
# transforms
# --------------------------------------------------------------------------

def rot_y(deg):
    a = math.radians(deg)
    return np.array([[math.cos(a), 0, math.sin(a)], [0, 1, 0], [-math.sin(a), 0, math.cos(a)]])


def random_rotation(rng):
    """Uniform rotation on SO(3) from a Shoemake uniform unit quaternion."""
    u1, u2, u3 = rng.random(3)
    q = np.array([math.sqrt(1 - u1) * math.sin(2 * math.pi * u2), math.sqrt(1 - u1) * math.cos(2 * math.pi * u2),
                  math.sqrt(u1) * math.sin(2 * math.pi * u3), math.sqrt(u1) * math.cos(2 * math.pi * u3)])
    x, y, z, w = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def axis_angle(axis, ang):
    axis = axis / np.linalg.norm(axis)
    x, y, z = axis
    c, s = math.cos(ang), math.sin(ang)
    C = 1 - c
    return np.array([[c + x * x * C, x * y * C - z * s, x * z * C + y * s],
                     [y * x * C + z * s, c + y * y * C, y * z * C - x * s],
                     [z * x * C - y * s, z * y * C + x * s, c + z * z * C]])


def affine(R, t, s=1.0):
    """Row-major 3x4 object-to-world matrix [s*R | t] as float32."""
    M = np.zeros((3, 4))
    M[:, :3] = np.asarray(R) * s
    M[:, 3] = t
    return M.astype(np.float32)


# --------------------------------------------------------------------------
# scene container
# --------------------------------------------------------------------------

@dataclass
class Scene:
    meshes: list                      # [(vtx float32 (nv,3), idx uint32 (nt,3))]
    M: np.ndarray                     # float32 (n,3,4) object->world, row-major
    mesh_id: np.ndarray               # uint32 (n,)
    material_id: np.ndarray           # uint32 (n,)
    mat_type: np.ndarray              # uint32 (m,)
    mat_albedo: np.ndarray            # float32 (m,3)
    mat_ior: np.ndarray               # float32 (m,)
    light_pos: np.ndarray             # float32 (L,3)
    light_I: np.ndarray               # float32 (L,3)
    background: tuple = (0.2, 0.3, 0.5)
    ambient: float = 0.1
    camera: dict = field(default_factory=dict)   # eye, target, up, vfov
    width: int = 64
    height: int = 64
    max_depth: int = 1
    name: str = ""

    @property
    def n_instances(self):
        return int(self.M.shape[0])

    def instanced_tris(self):
        return int(sum(self.meshes[m][1].shape[0] for m in self.mesh_id))

    def world_aabb(self):
        """Bounding box of all transformed mesh vertices (float64; for ray origins only)."""
        lo = np.full(3, np.inf)
        hi = np.full(3, -np.inf)
        for k in range(self.n_instances):
            v = self.meshes[self.mesh_id[k]][0].astype(np.float64)
            bl, bh = v.min(0), v.max(0)
            corners = np.array([[x, y, z] for x in (bl[0], bh[0]) for y in (bl[1], bh[1]) for z in (bl[2], bh[2])])
            w = corners @ self.M[k, :, :3].astype(np.float64).T + self.M[k, :, 3]
            lo = np.minimum(lo, w.min(0))
            hi = np.maximum(hi, w.max(0))
        return lo, hi


def _materials(types, albedo, ior):
    return (np.asarray(types, dtype=np.uint32), np.asarray(albedo, dtype=np.float32).reshape(-1, 3),
            np.asarray(ior, dtype=np.float32))


def tiny_scene():
    """One unit cube (12 tris) on a 10x10 ground quad, 3 instances, 64x64."""
    cube = cube_mesh(0.5)
    ground = quad_mesh(10.0, -0.5)
    M = np.stack([affine(np.eye(3), [0, 0, 0]), affine(np.eye(3), [0, 0, 0]), affine(rot_y(30.0), [2, 0, -1])])
    mt, ma, mi = _materials([MAT_DIFFUSE], [[0.8, 0.8, 0.8]], [1.0])
    return Scene(meshes=[cube, ground], M=M, mesh_id=np.array([1, 0, 0], np.uint32),
                 material_id=np.zeros(3, np.uint32), mat_type=mt, mat_albedo=ma, mat_ior=mi,
                 light_pos=np.array([[2, 4, 3]], np.float32), light_I=np.array([[1, 1, 1]], np.float32),
                 camera=dict(eye=(0, 2, 5), target=(0, 0, 0), up=(0, 1, 0), vfov=60.0),
                 width=64, height=64, max_depth=1, name="tiny")


def _random_instances(rng, n, n_meshes, box, counts=None):
    if counts is None:
        mesh_id = rng.integers(0, n_meshes, size=n).astype(np.uint32)
    else:
        mesh_id = np.repeat(np.arange(n_meshes), counts).astype(np.uint32)
        rng.shuffle(mesh_id)
    M = np.empty((n, 3, 4), np.float32)
    for k in range(n):
        s = rng.uniform(0.5, 2.0)
        R = random_rotation(rng)
        t = rng.uniform(-box, box, size=3)
        M[k] = affine(R, t, s)
    return M, mesh_id


def _random_materials(rng, n, p_diffuse=0.6, p_mirror=0.2):
    types = np.empty(n, np.uint32)
    albedo = np.empty((n, 3), np.float32)
    ior = np.ones(n, np.float32)
    for k in range(n):
        r = rng.random()
        if r < p_diffuse:
            types[k] = MAT_DIFFUSE
            albedo[k] = rng.uniform(0.2, 0.9, size=3)
        elif r < p_diffuse + p_mirror:
            types[k] = MAT_MIRROR
            albedo[k] = 0.9
        else:
            types[k] = MAT_GLASS
            albedo[k] = 1.0
            ior[k] = 1.5
    return types, albedo, ior


MEDIUM_MESH_SCALE = 10.0


def medium_meshes(rng):
    s = MEDIUM_MESH_SCALE
    return [make_mesh("uv", 80, 40, scale=s), make_mesh("ico", 5, scale=s), make_mesh("cube", scale=s),
            make_mesh("hf", 256, rng=rng, scale=s)]


def medium_scene(seed=SEED_SCENE, width=1920, height=1080, max_depth=4):
    """64 instances of 4 procedural meshes in a 100^3 box, 4 lights, 1920x1080."""
    rng = np.random.default_rng(seed)
    meshes = medium_meshes(rng)
    M, mesh_id = _random_instances(rng, 64, len(meshes), 50.0)
    mt, ma, mi = _random_materials(rng, 64)
    lp = np.array([[rng.uniform(-50, 50), rng.uniform(40, 60), rng.uniform(-50, 50)] for _ in range(4)], np.float32)
    return Scene(meshes=meshes, M=M, mesh_id=mesh_id, material_id=np.arange(64, dtype=np.uint32),
                 mat_type=mt, mat_albedo=ma, mat_ior=mi, light_pos=lp,
                 light_I=np.full((4, 3), 0.25, np.float32),
                 camera=dict(eye=(0, 0, 100), target=(0, 0, 0), up=(0, 1, 0), vfov=60.0),
                 width=width, height=height, max_depth=max_depth, name="medium")


LARGE_MESHES = [("uv", 64, 32), ("uv", 160, 80), ("uv", 320, 160), ("uv", 640, 320),
                ("ico", 3), ("ico", 4), ("ico", 5), ("ico", 7),
                ("hf", 64), ("hf", 128), ("hf", 256), ("hf", 512),
                ("torus", 48, 24), ("torus", 128, 64), ("torus", 256, 128), ("torus", 512, 256)]


def large_counts(tris, total=4096, power=-0.77):
    """Per-mesh instance counts proportional to tris^power, largest-remainder rounded."""
    w = np.asarray(tris, dtype=np.float64) ** power
    q = w / w.sum() * total
    c = np.floor(q).astype(int)
    rem = total - c.sum()
    order = np.argsort(-(q - c), kind="stable")
    c[order[:rem]] += 1
    return c


def large_scene(seed=SEED_SCENE, mesh_scale=1.0):
    """4096 instances of 16 procedural meshes (1,938,944 unique tris) in a 400^3 box."""
    rng = np.random.default_rng(seed)
    meshes = []
    for spec in LARGE_MESHES:
        kind, args = spec[0], spec[1:]
        meshes.append(make_mesh(kind, *args, rng=rng) if kind == "hf" else make_mesh(kind, *args))
    counts = large_counts([m[1].shape[0] for m in meshes])
    M, mesh_id = _random_instances(rng, 4096, len(meshes), 200.0, counts=counts)
    mt, ma, mi = _random_materials(rng, 4096)
    return Scene(meshes=meshes, M=M, mesh_id=mesh_id, material_id=np.arange(4096, dtype=np.uint32),
                 mat_type=mt, mat_albedo=ma, mat_ior=mi,
                 light_pos=np.zeros((0, 3), np.float32), light_I=np.zeros((0, 3), np.float32),
                 camera=dict(eye=(0, 0, 400), target=(0, 0, 0), up=(0, 1, 0), vfov=60.0),
                 width=0, height=0, max_depth=1, name="large")


def motion(M, frame, seed=SEED_MOTION):
    """Seeded per-instance motion for one frame: T += N(0,1)^3, rotate by N(0,2 deg) about a random axis."""
    rng = np.random.default_rng([seed, frame])
    out = np.empty_like(M)
    for k in range(M.shape[0]):
        A = M[k, :, :3].astype(np.float64)
        t = M[k, :, 3].astype(np.float64) + rng.normal(0.0, 1.0, 3)
        axis = rng.normal(size=3)
        ang = math.radians(rng.normal(0.0, 2.0))
        out[k, :, :3] = axis_angle(axis, ang) @ A
        out[k, :, 3] = t
    return out.astype(np.float32)


# --------------------------------------------------------------------------
# rays (rg_ray layout: o.xyz, tmin, d.xyz, tmax; float32)
# --------------------------------------------------------------------------

def random_rays(n, lo, hi, seed=SEED_RAYS, tmax_range=None):
    """n rays, origins uniform in [lo,hi], directions uniform on the sphere."""
    rng = np.random.default_rng(seed)
    r = np.empty((n, 8), np.float32)
    r[:, 0:3] = rng.uniform(lo, hi, size=(n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r[:, 4:7] = d
    r[:, 3] = 0.0
    if tmax_range is None:
        r[:, 7] = np.inf
    else:
        r[:, 7] = rng.uniform(tmax_range[0], tmax_range[1], size=n)
    return r


def rays_toward(origins, targets, tmin=0.0, tmax=np.inf):
    """Rays from each origin through each target point (unnormalised direction target-origin)."""
    o = np.asarray(origins, np.float32)
    d = (np.asarray(targets, np.float64) - o.astype(np.float64)).astype(np.float32)
    r = np.empty((o.shape[0], 8), np.float32)
    r[:, 0:3] = o
    r[:, 3] = tmin
    r[:, 4:7] = d
    r[:, 7] = tmax
    return r


def large_rays(scene, n, seed=SEED_RAYS):
    """Closest-hit and any-hit ray sets of the large workload (origins in the scene AABB)."""
    lo, hi = scene.world_aabb()
    closest = random_rays(n, lo, hi, seed=seed)
    anyhit = random_rays(n, lo, hi, seed=seed + 1, tmax_range=(1.0, 50.0))
    return closest, anyhit


# --------------------------------------------------------------------------
# serving stream
# --------------------------------------------------------------------------

SERVE_RESOLUTIONS = [(320, 240), (640, 480), (1280, 720), (1920, 1080), (3840, 2160)]


def serving_scenes():
    """The 8 resident scenes of the serving workload: the tiny scene and seven
    medium-style scenes (seeds 11..17), each with its own meshes, layout,
    materials and lights."""
    return [tiny_scene()] + [medium_scene(seed=10 + k) for k in range(1, 8)]


def serving_requests(n, rate=200.0, n_scenes=8, seed=SEED_SERVE):
    """Poisson arrival stream: (arrival_s, scene, width, height, max_depth, motion_seed)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n)
    t = np.cumsum(gaps)
    out = []
    for k in range(n):
        w, h = SERVE_RESOLUTIONS[rng.integers(0, len(SERVE_RESOLUTIONS))]
        out.append(dict(arrival=float(t[k]), scene=int(rng.integers(0, n_scenes)), width=w, height=h,
                        max_depth=int(rng.integers(1, 9)), motion_seed=int(rng.integers(0, 2**31))))
    return out
