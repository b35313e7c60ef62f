"""The seeded synthetic inputs match the recipe they stand for: mesh and
triangle counts, instance layout, materials, lights, camera and image size of
the tiny, medium and large configurations, the per-frame motion law and the
serving stream's arrival process; and each generator is deterministic."""
import numpy as np
import pytest

import scenegen as g


def _area2(v, idx):
    a, b, c = (v[idx[:, k]].astype(np.float64) for k in range(3))
    return np.linalg.norm(np.cross(b - a, c - a), axis=1)


def _scale_and_rotation(M):
    """Per instance: the uniform scale s and the residual of R^T R = I for
    M[:, :3] = s R."""
    A = M[:, :, :3].astype(np.float64)
    s = np.linalg.norm(A, axis=2).mean(axis=1)
    R = A / s[:, None, None]
    err = np.abs(np.einsum("nij,nik->njk", R, R) - np.eye(3)).max(axis=(1, 2))
    return s, err


def test_tiny_configuration():
    s = g.tiny_scene()
    assert (s.width, s.height, s.max_depth) == (64, 64, 1)
    assert s.n_instances == 3 and s.instanced_tris() == 26   # ground quad + two cubes
    assert len(s.light_pos) == 1


def test_medium_configuration():
    s = g.medium_scene()
    assert (s.width, s.height, s.max_depth) == (1920, 1080, 4)
    assert [m[1].shape[0] for m in s.meshes] == [6400, 20480, 12, 131072]
    assert sum(m[1].shape[0] for m in s.meshes) == 157_964
    assert s.n_instances == 64 and set(np.unique(s.mesh_id)) <= {0, 1, 2, 3}
    sc, err = _scale_and_rotation(s.M)
    assert ((sc > 0.5 - 1e-5) & (sc < 2.0 + 1e-5)).all() and err.max() < 1e-5
    assert (np.abs(s.M[:, :, 3]) <= 50.0).all()
    # materials: diffuse / mirror / glass near 60 / 20 / 20 %, glass IOR 1.5, mirror tint 0.9
    counts = np.bincount(s.mat_type, minlength=3)
    assert counts.sum() == 64 and counts[0] >= 28 and counts[1] >= 4 and counts[2] >= 4
    assert (s.mat_ior[s.mat_type == g.MAT_GLASS] == np.float32(1.5)).all()
    assert (s.mat_albedo[s.mat_type == g.MAT_MIRROR] == np.float32(0.9)).all()
    d = s.mat_albedo[s.mat_type == g.MAT_DIFFUSE]
    assert ((d >= 0.2) & (d <= 0.9)).all()
    # four lights above the scene at 0.25 each
    assert s.light_pos.shape == (4, 3) and (s.light_I == np.float32(0.25)).all()
    assert ((s.light_pos[:, 1] >= 40) & (s.light_pos[:, 1] <= 60)).all()
    assert (np.abs(s.light_pos[:, [0, 2]]) <= 50).all()
    assert tuple(s.camera["eye"]) == (0, 0, 100) and s.camera["vfov"] == 60.0
    # the UV sphere's pole rows hold exactly degenerate triangles (never hit)
    v, idx = s.meshes[0]
    assert (_area2(v, idx) == 0).sum() > 0


def test_generators_are_deterministic():
    a, b = g.medium_scene(), g.medium_scene()
    assert all(np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1]) for x, y in zip(a.meshes, b.meshes))
    for f in ["M", "mesh_id", "mat_type", "mat_albedo", "light_pos"]:
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    assert not np.array_equal(g.medium_scene(seed=11).M, a.M)
    assert np.array_equal(g.motion(a.M, 3), g.motion(b.M, 3))
    assert np.array_equal(g.random_rays(100, -1, 1), g.random_rays(100, -1, 1))


def test_motion_law():
    s = g.medium_scene()
    frames = [g.motion(s.M, k) for k in range(40)]
    dt = np.concatenate([f[:, :, 3] - s.M[:, :, 3] for f in frames]).astype(np.float64).ravel()
    # translation steps N(0, 1) per axis (7,680 samples)
    assert abs(dt.mean()) < 0.05 and abs(dt.std() - 1.0) < 0.05
    # rotation about a random axis by N(0, 2 deg): the linear part keeps its
    # scale and stays a scaled rotation
    for f in frames[:5]:
        sc0, _ = _scale_and_rotation(s.M)
        sc1, err = _scale_and_rotation(f)
        assert np.allclose(sc0, sc1, rtol=1e-5) and err.max() < 1e-5
    ang = []
    for f in frames:
        A0 = s.M[:, :, :3].astype(np.float64)
        A1 = f[:, :, :3].astype(np.float64)
        Q = np.einsum("nij,njk->nik", A1, np.linalg.inv(A0))
        ang.append(np.degrees(np.arccos(np.clip((np.trace(Q, axis1=1, axis2=2) - 1) / 2, -1, 1))))
    ang = np.concatenate(ang)
    # |N(0, 2)| has mean 2 sqrt(2/pi) = 1.596 degrees
    assert abs(ang.mean() - 1.596) < 0.1


@pytest.mark.slow
def test_large_configuration():
    s = g.large_scene()
    assert len(s.meshes) == 16
    assert sum(m[1].shape[0] for m in s.meshes) == 1_938_944
    assert s.n_instances == 4096 and len(s.light_pos) == 0
    counts = np.bincount(s.mesh_id, minlength=16)
    assert np.array_equal(counts, g.large_counts([m[1].shape[0] for m in s.meshes]))
    assert (np.abs(s.M[:, :, 3]) <= 200.0).all()


def test_serving_stream():
    reqs = g.serving_requests(4000)
    t = np.array([r["arrival"] for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    # Poisson arrivals at 200 requests per second: exponential gaps, mean 5 ms
    assert (gaps > 0).all() and abs(gaps.mean() - 0.005) < 0.00025 and abs(gaps.std() / gaps.mean() - 1) < 0.05
    assert {(r["width"], r["height"]) for r in reqs} == set(g.SERVE_RESOLUTIONS)
    assert {r["max_depth"] for r in reqs} == set(range(1, 9))
    assert {r["scene"] for r in reqs} == set(range(8))
    assert len(g.serving_scenes()) == 8
