"""Pins of the oracle's ambiguity classification, the rule that exempts a ray
from exact parity when the float32 path may legitimately answer otherwise
(a shared edge, a near tie in t, a grazing hit, a segment ending at a
surface).  A classifier that flagged nothing would make the GPU tests
stricter than float32 allows; one that flagged everything would make them
vacuous: each case below fails one of the two."""
import numpy as np

import oracle

f32 = np.float32


def quads(zs):
    """Unit quads (two triangles sharing the diagonal (-1,-1)-(1,1)) at the
    given heights, one identity instance."""
    O = oracle.OracleScene()
    v, idx = [], []
    for k, z in enumerate(zs):
        b = 4 * k
        v += [(-1, -1, z), (1, -1, z), (1, 1, z), (-1, 1, z)]
        idx += [(b, b + 1, b + 2), (b, b + 2, b + 3)]
    O.add_mesh(np.array(v, f32), np.array(idx, np.uint32))
    O.set_instances(np.array([[1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0]], f32), np.array([0], np.uint32))
    return O


def down(pts, tmax=np.inf, z=5.0):
    """Rays from height z straight down through the points (x, y)."""
    r = np.zeros((len(pts), 8), f32)
    for i, (x, y) in enumerate(pts):
        r[i] = [x, y, z, 0, 0, 0, -1, tmax]
    return r


MISS = 0xFFFFFFFF


def test_interior_hits_and_clear_misses_are_not_ambiguous():
    out = quads([0.0]).trace(down([(0.5, -0.5), (-0.5, 0.5), (0.999, 0.0), (1.01, 0.2), (3.0, 3.0)]))
    assert list(out["prim"][:3]) == [0, 1, 0] and (out["t"][:3] == 5.0).all()
    assert (out["inst"][3:] == MISS).all()
    assert not out["ambiguous"].any()


def test_shared_edge_is_ambiguous():
    # on the diagonal both triangles hit at the same t: the float32 path may
    # return either
    out = quads([0.0]).trace(down([(0.3, 0.3), (-0.7, -0.7)]))
    assert (out["inst"] == 0).all() and (out["t"] == 5.0).all()
    assert out["ambiguous"].all()


def test_outer_edge_within_the_error_band_is_ambiguous():
    # 1e-7 outside the quad: an exact miss that float32 may turn into a hit
    out = quads([0.0]).trace(down([(1 + 1e-7, 0.2), (0.2, -1 - 1e-7)]))
    assert (out["inst"] == MISS).all()
    assert out["ambiguous"].all()


def test_near_tie_in_t_is_ambiguous_and_a_clear_gap_is_not():
    near = quads([0.0, -1e-6]).trace(down([(0.5, -0.5)]))
    assert near["ambiguous"][0]
    apart = quads([0.0, -1.0]).trace(down([(0.5, -0.5)]))
    assert not apart["ambiguous"][0] and apart["t"][0] == 5.0


def test_grazing_hit_is_ambiguous():
    # cos(ray, normal) = 0.001 < 1/256: the hit point moves along the plane
    # by far more than the float32 error
    r = np.array([[-5, -0.5, 0.005, 0, 1, 0, -0.001, np.inf]], f32)
    out = quads([0.0]).trace(r)
    assert out["inst"][0] == 0 and abs(out["t"][0] - 5.0) < 1e-3
    assert out["ambiguous"][0]


def test_any_hit_segment_ending_at_the_surface_is_ambiguous():
    O = quads([0.0])
    for tmax, occluded, amb in [(4.9, False, False), (5.0, True, True), (5.0 * (1 + 1e-6), True, True),
                                (6.0, True, False)]:
        out = O.trace(down([(0.5, -0.5)], tmax=tmax), any_hit=True)
        assert out["occluded"][0] == occluded and out["ambiguous"][0] == amb, tmax


def test_error_band_width_at_an_outer_edge():
    """The band's width is the stated float32 error bound: for these rays
    (identity instance, origin height 5, unit direction, vertices of
    magnitude 1, hit distance 5) eta = 16 * 2^-24 * (5 + 5 * 1 + 1).  A ray
    passing 0.95 eta outside the quad's edge is flagged, one passing 1.05 eta
    outside is a clear miss."""
    eta = 16 * 2.0 ** -24 * (5 + 5 + 1)
    out = quads([0.0]).trace(down([(1 + 0.95 * eta, 0.2), (1 + 1.05 * eta, 0.2),
                                   (0.2, -1 - 0.95 * eta), (0.2, -1 - 1.05 * eta)]))
    assert (out["inst"] == MISS).all()
    assert list(out["ambiguous"]) == [True, False, True, False]
