"""Readings of the watertight triangle test pinned on the CPU in float32
(numpy rounds every operation to nearest, no FMA, as the CUDA code spells
out with intrinsics).

Woop, Benthin & Wald (JCGT 2013) permute the axes so that kz is the ray's
dominant axis and swap kx and ky when d_kz < 0 to keep the winding (for
back-face culling).  Without culling the swap negates the edge functions U, V,
W, their sum det and the scaled distance T together, so t = T/det and the
barycentrics V/det, W/det come out bit for bit the same: the traversal uses
the cyclic order (kz+1, kz+2, kz) and reads triangles stored in that order.
"""
import numpy as np

f32 = np.float32


def wbw(o, d, v0, v1, v2, swap):
    """Vectorised float32 watertight test (rows = cases): U, V, W, det, T."""
    n = o.shape[0]
    r = np.arange(n)
    kz = np.argmax(np.abs(d), axis=1)
    kx = (kz + 1) % 3
    ky = (kx + 1) % 3
    if swap:
        neg = d[r, kz] < 0
        kx, ky = np.where(neg, ky, kx), np.where(neg, kx, ky)
    Sz = f32(1) / d[r, kz]
    Sx = d[r, kx] * Sz
    Sy = d[r, ky] * Sz
    az, bz, cz = v0[r, kz] - o[r, kz], v1[r, kz] - o[r, kz], v2[r, kz] - o[r, kz]
    Ax = (v0[r, kx] - o[r, kx]) - Sx * az
    Ay = (v0[r, ky] - o[r, ky]) - Sy * az
    Bx = (v1[r, kx] - o[r, kx]) - Sx * bz
    By = (v1[r, ky] - o[r, ky]) - Sy * bz
    Cx = (v2[r, kx] - o[r, kx]) - Sx * cz
    Cy = (v2[r, ky] - o[r, ky]) - Sy * cz
    U = Cx * By - Cy * Bx
    V = Ax * Cy - Ay * Cx
    W = Bx * Ay - By * Ax
    det = (U + V) + W
    T = (U * (Sz * az) + V * (Sz * bz)) + W * (Sz * cz)
    return U, V, W, det, T


def cases(n, seed):
    rng = np.random.default_rng(seed)
    o = rng.uniform(-5, 5, (n, 3)).astype(f32)
    d = rng.normal(size=(n, 3)).astype(f32)
    # a share of rays with a negative dominant component and of tiny components
    d[: n // 4, 2] = -np.abs(d[: n // 4, 2]) - f32(2)
    d[n // 4: n // 2, 0] *= f32(1e-6)
    c = rng.uniform(-3, 3, (n, 3)).astype(f32)
    v0 = (c + rng.normal(size=(n, 3))).astype(f32)
    v1 = (c + rng.normal(size=(n, 3))).astype(f32)
    v2 = (c + rng.normal(size=(n, 3))).astype(f32)
    return o, d, v0, v1, v2


def bits(x):
    return np.asarray(x, f32).view(np.uint32)


def test_swap_negates_the_edge_functions_exactly():
    with np.errstate(all="ignore"):
        o, d, v0, v1, v2 = cases(200_000, 1)
        a = wbw(o, d, v0, v1, v2, swap=True)
        b = wbw(o, d, v0, v1, v2, swap=False)
        neg = d[np.arange(len(d)), np.argmax(np.abs(d), axis=1)] < 0
        assert neg.sum() > 50_000
        for x, y in zip(a, b):
            # where the swap applies, exactly opposite; elsewhere identical
            np.testing.assert_array_equal(bits(np.where(neg, -x, x)), bits(y))


def test_t_and_barycentrics_do_not_depend_on_the_swap():
    with np.errstate(all="ignore"):
        o, d, v0, v1, v2 = cases(200_000, 2)
        U1, V1, W1, det1, T1 = wbw(o, d, v0, v1, v2, swap=True)
        U2, V2, W2, det2, T2 = wbw(o, d, v0, v1, v2, swap=False)
        ok = det1 != 0
        assert ok.sum() > 190_000
        for num1, num2 in [(T1, T2), (V1, V2), (W1, W2)]:
            np.testing.assert_array_equal(bits((num1 / det1)[ok]), bits((num2 / det2)[ok]))
        # the inside test (all of U, V, W of one sign, zero counting as either)
        inside1 = ~(((U1 < 0) | (V1 < 0) | (W1 < 0)) & ((U1 > 0) | (V1 > 0) | (W1 > 0)))
        inside2 = ~(((U2 < 0) | (V2 < 0) | (W2 < 0)) & ((U2 > 0) | (V2 > 0) | (W2 > 0)))
        np.testing.assert_array_equal(inside1, inside2)
        assert inside1.sum() > 1000
