"""Readings of the watertight triangle test pinned on the CPU in float32
(numpy rounds every operation to nearest, no FMA, as the CUDA code spells
out with intrinsics).

Woop, Benthin & Wald (JCGT 2013) permute the axes so that kz is the ray's
dominant axis and swap kx and ky when d_kz < 0 to keep the winding (for
back-face culling).  Without culling the swap negates the edge functions U, V,
W, their sum det and the scaled distance T together, so t = T/det and the
barycentrics V/det, W/det come out bit for bit the same: the traversal uses
the cyclic order (kz+1, kz+2, kz) and reads triangles stored in that order.

The box tests are pinned the same way: the binary BVH's slab test and the
compressed 8-wide node's dequantising FMA test with its widening never reject
a box that the ray's segment meets (float64), and reject boxes it misses by a
clear margin; the outward quantisation of child boxes contains each box.
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


# ---------------------------------------------------------------- box test

K_IZE = f32(1.0) + f32(2.0) * (f32(3.0) * f32(2.0 ** -24)) / (f32(1.0) - f32(3.0) * f32(2.0 ** -24))
CULL = f32(1.0) + f32(1.0 / 4096.0)


def slab32(lo, hi, o, d, tmin, tlim):
    """The float32 box test as the traversal runs it: t = (plane - o) * (1/d)
    per axis, NaN-propagating min / max per axis, NaN-dropping max / min
    across axes, far distance scaled by 1 + 2 gamma_3, then clipped to tlim."""
    with np.errstate(all="ignore"):
        ix = f32(1) / d
        t0 = (lo - o) * ix
        t1 = (hi - o) * ix
        nmin = np.minimum(t0, t1)   # NaN if either is NaN
        nmax = np.maximum(t0, t1)
        tn = np.fmax(np.fmax(nmin[:, 0], nmin[:, 1]), np.fmax(nmin[:, 2], tmin))
        tf = np.fmin(np.fmin(nmax[:, 0], nmax[:, 1]), nmax[:, 2])
        tf = np.fmin(tf * K_IZE, tlim)
        return tn <= tf


def exact_hit(lo, hi, o, d, tmin, tmax):
    """Whether the segment [tmin, tmax] of the ray meets the closed box, in
    float64 (the float32 inputs are exact in it)."""
    lo, hi, o, d = (np.asarray(x, np.float64) for x in (lo, hi, o, d))
    tn = np.full(len(o), float(tmin))
    tf = np.full(len(o), float(tmax))
    with np.errstate(all="ignore"):
        for a in range(3):
            z = d[:, a] == 0
            ta, tb = (lo[:, a] - o[:, a]) / d[:, a], (hi[:, a] - o[:, a]) / d[:, a]
            tn = np.where(z, tn, np.maximum(tn, np.minimum(ta, tb)))
            tf = np.where(z, tf, np.minimum(tf, np.maximum(ta, tb)))
            inside = (lo[:, a] <= o[:, a]) & (o[:, a] <= hi[:, a])
            tf = np.where(z & ~inside, -np.inf, tf)
    return tn <= tf


def box_cases(n, seed):
    rng = np.random.default_rng(seed)
    c = rng.uniform(-20, 20, (n, 3))
    ext = rng.uniform(0, 3, (n, 3)) * (rng.random((n, 3)) > 0.1)   # some flat boxes
    lo, hi = (c - ext).astype(f32), (c + ext).astype(f32)
    o = rng.uniform(-30, 30, (n, 3)).astype(f32)
    # aim most rays at a point of the box's closure (corners, edges, faces included)
    target = lo + (hi - lo) * rng.choice([0.0, 0.5, 1.0, rng.random()], (n, 3)).astype(f32)
    d = (target - o).astype(f32)
    m = rng.random(n) < 0.2
    d[m] = rng.normal(size=(m.sum(), 3)).astype(f32)
    # axis-aligned rays, some with the origin on a slab plane (0 * inf = NaN)
    k = rng.random(n) < 0.2
    ax = rng.integers(0, 3, n)
    for a in range(3):
        sel = k & (ax == a)
        keep = d[sel, a].copy()
        d[sel] = 0
        d[sel, a] = np.where(keep == 0, 1, keep)
        on = sel & (rng.random(n) < 0.5)
        o[on, (a + 1) % 3] = rng.choice([0, 1], on.sum()).astype(f32) * (hi[on, (a + 1) % 3] - lo[on, (a + 1) % 3]) + lo[on, (a + 1) % 3]
    return lo, hi, o, d


def test_box_test_never_rejects_a_box_the_segment_meets():
    lo, hi, o, d = box_cases(400_000, 3)
    for tmax in [np.inf, 5.0, 40.0]:
        tlim = f32(tmax) * CULL if np.isfinite(tmax) else f32(np.inf)
        got = slab32(lo, hi, o, d, f32(0), tlim)
        want = exact_hit(lo, hi, o, d, 0.0, tmax)
        missed = want & ~got
        assert not missed.any(), f"tmax {tmax}: {missed.sum()} boxes rejected, e.g. case {np.nonzero(missed)[0][:3]}"
        assert want.sum() > 100_000
        # conservative, not permissive: a box the segment misses by more than
        # a relative 1e-4 (its copy grown by that much is still missed) is
        # rejected
        grow = (1e-4 * (1.0 + np.maximum(np.abs(lo).max(1), np.abs(o).max(1))))[:, None]
        far = ~exact_hit(lo - grow, hi + grow, o, d, 0.0, tmax)
        assert far.sum() > 50_000
        assert not (got & far).any()


def test_zero_direction_origin_on_plane_leaves_the_axis_open():
    # ray along +z, origin exactly on the box's x = lo plane: 0 * inf = NaN on x
    lo = np.array([[0, -1, 5]], f32)
    hi = np.array([[2, 1, 6]], f32)
    d = np.array([[0, 0, 1]], f32)
    for ox, want in [(0.0, True), (2.0, True), (1.0, True), (-1e-7, False), (2.0000002, False)]:
        o = np.array([[ox, 0, 0]], f32)
        assert slab32(lo, hi, o, d, f32(0), f32(np.inf))[0] == want, ox


# ---------------------------------------------------------------- compressed 8-wide node test
#
# A wide node stores its children's boxes as 8-bit integers against a float32
# origin p and a per-axis power of two 2^e, rounded outward:
#   qlo = floor(rd(lo - p) / 2^e),  qhi = ceil(ru(hi - p) / 2^e),
# with e the smallest exponent such that 255 * 2^e >= ru(max hi - p).  The
# traversal tests a child with one FMA per plane on the byte's float 1 + q 2^-15
# (a byte permute puts q in the mantissa under the exponent of 1; exact):
#   t = (1 + q 2^-15) * 2^15 S + (B - 2^15 S),  S = 2^e / d,  B = (p - o) / d,
# and widens the child intervals of each axis by
#   E = 8 * 2^-24 * (255 |S| + |B|) + 2^-7 |S|
# (the last term covers the roundings of B - 2^15 S and of the shifted
# planes, each at most 2^-9 |S| beyond those of B itself).  A plane offset
# B - 2^15 S that overflows is replaced by NaN, which leaves the axis open.

QERR = f32(8.0 * 2.0 ** -24)
PLANE_ERR = f32(2.0 ** -7)


def round_dir(x, up):
    """float64 -> float32, rounded down (up=False) or up."""
    r = x.astype(f32)
    if up:
        return np.where(r.astype(np.float64) < x, np.nextafter(r, f32(np.inf)), r)
    return np.where(r.astype(np.float64) > x, np.nextafter(r, f32(-np.inf)), r)


def exact_diff(a, b):
    """a - b of float32 arrays in float64, with a mask of the cases where that
    difference is exact (TwoSum error zero)."""
    a, b = a.astype(np.float64), b.astype(np.float64)
    s = a - b
    bb = s - a
    err = (a - (s - bb)) + (-b - bb)
    return s, err == 0


def exp_for(ext):
    """Smallest e in [-126, 127] with 255 * 2^e >= ext (ext >= 0)."""
    with np.errstate(divide="ignore"):
        e = np.where(ext > 0, np.ceil(np.log2(np.where(ext > 0, ext, 1.0) / 255.0)), -126).astype(np.int64)
    e = np.clip(e, -126, 127)
    for _ in range(3):
        e = np.where((e > -126) & (np.ldexp(255.0, e - 1) >= ext), e - 1, e)
        e = np.where((e < 127) & (np.ldexp(255.0, e) < ext), e + 1, e)
    return e


def quantize(lo, hi, p, e):
    """The builder's outward rounding of float32 child boxes against p, 2^e."""
    dlo, ok_lo = exact_diff(lo, p)
    dhi, ok_hi = exact_diff(hi, p)
    qlo = np.floor(round_dir(dlo, False).astype(np.float64) * np.ldexp(1.0, -e))
    qhi = np.ceil(round_dir(dhi, True).astype(np.float64) * np.ldexp(1.0, -e))
    return np.clip(qlo, 0, 255), np.clip(qhi, 0, 255), ok_lo & ok_hi


def fma32(a, b, c):
    """float32 fused multiply-add: the product of two float32 values is exact
    in float64, then the sum is rounded (to float64, then float32; where the
    exact sum needs more than 53 bits the double rounding can differ by an
    ulp, far inside the widening)."""
    with np.errstate(all="ignore"):
        return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(f32)


def wide_child_test(p, e, qlo, qhi, o, d, tmin, tlim):
    """The traversal's test of one child of a compressed node, in float32."""
    with np.errstate(all="ignore"):
        ix = f32(1) / d
        S = np.ldexp(f32(1), e).astype(f32) * ix          # exact: a power of two times 1/d
        B = (p - o) * ix
        U = S * f32(2.0 ** 15)                             # exact (or inf)
        E = fma32(QERR, fma32(f32(255), np.abs(S), np.abs(B)), PLANE_ERR * np.abs(S))
        C = fma32(f32(-(2.0 ** 15)), S, B)
        C = np.where(np.isinf(C), f32(np.nan), C)
        Cn, Cf = C - E, C + E
        neg = np.signbit(ix)
        vn = (1.0 + np.where(neg, qhi, qlo) * 2.0 ** -15).astype(f32)   # exact
        vf = (1.0 + np.where(neg, qlo, qhi) * 2.0 ** -15).astype(f32)
        tnear, tfar = fma32(vn, U, Cn), fma32(vf, U, Cf)
        tn = np.fmax(np.fmax(tnear[:, 0], tnear[:, 1]), np.fmax(tnear[:, 2], tmin))
        tf = np.fmin(np.fmin(tfar[:, 0], tfar[:, 1]), np.fmin(tfar[:, 2], tlim))
    return tn <= tf


def wide_cases(n, seed):
    """Child boxes of random wide nodes at three scales (some flat, some
    spanning the node), and rays aimed at points of their closure, random or
    axis-aligned."""
    rng = np.random.default_rng(seed)
    scale = rng.choice([1e-3, 1.0, 1e3], n)[:, None]
    p = (rng.uniform(-20, 20, (n, 3)) * scale).astype(f32)
    ext = rng.uniform(0, 10, (n, 3)) * scale * (rng.random((n, 3)) > 0.05)
    c0 = rng.random((n, 3)) * ext
    c1 = c0 + rng.random((n, 3)) * (ext - c0) * (rng.random((n, 3)) > 0.1)
    lo = round_dir(p + c0, True)
    hi = np.maximum(round_dir(p + c1, False), lo)
    mx = np.maximum(round_dir(p + ext, False), hi)
    dmx, ok = exact_diff(mx, p)
    e = exp_for(round_dir(dmx, True).astype(np.float64))
    qlo, qhi, okq = quantize(lo, hi, p, e)
    o = (rng.uniform(-30, 30, (n, 3)) * scale).astype(f32)
    blo = p.astype(np.float64) + qlo * np.ldexp(1.0, e)
    bhi = p.astype(np.float64) + qhi * np.ldexp(1.0, e)
    target = blo + (bhi - blo) * rng.choice([0.0, 0.5, 1.0, rng.random()], (n, 3))
    d = (target - o).astype(f32)
    m = rng.random(n) < 0.2
    d[m] = rng.normal(size=(m.sum(), 3)).astype(f32)
    k = rng.random(n) < 0.1
    ax = rng.integers(0, 3, n)
    for a in range(3):
        sel = k & (ax == a)
        keep = d[sel, a].copy()
        d[sel] = 0
        d[sel, a] = np.where(keep == 0, 1, keep)
    keep = (ok & okq).all(axis=1)
    return [x[keep] for x in (lo, hi, p, e, qlo, qhi, blo, bhi, o, d)]


def test_wide_quantisation_contains_the_box_and_is_tight():
    lo, hi, p, e, qlo, qhi, blo, bhi, *_ = wide_cases(300_000, 5)
    assert len(lo) > 290_000
    assert ((qlo >= 0) & (qlo <= qhi) & (qhi <= 255)).all()
    # outward: the dequantised box contains the float32 box, exactly
    assert (blo <= lo.astype(np.float64)).all() and (bhi >= hi.astype(np.float64)).all()
    # and at most one step looser on each side (the directed rounding of the
    # difference may cross one multiple of 2^e)
    step = np.ldexp(1.0, e)
    assert (lo.astype(np.float64) - blo < 2 * step).all()
    assert (bhi - hi.astype(np.float64) < 2 * step).all()
    # the scale: the smallest power of two that spans an extent in 255 steps
    ext = np.concatenate([np.ldexp(255.0, np.arange(-126, 128)), np.random.default_rng(9).uniform(0, 1e6, 10_000),
                          np.ldexp(np.random.default_rng(10).random(10_000), -120), [0.0]])
    ee = exp_for(ext)
    assert (np.ldexp(255.0, ee) >= ext).all()
    assert ((ee == -126) | (np.ldexp(255.0, ee - 1) < ext)).all()


def test_wide_node_test_never_rejects_a_child_the_segment_meets():
    lo, hi, p, e, qlo, qhi, blo, bhi, o, d = wide_cases(300_000, 6)
    nonzero = (np.abs(d) >= 1e-2 * np.abs(d).max(axis=1, keepdims=True)).all(axis=1)
    for tmax in [np.inf, 5.0, 40.0]:
        tm = tmax * 1.0
        tlim = f32(tm) * CULL if np.isfinite(tm) else f32(np.inf)
        got = wide_child_test(p, e, qlo, qhi, o, d, f32(0), tlim)
        want = exact_hit(blo, bhi, o, d, 0.0, tm)
        missed = want & ~got
        assert not missed.any(), f"tmax {tmax}: {missed.sum()} children rejected, e.g. case {np.nonzero(missed)[0][:3]}"
        assert want.sum() > 100_000
        # not permissive beyond the widening: with no near-zero direction
        # component, a child missed by a relative 1e-3 is rejected
        grow = (1e-3 * (np.abs(p).max(1) + np.abs(o).max(1) + np.abs(bhi - blo).max(1)))[:, None]
        far = nonzero & ~exact_hit(blo - grow, bhi + grow, o, d, 0.0, tm)
        assert far.sum() > 20_000
        assert not (got & far).any(), f"tmax {tmax}: {(got & far).sum()} far misses accepted"
