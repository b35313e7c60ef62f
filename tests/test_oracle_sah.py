"""Pins of the oracle's binned-SAH build (orc_sah_build) against closed forms
and invariants: rows of equal boxes along each axis give the balanced tree
the heuristic's cost 2 s^2 + 2 (16 - s)^2 (least at s = 8) implies; two distant
clusters are separated at the root; identical centroids are halved by
position; every tree is valid with contiguous leaf ranges; the surface-area
cost is below the LBVH's; and the hand-over to the Karras hierarchy below 40
levels: points 32x apart along one axis make the heuristic peel one point
per level, and the range left at level 40 gets the radix tree that equal
keys imply (split at the highest differing bit of the index range)."""
import numpy as np
import pytest

import oracle
import scenegen as g

LEAF = 0x80000000


def tree_ranges(child, n):
    """(first, last, depth) of every internal node; asserts each node and leaf
    is reached once from the root and each subtree's leaves are contiguous."""
    child = np.asarray(child, np.int64).reshape(-1, 2)
    m = max(n - 1, 0)
    seen = np.zeros(m, bool)
    depth = np.zeros(m, np.int64)
    order, stack = [], [0] if n > 1 else []
    while stack:
        k = stack.pop()
        assert not seen[k], f"node {k} reached twice"
        seen[k] = True
        order.append(k)
        for c in child[k]:
            if not c & LEAF:
                depth[c] = depth[k] + 1
                stack.append(int(c))
    assert len(order) == m
    size = np.zeros(m, np.int64)
    for k in reversed(order):
        size[k] = sum(1 if c & LEAF else size[c] for c in child[k])
    first = np.zeros(m, np.int64)
    leaves = np.zeros(n, bool)
    for k in order:
        f = first[k]
        for c in child[k]:
            if c & LEAF:
                assert (c & ~LEAF) == f, (k, c, f)
                assert not leaves[f]
                leaves[f] = True
                f += 1
            else:
                first[c] = f
                f += size[c]
    assert n <= 1 or leaves.all()
    return first, first + size - 1, depth


def boxes_mesh(lo, hi):
    """One triangle per box, spanning the box's lo and hi corners (its own
    bounding box is the box)."""
    lo, hi = np.asarray(lo, np.float32), np.asarray(hi, np.float32)
    n = lo.shape[0]
    v = np.empty((3 * n, 3), np.float32)
    v[0::3] = lo
    v[1::3] = hi
    v[2::3] = np.c_[hi[:, 0], lo[:, 1], hi[:, 2]]
    return v, np.arange(3 * n, dtype=np.uint32).reshape(n, 3)


def sah_cost(lohi_leaves, first, last):
    lo = np.array([lohi_leaves[f:l + 1, :3].min(0) for f, l in zip(first, last)], np.float64)
    hi = np.array([lohi_leaves[f:l + 1, 3:].max(0) for f, l in zip(first, last)], np.float64)
    d = hi - lo
    a = d[:, 0] * d[:, 1] + d[:, 1] * d[:, 2] + d[:, 2] * d[:, 0]
    return a.sum() / a[0]


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_row_of_equal_boxes_is_balanced(axis):
    k = np.arange(16, dtype=np.float32)
    lo = np.zeros((16, 3), np.float32)
    hi = np.ones((16, 3), np.float32)
    lo[:, axis] = k
    hi[:, axis] = k + 0.5
    v, i = boxes_mesh(lo, hi)
    r = oracle.sah_reference(v, i)
    first, last, _ = tree_ranges(r["child"], 16)
    for f, l, c in zip(first, last, r["child"]):
        n = l - f + 1
        left = 1 if c[0] & LEAF else None
        if left is None:
            left_last = last[c[0]]
            left = left_last - f + 1
        assert left == n // 2, (f, l, left)
    # leaves in spatial order along the axis
    assert np.array_equal(r["perm"], np.arange(16))


def test_distant_clusters_split_at_the_root():
    rng = np.random.default_rng(3)
    a = rng.uniform(0, 1, (40, 3)).astype(np.float32)
    b = rng.uniform(0, 1, (25, 3)).astype(np.float32) + np.float32([100, 0, 0])
    lo = np.r_[a, b]
    v, i = boxes_mesh(lo, lo + np.float32(0.05))
    r = oracle.sah_reference(v, i)
    first, last, _ = tree_ranges(r["child"], 65)
    c0 = int(r["child"][0][0])
    left = set(r["perm"][first[0]:(last[c0] if not c0 & LEAF else 0) + 1].tolist())
    assert left in (set(range(40)), set(range(40, 65)))


def test_identical_centroids_are_halved():
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    i = np.zeros((37, 3), np.uint32) + [0, 1, 2]
    r = oracle.sah_reference(v, i)
    first, last, _ = tree_ranges(r["child"], 37)
    assert np.array_equal(np.sort(r["perm"]), np.arange(37))
    for k, c in enumerate(r["child"]):
        n = last[k] - first[k] + 1
        if n <= 2:
            continue
        left = 1 if c[0] & LEAF else last[c[0]] - first[k] + 1
        assert left == n // 2


def test_large_box_is_split_off_alone():
    """Fourteen small boxes in a row, one more small box at x = 23 and a
    10-unit cube at x = 20..30.  Isolating the cube costs 23.75 * 15 + 300 =
    656.25 (half areas times counts), pairing it with its small neighbour
    13.75 * 14 + 240 * 2 = 672.5, so the root splits the cube off alone; the
    small neighbour sits one bin below the cube (bins 14 and 15 of the 16),
    so only a binning with all 16 bins can separate them."""
    lo = np.zeros((16, 3), np.float32)
    hi = np.zeros((16, 3), np.float32)
    for k in range(14):
        lo[k], hi[k] = [k, 0, 0], [k + 0.5, 0.5, 0.5]
    lo[14], hi[14] = [23, 0, 0], [23.5, 0.5, 0.5]
    lo[15], hi[15] = [20, -5, -5], [30, 5, 5]
    v, i = boxes_mesh(lo, hi)
    r = oracle.sah_reference(v, i)
    assert int(r["child"][0][1]) == LEAF | 15 and r["perm"][15] == 15
    tree_ranges(r["child"], 16)


def test_equal_costs_keep_the_first_axis():
    """Four equal boxes at the corners of a square in the xy plane: the x and
    y splits cost the same (2 * 11 each side), and the first candidate in
    the order of axes wins, so the root separates the two columns."""
    lo = np.array([[0, 0, 0], [4, 0, 0], [0, 4, 0], [4, 4, 0]], np.float32)
    v, i = boxes_mesh(lo, lo + np.float32(1))
    r = oracle.sah_reference(v, i)
    assert list(r["perm"]) == [0, 2, 1, 3]


@pytest.mark.parametrize("mesh", ["ico4", "soup", "large1"])
def test_valid_and_cheaper_than_lbvh(mesh):
    if mesh == "ico4":
        v, i = g.make_mesh("ico", 4)
    elif mesh == "soup":
        rng = np.random.default_rng(7)
        v = rng.normal(size=(5000, 3)).astype(np.float32)
        i = rng.integers(0, 5000, size=(7001, 3)).astype(np.uint32)
    else:
        v, i = g.large_scene().meshes[1]          # 25,600 triangles
    n = i.shape[0]
    r = oracle.sah_reference(v, i)
    assert np.array_equal(np.sort(r["perm"]), np.arange(n))
    first, last, depth = tree_ranges(r["child"], n)
    ref = oracle.lbvh_reference(v, i)
    cs = sah_cost(r["lohi"][r["perm"]], first, last)
    cl = sah_cost(ref["lohi"][ref["perm"]], ref["first"], ref["last"])
    assert cs < 0.97 * cl, (cs, cl)


def chain_to_level_40(k=42, m=9):
    """Points on the x axis: k chain points at x = 2^(120 - 5j) and m tail
    points at x = t 2^-100.  Each chain point lies 32x beyond the next, so in
    any range the largest one is alone in bin 15 and all others share bin 0;
    with zero y and z extents every split costs 0 and the first boundary of
    axis 0 wins.  The heuristic therefore peels one chain point per level, and
    the range left at level 40 (the last k - 40 chain points and the tail) is
    handed to the Karras hierarchy of its keys, which are all 0 (they quantise
    below the first Morton cell)."""
    x = np.r_[np.float32(2.0) ** (120 - 5 * np.arange(k)), np.arange(m) * np.float32(2.0 ** -100)].astype(np.float32)
    p = np.c_[x, np.zeros_like(x), np.zeros_like(x)]
    return boxes_mesh(p, p)


def karras_equal_keys(r, d, b):
    """Children of the radix tree over r equal keys, internal node j numbered
    d + j and leaf j numbered b + j.  With every key equal, a node over the
    index range [f, l] splits after gamma, where the highest bit in which f
    and l differ turns on; as in Karras 2012 the root is node 0, a left
    child [f, gamma] is node gamma and a right child [gamma + 1, l] is node
    gamma + 1."""
    child = {}
    todo = [(0, 0, r - 1)]
    while todo:
        node, f, l = todo.pop()
        top = 1 << ((f ^ l).bit_length() - 1)
        gamma = (l & ~(top - 1)) - 1
        child[d + node] = (LEAF | (b + gamma) if gamma == f else d + gamma,
                           LEAF | (b + gamma + 1) if gamma + 1 == l else d + gamma + 1)
        if gamma != f:
            todo.append((gamma, f, gamma))
        if gamma + 1 != l:
            todo.append((gamma + 1, gamma + 1, l))
    return child


@pytest.mark.parametrize("bits", [10, 21])
def test_hand_over_to_karras_at_level_40(bits):
    k, m = 42, 9
    v, i = chain_to_level_40(k, m)
    n = k + m
    r = oracle.sah_reference(v, i, bits)
    first, last, depth = tree_ranges(r["child"], n)
    # levels 0..39: node L peels chain point L into leaf n - 1 - L
    for lv in range(40):
        assert tuple(int(c) for c in r["child"][lv]) == (lv + 1, LEAF | (n - 1 - lv)), lv
    assert np.array_equal(r["perm"][n - 40:], np.arange(40)[::-1])
    # level 40: the Karras tree of the remaining r = n - 40 points, in their
    # Morton order (all keys 0, so index order: chain points 40, 41, the tail)
    rest = n - 40
    assert np.array_equal(r["perm"][:rest], np.arange(40, n))
    want = karras_equal_keys(rest, 40, 0)
    assert len(want) == rest - 1
    for node, ch in want.items():
        assert tuple(int(c) for c in r["child"][node]) == ch, node
    assert depth.max() == 40 + (rest - 1).bit_length() - 1
