"""Pins of the oracle's FXAA (Lottes 2009, as restated in oracle.cpp) against
values worked out by hand from the method's steps.

Notation: sub(s) = 0.75 * (s^2 (3 - 2 s))^2 is the sub-pixel offset for a
normalised contrast s; an edge-end blend moves a pixel by 0.5 - d / L across
the edge (d: distance to the nearer edge end, L: edge length)."""
import numpy as np
import pytest

import oracle


def sub(s):
    return 0.75 * (s * s * (3 - 2 * s)) ** 2


def block_image(h=40, w=50):
    """White, with a black block in rows >= 10, columns 20..27."""
    img = np.ones((h, w, 4), np.float32)
    img[10:, 20:28, :3] = 0
    return img


def test_constant_image_unchanged():
    img = np.full((9, 13, 4), 0.37, np.float32)
    assert np.array_equal(oracle.fxaa(img), img)


def test_low_contrast_unchanged():
    # luma step sqrt(0.52) - sqrt(0.5) = 0.014 < max(0.0312, 0.125 * 0.72)
    img = np.full((8, 8, 4), 0.5, np.float32)
    img[:, 4:, :3] = 0.52
    assert np.array_equal(oracle.fxaa(img), img)


def test_block_top_edge_blends_by_edge_distance():
    """Top edge of the block (between rows 9 and 10, 8 pixels long).

    Black pixel (24, 10): the edge is horizontal, the larger step is upward
    (to white), edge luma 0.5.  Searching at y = 9.5 the bilinear luma is 0.5
    over the block and 1 beyond it: the ends are found at x = 19 (5 unit
    steps) and x = 28 (4 steps), so d = 4, L = 9.  The pixel is darker than
    the edge luma while the luma at the end is above it, so it blends by
    0.5 - 4/9 = 1/18; its sub-pixel term, sub(1/3) = 0.0504, is smaller.  The
    sample 1/18 of a pixel upward reads 1/18 of white.

    Black corner pixel (20, 10): the orientation tests tie (3 = 3) and pick
    horizontal; the ends are x = 19 (1 step) and x = 28.5 (steps 1,1,1,1,1,
    1.5,2: the sample at 28.5 averages columns 28 and 29, both white above and
    below), so d = 1, L = 9.5: offset 0.5 - 1/9.5.

    White pixel (24, 9) above the edge: its luma is above the edge luma and
    the end luma too, so no edge blend; the 3x3 mean is 8/12, contrast s =
    1/3, offset sub(1/3) toward the black pixel below."""
    out = oracle.fxaa(block_image())
    np.testing.assert_allclose(out[10, 24, :3], 1 / 18, atol=2e-6)
    np.testing.assert_allclose(out[10, 20, :3], 0.5 - 1 / 9.5, atol=2e-6)
    np.testing.assert_allclose(out[9, 24, :3], 1 - sub(1 / 3), atol=2e-6)
    # far from the block nothing changes, alpha never does
    assert np.array_equal(out[2, 2], block_image()[2, 2])
    assert np.array_equal(out[..., 3], block_image()[..., 3])


def test_transposed_block_takes_the_vertical_branch():
    """The same block transposed: the edge is vertical and the search runs
    along y; the pixels that were not ties give the transposed values."""
    img = np.ascontiguousarray(block_image().transpose(1, 0, 2))
    out = oracle.fxaa(img)
    np.testing.assert_allclose(out[24, 10, :3], 1 / 18, atol=2e-6)
    np.testing.assert_allclose(out[24, 9, :3], 1 - sub(1 / 3), atol=2e-6)


@pytest.mark.parametrize("h", [5, 64])
def test_straight_edge_sub_pixel_only(h):
    """A vertical edge through the whole image (clamped addressing continues
    it): the search finds no end (26.5 pixels both ways, end luma equal to
    the edge luma), so the edge blend is 0 and only sub(1/3) remains: the
    dark pixel takes sub(1/3) of white, the bright one gives it away."""
    img = np.zeros((h, 16, 4), np.float32)
    img[:, 8:, :3] = 1
    out = oracle.fxaa(img)
    np.testing.assert_allclose(out[h // 2, 7, :3], sub(1 / 3), atol=2e-6)
    np.testing.assert_allclose(out[h // 2, 8, :3], 1 - sub(1 / 3), atol=2e-6)
    np.testing.assert_array_equal(out[:, :6], img[:, :6])


def test_output_is_a_blend_of_the_pixel_and_one_neighbour():
    """Each output colour is a bilinear sample at most 0.75 pixel from the
    pixel's centre along one axis: per channel it lies between the pixel and
    one of its four neighbours, and a pixel that moves does so by the same
    fraction in every channel."""
    rng = np.random.default_rng(5)
    img = rng.uniform(0, 1, (23, 31, 4)).astype(np.float32)
    img[..., 3] = rng.integers(0, 2, (23, 31))
    out = oracle.fxaa(img).astype(np.float64)
    src = img.astype(np.float64)
    pad = np.pad(src, ((1, 1), (1, 1), (0, 0)), mode="edge")
    assert np.array_equal(out[..., 3], src[..., 3])
    for y in range(23):
        for x in range(31):
            c = src[y, x, :3]
            ok = False
            for dy, dx in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                nb = pad[y + 1 + dy, x + 1 + dx, :3]
                lo, hi = np.minimum(c, nb) - 1e-6, np.maximum(c, nb) + 1e-6
                if np.all((out[y, x, :3] >= lo) & (out[y, x, :3] <= hi)):
                    d = nb - c
                    big = np.abs(d) > 1e-3
                    if not big.any():
                        ok = True
                        break
                    t = (out[y, x, :3] - c)[big] / d[big]
                    if np.all(t > -1e-4) and np.all(t < 0.75 + 1e-4) and np.ptp(t) < 1e-4:
                        ok = True
                        break
            assert ok, (y, x)


def test_tiny_sizes():
    for h, w in [(1, 1), (1, 7), (7, 1), (2, 2)]:
        img = np.random.default_rng(h * 10 + w).uniform(0, 1, (h, w, 4)).astype(np.float32)
        out = oracle.fxaa(img)
        assert out.shape == img.shape and np.all(np.isfinite(out))


def straight_edge(left, right, h=6, w=12):
    img = np.ones((h, w, 4), np.float32)
    img[:, : w // 2, :3] = left
    img[:, w // 2:, :3] = right
    return img


@pytest.mark.parametrize("left,right,why", [
    # luma weights 0.299 / 0.587 / 0.114: lumas 0.547 | 0.698, range 0.151
    # above 0.125 * 0.698; with red and green weights swapped the lumas would
    # be 0.766 | 0.698 and the range (0.068) below 0.125 * 0.766
    ((1.0, 0.0, 0.0), (0.55, 0.55, 0.0), "weights"),
    # luma is the square root: 0.141 | 0.2, range 0.059 above 0.0312; the
    # linear values (0.02 | 0.04) would stay below it
    ((0.02, 0.02, 0.02), (0.04, 0.04, 0.04), "square root"),
    # range 0.837 - 0.707 = 0.130 between 0.125 and 0.25 of the brighter luma
    ((0.5, 0.5, 0.5), (0.7, 0.7, 0.7), "relative threshold"),
])
def test_edge_thresholds(left, right, why):
    """A straight edge above the contrast threshold: both edge pixels move
    by sub(1/3) toward each other (no edge end is found), whatever the two
    colours, since the contrast is normalised by the range."""
    img = straight_edge(left, right)
    out = oracle.fxaa(img)
    a, b = np.array(left, np.float64), np.array(right, np.float64)
    np.testing.assert_allclose(out[3, 5, :3], a + sub(1 / 3) * (b - a), atol=2e-6, err_msg=why)
    np.testing.assert_allclose(out[3, 6, :3], b + sub(1 / 3) * (a - b), atol=2e-6, err_msg=why)
    assert np.array_equal(out[:, :4], img[:, :4])


def test_edge_end_at_a_quarter_of_the_step():
    """The black block of block_image on a grey floor (0.49, luma 0.7)
    instead of a white one: searching along the top edge at y = 9.5 the
    bilinear luma is 0.5 over the block and 0.85 beyond it, 0.35 from the
    edge luma.  That is at least a quarter of the pixel's luma step (1), so
    the ends are found at x = 19 and 28 as on the white floor, and the black
    pixel (24, 10) blends by 0.5 - 4/9 = 1/18 again; a search that needed
    half the step would run to the image border and leave sub(1/3)."""
    img = block_image()
    img[10:, :20, :3] = 0.49
    img[10:, 28:, :3] = 0.49
    out = oracle.fxaa(img)
    np.testing.assert_allclose(out[10, 24, :3], 1 / 18, atol=2e-6)
