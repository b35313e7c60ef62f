"""Whitted render on the GPU vs the FP64 oracle and closed forms.

Pixels must agree within 2e-3 absolute per channel, except pixels whose ray
tree holds a ray the oracle flags ambiguous (counted, bounded)."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2001_09792_gb300 as rg
import scenegen as g

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("librg")]
PIX_TOL = 2e-3
KAPPA = 16.0
REL_T = 1e-5
AMB = float(np.float32(0.1))


def render(scene, gs=None, w=None, h=None, depth=None, camera=None):
    own = gs is None
    if own:
        gs = rg.GpuScene(scene)
    try:
        img = rg.rg_render(gs.h, camera or scene.camera, w or scene.width, h or scene.height,
                           depth or scene.max_depth)
        rg.rg_sync(gs.h)
        return img.cpu().numpy().reshape(-1, 4).astype(np.float64)
    finally:
        if own:
            gs.close()


def compare(img, ref, pixels=None, max_exempt=1e-4, label=""):
    """Pixels whose ray tree holds no ambiguous ray must agree within PIX_TOL;
    pixels that differ must all be flagged, and their fraction is bounded."""
    if pixels is not None:
        img = img[pixels]
    ok = ~ref["ambiguous"]
    err = np.abs(img - ref["rgba"])
    worst = err[ok].max() if ok.any() else 0.0
    bad = ok & (err.max(1) > PIX_TOL)
    assert not bad.any(), f"{label}: {bad.sum()} pixels off by up to {err[bad].max():.3e}, e.g. {np.nonzero(bad)[0][:5]}"
    differ = err.max(1) > PIX_TOL
    frac = differ.mean()
    assert frac <= max_exempt, f"{label}: {differ.sum()} exempt pixels differ ({frac:.2e})"
    return worst, frac


def test_tiny_scene_full_image():
    s = g.tiny_scene()
    img = render(s)
    ref = oracle.OracleScene(s).render(s.camera, s.width, s.height, s.max_depth, kappa=KAPPA, rel_t=REL_T)
    worst, frac = compare(img, ref, label="tiny")
    assert img[:, 3].mean() > 0.3


@pytest.mark.parametrize("depth", [1, 2, 4])
def test_medium_scene_sampled_pixels(depth):
    """1920x1080 at the given depth, rendered whole on the GPU; a seeded sample
    of pixels is rendered by the oracle."""
    s = g.medium_scene()
    img = render(s, depth=depth)
    pix = np.random.default_rng(depth).choice(s.width * s.height, 30_000, replace=False).astype(np.uint32)
    ref = oracle.OracleScene(s).render(s.camera, s.width, s.height, depth, pixels=pix, kappa=KAPPA, rel_t=REL_T)
    worst, frac = compare(img, ref, pixels=pix, label=f"medium d{depth}")
    print(f"medium depth {depth}: worst {worst:.2e}, differing {frac:.2e}, ambiguous {ref['ambiguous'].mean():.2e}")


def test_ragged_resolution_and_camera():
    s = g.tiny_scene()
    # (a target on a cube edge would put the whole centre column on that edge)
    cam = dict(eye=(3, 1.5, 4), target=(0.4, 0.1, -0.3), up=(0, 1, 0), vfov=45.0)
    img = render(s, w=97, h=33, camera=cam)
    ref = oracle.OracleScene(s).render(cam, 97, 33, 1, kappa=KAPPA, rel_t=REL_T)
    compare(img, ref, label="ragged")


def _scene(meshes, M, mats, light_pos, light_I=(1, 1, 1)):
    n = len(M)
    return g.Scene(meshes=[m for m in meshes], M=np.stack(M), mesh_id=np.arange(n, dtype=np.uint32),
                   material_id=np.arange(n, dtype=np.uint32), mat_type=np.array([m[0] for m in mats], np.uint32),
                   mat_albedo=np.array([m[1] for m in mats], np.float32),
                   mat_ior=np.array([m[2] for m in mats], np.float32),
                   light_pos=np.array([light_pos], np.float32), light_I=np.array([light_I], np.float32))


def test_closed_form_lambert():
    v, i = g.quad_mesh(20.0, 0.0)
    a = 0.75
    s = _scene([(v, i)], [g.affine(np.eye(3), [0, 0, 0])], [(0, (a, a, a), 1.0)], (3.0, 4.0, 0.0))
    cam = dict(eye=(0, 10, 0), target=(0, 0, 0), up=(0, 0, -1), vfov=10.0)
    img = render(s, w=1, h=1, depth=1, camera=cam)
    eps = 1e-4
    cos = (4 - eps) / math.sqrt(9 + (4 - eps) ** 2)
    want = a * AMB + a * cos
    np.testing.assert_allclose(img[0], [want, want, want, 1.0], atol=1e-5)


def test_closed_form_mirror_and_depth_limit():
    fv, fi = g.quad_mesh(20.0, 0.0)
    wv = np.array([[3, -10, -10], [3, 10, -10], [3, 10, 10], [3, -10, 10]], np.float32)
    wi = np.array([[0, 1, 2], [0, 2, 3]], np.uint32)
    a, tint = 0.625, 0.875
    s = _scene([(fv, fi), (wv, wi)], [g.affine(np.eye(3), [0, 0, 0])] * 2,
               [(1, (tint, tint, tint), 1.0), (0, (a, a, a), 1.0)], (2.0, 2.0, 0.0))
    cam = dict(eye=(0, 1, 0), target=(1, 0, 0), up=(0, 1, 0), vfov=1.0)
    img = render(s, w=1, h=1, depth=2, camera=cam)
    lx, ly = -1 + 3e-4, -1e-4
    want = tint * (a * AMB + a * (-lx / math.hypot(lx, ly)))
    np.testing.assert_allclose(img[0, :3], [want] * 3, atol=1e-5)
    img = render(s, w=1, h=1, depth=1, camera=cam)
    np.testing.assert_allclose(img[0], [0, 0, 0, 1], atol=0)


def test_closed_form_glass_slab_series():
    fv, fi = g.quad_mesh(40.0, 0.0)
    cv, ci = g.cube_mesh(0.5)
    a = 0.5
    s = _scene([(fv, fi), (cv, ci)], [g.affine(np.eye(3), [0, 0, 0]), g.affine(np.diag([10.0, 1.0, 10.0]), [0, 3, 0])],
               [(0, (a, a, a), 1.0), (2, (1, 1, 1), 1.5)], (0.0, 2.0, 0.0))
    cam = dict(eye=(0, 10, 0), target=(0, 0, 0), up=(0, 0, -1), vfov=1.0)
    img = render(s, w=1, h=1, depth=8, camera=cam)
    R0 = 0.04
    floor = a * AMB + a
    bg = np.array([0.2, 0.3, 0.5])

    def down(d):
        return np.zeros(3) if d >= 8 else R0 * up(d + 1) + (1 - R0) * floor

    def up(d):
        return np.zeros(3) if d >= 8 else R0 * down(d + 1) + (1 - R0) * bg

    want = R0 * bg + (1 - R0) * down(2)
    np.testing.assert_allclose(img[0, :3], want, atol=1e-5)
    assert img[0, 3] == 1.0


def test_total_internal_reflection_scene_vs_oracle():
    """A glass sphere and mirrors at max depth 8: many TIR paths."""
    rng = np.random.default_rng(3)
    meshes = [g.make_mesh("ico", 3), g.quad_mesh(60.0, -6.0), g.cube_mesh(0.5)]
    M = [g.affine(np.eye(3), [0, 0, 0]), g.affine(np.eye(3), [0, 0, 0]), g.affine(g.random_rotation(rng), [8, 0, -4], 6)]
    mats = [(2, (1, 1, 1), 1.5), (0, (0.7, 0.6, 0.5), 1.0), (1, (0.9, 0.9, 0.9), 1.0)]
    s = _scene(meshes, M, mats, (10, 30, 20))
    cam = dict(eye=(0, 4, 18), target=(0, 0, 0), up=(0, 1, 0), vfov=50.0)
    img = render(s, w=160, h=120, depth=8, camera=cam)
    ref = oracle.OracleScene(s).render(cam, 160, 120, 8, kappa=KAPPA, rel_t=REL_T)
    compare(img, ref, label="glass")


def test_refit_render_equals_fresh_render():
    s = g.medium_scene(width=320, height=180, max_depth=3)
    M2 = g.motion(s.M, 2)
    with rg.GpuScene(s) as gs:
        gs.refit(M2)
        a = render(s, gs=gs)
    s.M = M2
    b = render(s)
    np.testing.assert_allclose(a, b, atol=1e-5)


def test_render_repeatable(tmp_path):
    s = g.medium_scene(width=640, height=360, max_depth=4)
    with rg.GpuScene(s) as gs:
        a = render(s, gs=gs)
        b = render(s, gs=gs)
    np.testing.assert_allclose(a, b, atol=1e-5)


@pytest.mark.parametrize("lights", [4, 1])
def test_paired_launches_equal_separate_launches(lights):
    """Tracing a level's shadow rays in one launch with the next level's
    closest-hit rays gives the image of separate launches (up to the order of
    float additions into a pixel) from the same rays, in max_depth - 1 pairs."""
    s = g.medium_scene(width=480, height=270, max_depth=5)
    s.light_pos, s.light_I = s.light_pos[:lights], s.light_I[:lights]
    out = {}
    for name, flags in [("pair", rg.RG_SCENE_TIMING | rg.RG_SCENE_COUNT),
                        ("apart", rg.RG_SCENE_TIMING | rg.RG_SCENE_COUNT | rg.RG_SCENE_NO_PAIR)]:
        with rg.GpuScene(s, flags=flags) as gs:
            rg.rg_reset_stats(gs.h)
            img = render(s, gs=gs)
            out[name] = (img, rg.rg_get_stats(gs.h))
    (a, sa), (b, sb) = out["pair"], out["apart"]
    np.testing.assert_allclose(a, b, atol=1e-5)
    for k in ["closest_rays", "shadow_rays", "node_visits", "tri_tests", "inst_entries", "any_node_visits",
              "any_tri_tests", "any_inst_entries"]:
        assert sa[k] == sb[k], k
    assert sa["pair_launches"] == s.max_depth - 1 and sb["pair_launches"] == 0
    assert sa["trace_launches"] == 1 and sa["any_launches"] == 1
    assert sb["trace_launches"] == s.max_depth and sb["any_launches"] == s.max_depth
    assert sa["kernel_launches"] == sb["kernel_launches"] - (s.max_depth - 1)


def test_shared_scenes_render_concurrently():
    """Two scenes over the same BLAS (rg_scene_create_shared), each with its
    own instance transforms, render on two streams at once; each image equals
    the render of a fresh scene with those transforms.  The shared BLAS
    outlive the scene that built them, and a shared set takes no new BLAS."""
    s = g.medium_scene(width=320, height=180, max_depth=4)
    Ms = [g.motion(s.M, 3), g.motion(s.M, 8)]
    refs = []
    for M in Ms:
        s2 = g.medium_scene(width=320, height=180, max_depth=4)
        s2.M = M
        refs.append(render(s2))
    a = rg.GpuScene(s)
    b = a.shared()
    try:
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        imgs = []
        for gs, M, st in zip([a, b], Ms, streams):
            with torch.cuda.stream(st):
                inst = torch.from_numpy(rg.pack_instances(M, [gs.blas[m] for m in s.mesh_id], s.material_id)).cuda()
                rg.rg_tlas_build(gs.h, inst, stream=st)
                imgs.append(rg.rg_render(gs.h, s.camera, s.width, s.height, s.max_depth, stream=st))
        torch.cuda.synchronize()
        for img, ref in zip(imgs, refs):
            np.testing.assert_allclose(img.cpu().numpy().reshape(-1, 4).astype(np.float64), ref, atol=1e-5)
        v, i = g.cube_mesh(0.5)
        with pytest.raises(rg.RgError) as e:
            rg.rg_blas_build(b.h, torch.from_numpy(v).cuda(), torch.from_numpy(i.view(np.int32)).cuda())
        assert e.value.status == rg.RG_ERR_INVALID_ARG
        a.close()                                   # b keeps the BLAS
        img = render(s, gs=b)
        b_ref = g.medium_scene(width=320, height=180, max_depth=4)
        b_ref.M = Ms[1]
        np.testing.assert_allclose(img, render(b_ref), atol=1e-5)
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("lights,bvh", [(4, 0), (0, 0), (4, rg.RG_SCENE_COMPRESSED)])
def test_frugal_queues_equal_worst_case_queues(lights, bvh):
    """Queues sized from each level's ray count (the host waits per level,
    RG_SCENE_FRUGAL) and queues sized once for the frame's worst case (no host
    wait) render the same image from the same rays and traversal work, on the
    binary and on the compressed BVH."""
    s = g.medium_scene(width=480, height=270, max_depth=6)
    s.light_pos, s.light_I = s.light_pos[:lights], s.light_I[:lights]
    out = {}
    for name, flags in [("frugal", rg.RG_SCENE_FRUGAL), ("worst", 0)]:
        with rg.GpuScene(s, flags=flags | bvh | rg.RG_SCENE_COUNT) as gs:
            rg.rg_reset_stats(gs.h)
            img = render(s, gs=gs)
            out[name] = (img, rg.rg_get_stats(gs.h))
    (a, sa), (b, sb) = out["frugal"], out["worst"]
    np.testing.assert_allclose(a, b, atol=1e-5)
    for k in ["closest_rays", "shadow_rays", "node_visits", "tri_tests", "inst_entries", "any_node_visits",
              "any_tri_tests", "any_inst_entries"]:
        assert sa[k] == sb[k], k
    assert sa["closest_rays"] > s.width * s.height


def test_deep_render_beyond_the_worst_case_budget():
    """A render whose worst-case queues exceed the budget (960x540, depth 10:
    up to 512 rays per pixel at the last level) takes the per-level path and
    agrees with the oracle on sampled pixels."""
    s = g.medium_scene(width=960, height=540, max_depth=10)
    img = render(s)
    pix = np.random.default_rng(10).choice(s.width * s.height, 10_000, replace=False).astype(np.uint32)
    ref = oracle.OracleScene(s).render(s.camera, s.width, s.height, s.max_depth, pixels=pix, kappa=KAPPA, rel_t=REL_T)
    compare(img, ref, pixels=pix, label="deep")


def test_split_shadow_rays_see_an_occluder_near_the_light():
    """Depth 1 with few shadow rays: each is traced as 8 segments.  A small
    occluder at 90 % of the way to the light lies in the last segments only;
    the pixels it shadows get the ambient term alone, the others the Lambert
    term too, as the oracle renders them."""
    v, i = g.quad_mesh(20.0, 0.0)
    ov, oi = g.quad_mesh(0.4, 0.0)
    a = 0.75
    s = _scene([(v, i), (ov, oi)], [g.affine(np.eye(3), [0, 0, 0]), g.affine(np.eye(3), [0, 9.0, 0])],
               [(0, (a, a, a), 1.0), (0, (a, a, a), 1.0)], (0.0, 10.0, 0.0))
    cam = dict(eye=(0, 6, 14), target=(0, 0, 0), up=(0, 1, 0), vfov=50.0)
    w = h = 96
    img = render(s, w=w, h=h, depth=1, camera=cam)
    ref = oracle.OracleScene(s).render(cam, w, h, 1, kappa=KAPPA, rel_t=REL_T)
    compare(img, ref, label="occluder near the light")
    ground = img[:, 3] == 1.0
    shadowed = ground & (np.abs(img[:, 0] - a * AMB) < 1e-6)
    assert shadowed.sum() > 100 and (ground & ~shadowed).sum() > 1000
