"""The continuous-batching render server.

* Each request's image equals rg_tlas_refit + rg_render of that request alone
  (same instance transforms), whether it runs alone or in a mix of scenes,
  resolutions and depths, up to the order of float additions into a pixel.
* The server traces exactly the closest-hit and shadow rays the one-at-a-time
  renders trace (the same ray trees).
* A ring much smaller than the work wraps around many times; requests
  submitted mid-flight join as slots free; the CUDA-graph step and the
  direct-launch step agree.
* A batched render agrees with the FP64 oracle on sampled pixels.
* The autotuner sets valid shapes and round-trips its JSON cache."""
import dataclasses
import json

import numpy as np
import pytest
import torch

import oracle
import paper_2001_09792_gb300 as rg
import scenegen as g
from test_gpu_render import KAPPA, REL_T, compare

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("librg")]
ATOL = 1e-5


@pytest.fixture(scope="module")
def scenes():
    """The serving scene set: the tiny scene plus 7 medium-style seeds."""
    descs = g.serving_scenes()
    gss = [rg.GpuScene(s) for s in descs]
    yield descs, gss
    for gs in gss:
        gs.close()


def alone(desc, gs, M, camera, w, h, depth):
    gs.refit(M)
    rg.rg_reset_stats(gs.h)
    img = rg.rg_render(gs.h, camera, w, h, depth)
    rg.rg_sync(gs.h)
    st = rg.rg_get_stats(gs.h)
    gs.refit(desc.M)
    rg.rg_sync(gs.h)
    return img.cpu().numpy(), st["closest_rays"], st["shadow_rays"]


def make_requests(descs, n, seed, sizes, depths=range(1, 9)):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        sid = int(rng.integers(0, len(descs)))
        w, h = sizes[int(rng.integers(0, len(sizes)))]
        depth = int(rng.choice(list(depths)))
        M = g.motion(descs[sid].M, int(rng.integers(0, 1000)))
        out.append(dict(scene=sid, w=w, h=h, depth=depth, M=M, camera=descs[sid].camera))
    return out


def run_server(gss, reqs, feed_every=None, **kw):
    """Submits the requests (all at once, or `feed_every` steps apart) and
    steps until all complete; returns images, completions, stats."""
    srv = rg.rg_server_create(**kw)
    try:
        ids = [rg.rg_server_add_scene(srv, gs.h) for gs in gss]
        assert ids == list(range(len(gss)))
        imgs = [torch.full((q["h"], q["w"], 4), float("nan"), device="cuda") for q in reqs]
        done = []
        k = 0
        steps = 0
        while True:
            while k < len(reqs) and (feed_every is None or steps >= k * feed_every):
                q = reqs[k]
                rg.rg_server_submit(srv, q["scene"], q["camera"], q["w"], q["h"], q["depth"], imgs[k], q["M"], tag=k)
                k += 1
            st = rg.rg_server_get_stats(srv)
            if k == len(reqs) and st["pending"] == 0 and st["active"] == 0:
                break
            rg.rg_server_step(srv)
            steps += 1
            done += rg.rg_server_poll(srv)
            assert steps < 100_000
        stats = rg.rg_server_get_stats(srv)
    finally:
        rg.rg_server_destroy(srv)
    return [i.cpu().numpy() for i in imgs], done, stats


def check_against_alone(descs, gss, reqs, imgs, stats=None):
    tot_c = tot_s = 0
    for q, img in zip(reqs, imgs):
        ref, nc, ns = alone(descs[q["scene"]], gss[q["scene"]], q["M"], q["camera"], q["w"], q["h"], q["depth"])
        np.testing.assert_allclose(img, ref, atol=ATOL, rtol=0, err_msg=str({k: q[k] for k in ("scene", "w", "h", "depth")}))
        tot_c += nc
        tot_s += ns
    if stats is not None:
        assert stats["closest_rays"] == tot_c
        assert stats["shadow_rays"] == tot_s


def test_single_request_equals_render(scenes):
    descs, gss = scenes
    for sid, (w, h, depth) in [(0, (64, 64, 1)), (1, (320, 180, 4))]:
        reqs = [dict(scene=sid, w=w, h=h, depth=depth, M=descs[sid].M, camera=descs[sid].camera)]
        imgs, done, st = run_server(gss, reqs)
        assert len(done) == 1 and done[0]["tag"] == 0
        check_against_alone(descs, gss, reqs, imgs, st)


@pytest.mark.parametrize("lanes", [1, 4])
def test_mix_equals_alone(scenes, lanes):
    """24 requests over all 8 scenes at mixed resolutions and depths 1-8,
    each with its own instance motion, through a batch limit that makes the
    steps interleave them; in one lane, and spread over four lanes whose
    steps run at the same time."""
    descs, gss = scenes
    reqs = make_requests(descs, 24, seed=7, sizes=[(160, 120), (320, 240), (640, 360), (97, 33)])
    imgs, done, st = run_server(gss, reqs, ring_log2=22, batch_rays=1 << 18, admit_rays=1 << 21, lanes=lanes)
    assert sorted(d["tag"] for d in done) == list(range(len(reqs)))
    # requests were in flight together and finished over many steps
    spans = [(d["admitted_step"], d["completed_step"]) for d in done]
    most = max(sum(a <= t <= c for a, c in spans) for t in range(1, st["steps"] + 1))
    assert most >= 8
    assert len({c for _, c in spans}) > 3
    assert st["ring_peak"] <= (1 << 22)
    check_against_alone(descs, gss, reqs, imgs, st)


@pytest.mark.parametrize("lanes", [1, 4])
def test_ring_counters_wrap_past_2_32(scenes, monkeypatch, lanes):
    """The ring positions are free-running 32-bit counters, so a long-running
    server wraps them after 2^32 path rays.  A server whose empty rings start
    1,000 positions below 2^32 (test hook RG_TEST_RING_START, read when the
    server is created) runs a mixed request set across the wrap (every
    request has more than 1,000 primary rays, so every lane that takes one
    wraps): every image equals its render alone, and the server traces the
    same rays."""
    monkeypatch.setenv("RG_TEST_RING_START", str(2 ** 32 - 1_000))
    descs, gss = scenes
    reqs = make_requests(descs, 12, seed=21, sizes=[(160, 120), (320, 240), (97, 33)])
    imgs, done, st = run_server(gss, reqs, ring_log2=20, batch_rays=1 << 16, lanes=lanes)
    assert sorted(d["tag"] for d in done) == list(range(len(reqs)))
    check_against_alone(descs, gss, reqs, imgs, st)


def test_small_ring_wraps_and_admits_mid_flight(scenes):
    descs, gss = scenes
    reqs = make_requests(descs, 20, seed=11, sizes=[(128, 96), (160, 120), (61, 17)], depths=[2, 4, 8])
    imgs, done, st = run_server(gss, reqs, feed_every=3, ring_log2=16, batch_rays=1 << 13, admit_rays=1 << 15)
    # the ring (65,536 rays) is passed several times over, and fills up
    # enough for newest-first steps
    assert st["closest_rays"] > 2 * (1 << 16)
    assert st["ring_peak"] <= (1 << 16)
    assert st["newest_first_steps"] > 0
    # requests fed later are admitted later
    adm = {d["tag"]: d["admitted_step"] for d in done}
    assert adm[len(reqs) - 1] > adm[0]
    check_against_alone(descs, gss, reqs, imgs, st)


def test_graph_and_direct_launch_agree(scenes):
    descs, gss = scenes
    reqs = make_requests(descs, 6, seed=13, sizes=[(200, 150)])
    a, _, sa = run_server(gss, reqs, batch_rays=1 << 16)
    b, _, sb = run_server(gss, reqs, batch_rays=1 << 16, flags=rg.RG_SERVER_NO_GRAPH)
    for x, y in zip(a, b):
        np.testing.assert_allclose(x, y, atol=ATOL, rtol=0)
    assert sa["steps"] == sb["steps"] and sa["closest_rays"] == sb["closest_rays"]
    assert sa["graph_launches"] > 0 and sb["graph_launches"] == 0
    assert sa["kernel_launches"] == sb["kernel_launches"]


def test_batched_render_vs_oracle(scenes):
    descs, gss = scenes
    sid = 3
    s = descs[sid]
    M = g.motion(s.M, 5)
    reqs = [dict(scene=sid, w=480, h=270, depth=5, M=M, camera=s.camera)]
    reqs += make_requests(descs, 5, seed=17, sizes=[(160, 120)])
    imgs, _, _ = run_server(gss, reqs, batch_rays=1 << 16)
    s2 = dataclasses.replace(s, M=M)
    pix = np.random.default_rng(1).choice(480 * 270, 20_000, replace=False).astype(np.uint32)
    ref = oracle.OracleScene(s2).render(s.camera, 480, 270, 5, pixels=pix, kappa=KAPPA, rel_t=REL_T)
    compare(imgs[0].reshape(-1, 4).astype(np.float64), ref, pixels=pix, label="served")


def test_autotune_sets_valid_shapes_and_caches(scenes, tmp_path):
    descs, gss = scenes
    s = descs[1]
    cache = tmp_path / "shapes.json"
    scratch = torch.empty((270, 480, 4), device="cuda")
    srv = rg.rg_server_create(batch_rays=1 << 20)
    try:
        sid = rg.rg_server_add_scene(srv, gss[1].h)
        out = rg.rg_server_autotune(srv, sid, s.camera, 480, 270, 4, scratch, cache_path=str(cache))
        for o in out:
            assert o["block"] in (64, 128, 256) and 1 <= o["refill"] <= 32 and o["ms"] > 0
            assert o["stack"] in (0, 8, 16) and (o["stack"] == 0 or o["block"] == 128)
        assert rg.rg_server_get_shape(srv, 0) == {k: out[0][k] for k in ("block", "blocks_per_sm", "refill", "stack")}
        st = rg.rg_server_get_stats(srv)
        assert st["active"] == 0 and st["ring_rays"] == 0
        # the tuned server still renders correctly
        img = torch.empty((120, 160, 4), device="cuda")
        rg.rg_server_submit(srv, sid, s.camera, 160, 120, 4, img, s.M)
        rg.rg_server_drain(srv)
        ref, _, _ = alone(s, gss[1], s.M, s.camera, 160, 120, 4)
        np.testing.assert_allclose(img.cpu().numpy(), ref, atol=ATOL, rtol=0)
    finally:
        rg.rg_server_destroy(srv)
    entries = json.loads(cache.read_text())
    assert len(entries) == 1 and entries[0]["sms"] > 0
    assert entries[0]["closest"]["block"] == out[0]["block"]
    # a second server takes the cached shapes without timing
    srv = rg.rg_server_create()
    try:
        sid = rg.rg_server_add_scene(srv, gss[1].h)
        again = rg.rg_server_autotune(srv, sid, s.camera, 480, 270, 4, scratch, cache_path=str(cache))
        assert [{k: a[k] for k in ("block", "blocks_per_sm", "refill", "stack")} for a in again] == \
               [{k: o[k] for k in ("block", "blocks_per_sm", "refill", "stack")} for o in out]
        assert again[0]["ms"] < 0
    finally:
        rg.rg_server_destroy(srv)


@pytest.mark.parametrize("stack", [8, 16])
def test_short_stack_shapes_serve_the_same_image(scenes, stack):
    """Both traversals with a short stack of 8 or 16 entries in shared memory
    (the rest in local memory) give the image of the default shapes: where a
    stack entry lives does not change the traversal."""
    descs, gss = scenes
    s = descs[1]
    imgs = []
    for sd in (0, stack):
        srv = rg.rg_server_create(batch_rays=1 << 18)
        try:
            sid = rg.rg_server_add_scene(srv, gss[1].h)
            for which in (0, 1):
                rg.rg_server_set_shape(srv, which, 128, 0, 32, sd)
                assert rg.rg_server_get_shape(srv, which)["stack"] == sd
            img = torch.empty((180, 240, 4), device="cuda")
            rg.rg_server_submit(srv, sid, s.camera, 240, 180, 6, img, s.M)
            rg.rg_server_drain(srv)
            imgs.append(img.cpu().numpy())
        finally:
            rg.rg_server_destroy(srv)
    np.testing.assert_allclose(imgs[1], imgs[0], atol=ATOL, rtol=0)
    srv = rg.rg_server_create()
    try:
        with pytest.raises(rg.RgError):
            rg.rg_server_set_shape(srv, 0, 256, 0, 32, 8)  # short stacks only with 128 threads
    finally:
        rg.rg_server_destroy(srv)


def test_bad_requests_rejected(scenes):
    descs, gss = scenes
    srv = rg.rg_server_create(ring_log2=16)
    try:
        sid = rg.rg_server_add_scene(srv, gss[0].h)
        img = torch.empty((64, 64, 4), device="cuda")
        cam = descs[0].camera
        for args in [(sid, cam, 64, 64, 0), (sid, cam, 64, 64, 16), (sid + 5, cam, 64, 64, 1)]:
            with pytest.raises(rg.RgError) as e:
                rg.rg_server_submit(srv, *args, img)
            assert e.value.status == rg.RG_ERR_INVALID_ARG
        big = torch.empty((256, 256, 4), device="cuda")   # 65,536 px > half the ring
        with pytest.raises(rg.RgError):
            rg.rg_server_submit(srv, sid, cam, 256, 256, 1, big)
        # a singular per-request transform is reported by the step that refits it
        M = descs[0].M.copy()
        M[1, :, :3] = 0
        rg.rg_server_submit(srv, sid, cam, 64, 64, 1, img, M)
        with pytest.raises(rg.RgError) as e:
            rg.rg_server_drain(srv)
        assert e.value.status == rg.RG_ERR_SINGULAR
    finally:
        rg.rg_server_destroy(srv)


def test_admission_bound_keeps_requests_apart(scenes):
    """In one lane with the default bound (one batch of rays in flight), a
    request larger than the bound is admitted alone into the empty ring; the
    small ones are admitted together once the rays in flight fall below the
    bound."""
    descs, gss = scenes
    reqs = [dict(scene=1, w=320, h=240, depth=3, M=descs[1].M, camera=descs[1].camera),
            dict(scene=2, w=64, h=48, depth=3, M=descs[2].M, camera=descs[2].camera),
            dict(scene=3, w=64, h=48, depth=3, M=descs[3].M, camera=descs[3].camera)]
    imgs, done, st = run_server(gss, reqs, batch_rays=1 << 16, lanes=1)   # 76,800 px > 65,536: alone
    spans = {d["tag"]: (d["admitted_step"], d["completed_step"]) for d in done}
    assert spans[0][0] == 1 and spans[1][0] > 1             # the large one alone first
    assert spans[1][0] == spans[2][0]                       # the small ones together
    check_against_alone(descs, gss, reqs, imgs, st)


def test_paired_steps_equal_separate_steps(scenes):
    """Tracing a step's shadow rays in the next step (one launch with its
    closest-hit rays) gives the images and ray counts of tracing them in the
    step itself; each request then completes exactly one step later."""
    descs, gss = scenes
    reqs = make_requests(descs, 10, seed=19, sizes=[(160, 120), (97, 33), (320, 180)], depths=[1, 3, 6])
    a, da, sa = run_server(gss, reqs, batch_rays=1 << 16, lanes=1)
    b, db, sb = run_server(gss, reqs, batch_rays=1 << 16, flags=rg.RG_SERVER_NO_PAIR, lanes=1)
    for x, y in zip(a, b):
        np.testing.assert_allclose(x, y, atol=ATOL, rtol=0)
    assert sa["closest_rays"] == sb["closest_rays"] and sa["shadow_rays"] == sb["shadow_rays"]
    ca = {d["tag"]: (d["admitted_step"], d["completed_step"]) for d in da}
    cb = {d["tag"]: (d["admitted_step"], d["completed_step"]) for d in db}
    for t in ca:
        assert ca[t][0] == cb[t][0] and ca[t][1] == cb[t][1] + 1, (t, ca[t], cb[t])
    # six kernels per paired step, seven apart (one lane: a server step is a lane step)
    assert sa["lane_steps"] == sa["steps"] and sb["lane_steps"] == sb["steps"]
    assert sa["kernel_launches"] - 6 * sa["lane_steps"] == sb["kernel_launches"] - 7 * sb["lane_steps"]


def test_lanes_run_steps_side_by_side(scenes):
    """Requests spread over four lanes whose steps run at the same time: the
    server books more lane steps than it takes server steps, and every image
    equals its render alone."""
    descs, gss = scenes
    reqs = make_requests(descs, 16, seed=23, sizes=[(320, 240), (640, 360)], depths=[2, 4])
    imgs, done, st = run_server(gss, reqs, batch_rays=1 << 17, lanes=4)
    assert sorted(d["tag"] for d in done) == list(range(len(reqs)))
    assert st["lane_steps"] > st["steps"]
    check_against_alone(descs, gss, reqs, imgs, st)


def test_single_request_completes_after_its_shadow_rays(scenes):
    """A depth-1 request: its rays are traced and shaded in the first step;
    the second step (an otherwise empty ring) traces its shadow rays."""
    descs, gss = scenes
    s = descs[1]
    req = [dict(scene=1, w=64, h=48, depth=1, M=s.M, camera=s.camera)]
    imgs, done, st = run_server(gss, req)
    assert done[0]["admitted_step"] == 1 and done[0]["completed_step"] == 2 and st["steps"] == 2
    check_against_alone(descs, gss, req, imgs, st)


def test_compressed_scene_served_from_its_binary_bvh(scenes):
    """A scene made with RG_SCENE_COMPRESSED is served from its binary float32
    BVH; since the two forms give bit-identical hit records, the served image
    equals rg_render of the compressed scene alone and the ray counts agree."""
    descs, _ = scenes
    desc = descs[1]
    gs = rg.GpuScene(desc, flags=rg.RG_SCENE_COMPRESSED)
    try:
        reqs = [dict(scene=0, w=320, h=180, depth=4, M=g.motion(desc.M, 5), camera=desc.camera)]
        imgs, done, st = run_server([gs], reqs)
        assert len(done) == 1
        check_against_alone([desc], [gs], reqs, imgs, st)
    finally:
        gs.close()
