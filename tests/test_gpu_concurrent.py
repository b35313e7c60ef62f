"""Concurrent rg_trace_rays calls on one scene (each call takes a work counter
of its own): closest-hit and any-hit queries issued on several streams at the
same time give records bit-identical to the same calls made one after the
other, and a TLAS rebuild ordered after them by events is seen by the next
calls."""
import numpy as np
import pytest
import torch

import paper_2001_09792_gb300 as rg
import scenegen as g
from test_gpu_trace import _random_scene

pytestmark = pytest.mark.gpu


def _rays(s, n, seed):
    lo, hi = s.world_aabb()
    return torch.from_numpy(np.ascontiguousarray(g.random_rays(n, lo - 5, hi + 5, seed=seed), np.float32)).cuda()


def test_calls_on_several_streams_match_serial_calls():
    s = _random_scene(81, 700)
    sets = [(_rays(s, 150_000 + 977 * k, 90 + k), rg.RG_ANY if k % 3 == 2 else rg.RG_CLOSEST) for k in range(12)]
    with rg.GpuScene(s, flags=rg.RG_SCENE_SAH_TLAS) as gs:
        ref = []
        for rays, flags in sets:
            ref.append(rg.rg_trace_rays(gs.h, rays, flags).clone())
        torch.cuda.synchronize()
        streams = [torch.cuda.Stream() for _ in range(4)]
        start = torch.cuda.Event()
        start.record()
        outs = []
        for k, (rays, flags) in enumerate(sets):
            st = streams[k % len(streams)]
            st.wait_event(start)
            hits = torch.empty((rays.shape[0], 5), dtype=torch.int32, device="cuda")
            rg.rg_trace_rays(gs.h, rays, flags, hits, stream=st)
            outs.append(hits)
        for st in streams:
            torch.cuda.current_stream().wait_stream(st)
        torch.cuda.synchronize()
        rg.rg_sync(gs.h)
        for k, (a, b) in enumerate(zip(ref, outs)):
            assert torch.equal(a, b), f"call {k} differs"
        assert any((h[:, 0] != -1).any() for h in outs)


def test_rebuild_between_concurrent_steps():
    """Two steps of (TLAS rebuild; closest-hit and any-hit on two streams),
    the rebuild of the second waiting for both queries of the first: each
    step answers like the same calls made serially on its transforms."""
    s = _random_scene(82, 500)
    closest, anyhit = _rays(s, 120_000, 83), _rays(s, 110_000, 84)
    M2 = g.motion(s.M, 5)
    with rg.GpuScene(s, flags=rg.RG_SCENE_SAH_TLAS) as gs:
        blas = [gs.blas[m] for m in s.mesh_id]
        insts = [torch.from_numpy(rg.pack_instances(M, blas, s.material_id)).cuda() for M in (s.M, M2)]
        serial = []
        for inst in insts:
            rg.rg_tlas_build(gs.h, inst)
            serial.append((rg.rg_trace_rays(gs.h, closest, rg.RG_CLOSEST).clone(),
                           rg.rg_trace_rays(gs.h, anyhit, rg.RG_ANY).clone()))
        torch.cuda.synchronize()
        main, side = torch.cuda.current_stream(), torch.cuda.Stream()
        got = []
        for inst in insts:
            rg.rg_tlas_build(gs.h, inst)
            built = torch.cuda.Event()
            built.record(main)
            side.wait_event(built)
            hc = rg.rg_trace_rays(gs.h, closest, rg.RG_CLOSEST)
            ha = torch.empty((anyhit.shape[0], 5), dtype=torch.int32, device="cuda")
            rg.rg_trace_rays(gs.h, anyhit, rg.RG_ANY, ha, stream=side)
            done = torch.cuda.Event()
            done.record(side)
            main.wait_event(done)
            got.append((hc, ha))
        torch.cuda.synchronize()
        rg.rg_sync(gs.h)
        for k, ((c0, a0), (c1, a1)) in enumerate(zip(serial, got)):
            assert torch.equal(c0, c1), f"step {k}: closest-hit records differ"
            assert torch.equal(a0, a1), f"step {k}: any-hit records differ"
        assert not torch.equal(serial[0][0], serial[1][0])  # the motion changed the answers
