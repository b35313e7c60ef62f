"""Large incoherent ray queries at full size: 4,096 instances of 16 meshes
(1,938,944 unique triangles, about 60M instanced), a full TLAS rebuild after
seeded motion, then 16,777,216 closest-hit rays and 16,777,216 any-hit rays
each traced in one launch, on binned-SAH BLAS and TLAS as the benchmark
builds them.
The oracle checks a seeded sample of each set."""
import numpy as np
import pytest
import torch

import oracle
import paper_2001_09792_gb300 as rg
import scenegen as g
from test_gpu_trace import KAPPA, MAX_EXEMPT, MISS, REL_T, compare_closest

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("librg")]
N_RAYS = 1 << 24
SAMPLE = 20_000


@pytest.fixture(scope="module")
def large():
    s = g.large_scene()
    assert sum(m[1].shape[0] for m in s.meshes) == 1_938_944
    assert s.n_instances == 4096
    gs = rg.GpuScene(s, flags=rg.RG_SCENE_SAH_TLAS, morton_flags=rg.RG_BLAS_SAH)   # the builds the benchmark times
    M1 = g.motion(s.M, 1)
    host = gs.inst_host.copy()
    host[:, :12] = M1.reshape(-1, 12)
    rg.rg_tlas_build(gs.h, torch.from_numpy(host).cuda())   # full rebuild for frame 1
    rg.rg_sync(gs.h)
    s.M = M1
    O = oracle.OracleScene(s)
    yield s, gs, O
    gs.close()


def test_large_closest_hit_full_launch(large):
    s, gs, O = large
    closest, _ = g.large_rays(s, N_RAYS)
    d_rays = torch.from_numpy(closest).cuda()
    hits = rg.rg_trace_rays(gs.h, d_rays)
    rg.rg_sync(gs.h)
    idx = np.random.default_rng(5).choice(N_RAYS, SAMPLE, replace=False)
    h = rg.split_hits(hits[torch.from_numpy(idx).cuda()])
    ref = O.trace(closest[idx], kappa=KAPPA, rel_t=REL_T)
    frac = compare_closest(h, ref, label="large")
    assert (ref["inst"] != MISS).mean() > 0.3
    print(f"large closest: {frac:.2e} differ, {ref['ambiguous'].mean():.2e} ambiguous")


def test_large_any_hit_full_launch(large):
    s, gs, O = large
    _, anyhit = g.large_rays(s, N_RAYS)
    hits = rg.rg_trace_rays(gs.h, torch.from_numpy(anyhit).cuda(), rg.RG_ANY)
    rg.rg_sync(gs.h)
    idx = np.random.default_rng(6).choice(N_RAYS, SAMPLE, replace=False)
    h = rg.split_hits(hits[torch.from_numpy(idx).cuda()])
    ref = O.trace(anyhit[idx], any_hit=True, kappa=KAPPA, rel_t=REL_T)
    occ = h["inst"] != MISS
    ok = ~ref["ambiguous"]
    assert np.array_equal(occ[ok], ref["occluded"][ok])
    assert (occ != ref["occluded"]).mean() <= MAX_EXEMPT
    assert 0.02 < ref["occluded"].mean() < 0.98
