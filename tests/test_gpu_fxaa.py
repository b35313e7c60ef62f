"""FXAA on the GPU against the oracle's float32 restatement: bit for bit (both
sides take every threshold decision in float32 with the same operation
order), on hand-pinned edge images, random images, tiny and ragged sizes,
and rendered frames."""
import numpy as np
import pytest
import torch

import oracle
import paper_2001_09792_gb300 as rg
import scenegen as g
from test_oracle_fxaa import block_image

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("librg")]


def gpu_fxaa(img):
    d = torch.from_numpy(np.ascontiguousarray(img, np.float32)).cuda()
    out = rg.rg_fxaa(d)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def assert_bitwise(a, b):
    bad = a.view(np.uint32) != b.view(np.uint32)
    assert not bad.any(), f"{bad.any(-1).sum()} pixels differ, first at {np.argwhere(bad)[:3].tolist()}"


def test_pinned_edge_images():
    img = block_image()
    assert_bitwise(gpu_fxaa(img), oracle.fxaa(img))
    t = np.ascontiguousarray(img.transpose(1, 0, 2))
    assert_bitwise(gpu_fxaa(t), oracle.fxaa(t))
    v = np.zeros((64, 16, 4), np.float32)
    v[:, 8:, :3] = 1
    assert_bitwise(gpu_fxaa(v), oracle.fxaa(v))


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (7, 1), (2, 2), (33, 97), (16, 16), (17, 15)])
def test_random_images(shape):
    rng = np.random.default_rng(shape[0] * 1000 + shape[1])
    img = rng.uniform(0, 1.5, (*shape, 4)).astype(np.float32)
    # sparse steps on a smooth ramp as well: many pixels below and above the threshold
    ramp = np.linspace(0, 1, shape[0] * shape[1], dtype=np.float32).reshape(shape)
    img2 = np.repeat(ramp[..., None], 4, -1) + (rng.uniform(0, 1, (*shape, 1)) < 0.1) * np.float32(0.5)
    assert_bitwise(gpu_fxaa(img), oracle.fxaa(img))
    assert_bitwise(gpu_fxaa(img2.astype(np.float32)), oracle.fxaa(img2.astype(np.float32)))


@pytest.mark.parametrize("which", ["tiny", "medium"])
def test_rendered_frames(which):
    s = g.tiny_scene() if which == "tiny" else g.medium_scene()
    with rg.GpuScene(s) as gs:
        img = rg.rg_render(gs.h, s.camera, s.width, s.height, s.max_depth)
        out = rg.rg_fxaa(img)
        torch.cuda.synchronize()
        host = img.cpu().numpy()
        got = out.cpu().numpy()
    ref = oracle.fxaa(host)
    assert_bitwise(got, ref)
    changed = np.any(got != host, axis=-1).mean()
    assert 0.001 < changed < 0.5     # edges are smoothed, flat regions kept


def test_rejects_aliasing_and_accepts_empty():
    img = torch.zeros((4, 4, 4), device="cuda")
    L = rg.lib()
    import ctypes
    p = ctypes.c_void_p(img.data_ptr())
    assert L.rg_fxaa(p, 4, 4, p, None) == rg.RG_ERR_INVALID_ARG
    assert L.rg_fxaa(p, 0, 4, None, None) == rg.RG_OK
