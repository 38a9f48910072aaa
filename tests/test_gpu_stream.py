"""Out-of-core rendering (spl_render_stream): particles stay in host memory
and pass through the device in chunks, double-buffered on a copy stream.

The image must not depend on the chunking: the additive form is linear in
the particle set (Sec. 2), so a streamed render equals the render of the
loaded set up to FP32 summation order, and both stay within the FP32
tolerance of the FP64 oracle.
"""
import ctypes as C
import os

import numpy as np
import pytest

import oracle
from paper_1309_1114_gb300 import scenes
from tests._metrics import rel_pixel_error
from tests.test_gpu_parity import gpu_render, random_scene

pytestmark = pytest.mark.gpu
TOL32 = 1e-4


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


@pytest.fixture(scope="module")
def rnd(torch_cuda):
    from paper_1309_1114_gb300.splotch import Renderer
    r = Renderer(0)
    yield r
    r.close()


def streamed(r, torch, parts, pal, cam, chunk, fp16=None, pinned=False, h_log2_min=None,
             **params):
    r.set_colormap(pal)
    r.set_params(**params)
    r.set_camera(cam)
    if pinned:
        parts = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in parts.items()}
        if fp16 is not None:
            fp16 = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in fp16.items()}
    img = torch.full((cam["height"], cam["width"], 3), float("nan"), device="cuda")
    r.render_stream(parts, chunk, img, fp16, h_log2_min=h_log2_min)
    torch.cuda.synchronize()
    return img.cpu().numpy().astype(np.float64)


def same(a, b, tol=1e-5):
    M = np.abs(b).reshape(-1, 3).max(0)
    return rel_pixel_error(a, b, M=M) <= tol


@pytest.mark.parametrize("chunk,pinned", [(70_001, True), (50_000, False), (10**9, True)])
def test_stream_equals_loaded_render_and_oracle(rnd, torch_cuda, chunk, pinned):
    sc = scenes.make("uniform", n=200_000, width=256)
    cam = sc.cams[0]
    base = gpu_render(rnd, torch_cuda, sc.parts, sc.palette, cam)
    got = streamed(rnd, torch_cuda, sc.parts, sc.palette, cam, chunk, pinned=pinned)
    assert np.isfinite(got).all()
    assert same(got, base)
    o = oracle.render(sc.parts, sc.palette, cam, {}, nthreads=os.cpu_count() or 1)
    B, _ = oracle.ambiguity(sc.parts, sc.palette, cam)
    assert rel_pixel_error(got, o, B) <= TOL32
    st = rnd.stats()
    assert st["n_particles"] == 200_000
    assert st["n_active"] == int(np.sum(oracle.project(sc.parts, sc.palette, cam)["cls"] >= 0))


def test_stream_with_large_particles_split_tiles_and_ea_map(rnd, torch_cuda):
    # heavy-tailed radii: point, tile and large passes and split tiles in every chunk
    sc = scenes.make("pareto", n=400_000, width=512)
    cam = sc.cams[0]
    for mode in (0, 1):
        base = gpu_render(rnd, torch_cuda, sc.parts, sc.palette, cam, mode=mode)
        got = streamed(rnd, torch_cuda, sc.parts, sc.palette, cam, 123_457, pinned=True, mode=mode)
        assert same(got, base)
        st = rnd.stats()
        assert st["n_large"] > 0 and st["n_point"] > 0
    o = oracle.render(sc.parts, sc.palette, cam, {"mode": 1}, nthreads=os.cpu_count() or 1)
    B, _ = oracle.ambiguity(sc.parts, sc.palette, cam, {"mode": 1})
    assert rel_pixel_error(got, o, B) <= TOL32
    rnd.set_params()


def test_stream_fp16_attributes(rnd, torch_cuda):
    from tests._codes import log16_h
    sc = scenes.make("precision", n=300_000, width=384)
    cam = sc.cams[0]
    half = {k: sc.fp16[k] for k in ("I", "s")}
    logh = dict(half, h=log16_h(sc.parts["h"], -14.0))
    for fp16, lmin in ((sc.fp16, None), (half, None), (logh, -14.0)):
        base = gpu_render(rnd, torch_cuda, sc.parts, sc.palette, cam, fp16=fp16, h_log2_min=lmin)
        got = streamed(rnd, torch_cuda, sc.parts, sc.palette, cam, 99_999, fp16=fp16, pinned=True,
                       h_log2_min=lmin)
        assert same(got, base)


def test_stream_tiny_chunks_and_empty(rnd, torch_cuda):
    parts, cam = random_scene(5, 37, 48, 40)
    pal = scenes.ramp_palette()
    got = streamed(rnd, torch_cuda, parts, pal, cam, 1)            # one particle per chunk
    o = oracle.render(parts, pal, cam, {})
    B, _ = oracle.ambiguity(parts, pal, cam)
    assert rel_pixel_error(got, o, B) <= TOL32
    empty = {k: v[:0] for k, v in parts.items()}
    got = streamed(rnd, torch_cuda, empty, pal, cam, 8)
    assert (got == 0).all()
    got = streamed(rnd, torch_cuda, empty, pal, cam, 8, mode=1)
    assert (got == 0).all()
    rnd.set_params()


def test_stream_rejects_device_particles_and_bad_chunks(rnd, torch_cuda):
    from paper_1309_1114_gb300 import splotch as S
    parts, cam = random_scene(6, 10, 16, 16)
    rnd.set_colormap(scenes.ramp_palette())
    rnd.set_camera(cam)
    img = torch_cuda.zeros((16, 16, 3), device="cuda")
    dev = {k: torch_cuda.from_numpy(v).cuda() for k, v in parts.items()}
    with pytest.raises(S.SplotchError):
        rnd.render_stream(dev, 4, img)
    with pytest.raises(S.SplotchError):
        rnd.render_stream(parts, 0, img)
    # the context's own particles are untouched: render() still sees the loaded set
    base = gpu_render(rnd, torch_cuda, parts, scenes.ramp_palette(), cam)
    streamed(rnd, torch_cuda, {k: v[:3] for k, v in parts.items()}, scenes.ramp_palette(), cam, 2)
    again = img.clone()
    rnd.render(again)
    torch_cuda.cuda.synchronize()
    assert same(again.cpu().numpy().astype(np.float64), base)
