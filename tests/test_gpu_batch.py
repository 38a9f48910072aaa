"""Batched rendering: many views in one persistent, graph-captured launch.

A batch renders the same particle set for several cameras and resolutions;
every view must equal the single-view render of the same camera (GPU vs GPU,
1e-5) and the FP64 oracle (1e-4).  The second call with the same
configuration replays a captured CUDA graph, also after the cameras moved.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1309_1114_gb300 import scenes
from tests._metrics import pick_pixels, rel_pixel_error
from tests.test_gpu_parity import gpu_render

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


def small_orbit(n_views=7, az0=0.0, step=51.0):
    sizes = [(160, 120), (96, 96), (201, 77), (64, 64), (128, 160), (33, 47), (250, 250)]
    cams = []
    for k in range(n_views):
        w, h = sizes[k % len(sizes)]
        cams.append(scenes.camera(w, h, azimuth_deg=az0 + k * step))
    return cams


def batch_render(r, torch, cams, **params):
    if params:
        r.set_params(**params)
    imgs = [torch.full((c["height"], c["width"], 3), float("nan"), device="cuda") for c in cams]
    r.render_batch(cams, imgs)
    torch.cuda.synchronize()
    return [im.cpu().numpy().astype(np.float64) for im in imgs]


@pytest.fixture(scope="module")
def scene():
    return scenes.make("clustered", n=200_000)


def test_batch_equals_single_views_and_oracle(rnd, torch_cuda, scene):
    cams = small_orbit()
    rnd.load(scene.parts)
    rnd.set_colormap(scene.palette)
    rnd.set_params()
    got = batch_render(rnd, torch_cuda, cams)
    nt = os.cpu_count() or 1
    for cam, g in zip(cams, got):
        assert np.isfinite(g).all()
        single = gpu_render(rnd, torch_cuda, scene.parts, scene.palette, cam)
        M = np.abs(single).reshape(-1, 3).max(0)
        assert rel_pixel_error(g, single, M=M) < 1e-5
        o = oracle.render(scene.parts, scene.palette, cam, {}, nthreads=nt)
        B, _ = oracle.ambiguity(scene.parts, scene.palette, cam)
        assert rel_pixel_error(g, o, B) <= TOL32


@pytest.mark.parametrize("tile", [16, 32, 64])
def test_graph_replay_and_moved_cameras(rnd, torch_cuda, scene, tile):
    rnd.load(scene.parts)
    rnd.set_colormap(scene.palette)
    cams = small_orbit(5)
    first = batch_render(rnd, torch_cuda, cams, tile_px=tile)     # eager + capture
    again = batch_render(rnd, torch_cuda, cams)                   # replay
    for a, b in zip(first, again):
        M = np.abs(a).reshape(-1, 3).max(0)
        assert rel_pixel_error(b, a, M=M) < 1e-5
    moved = small_orbit(5, az0=13.0)                              # same sizes: replay
    got = batch_render(rnd, torch_cuda, moved)
    for cam, g in zip(moved, got):
        single = gpu_render(rnd, torch_cuda, scene.parts, scene.palette, cam, tile_px=tile)
        M = np.abs(single).reshape(-1, 3).max(0)
        assert rel_pixel_error(g, single, M=M) < 1e-5
    rnd.set_params()


def test_graph_replay_survives_list_growth(rnd, torch_cuda):
    # the replayed lists outgrow the captured capacity: detected, re-rendered
    p_small = scenes.make("uniform", n=20_000).parts
    big = scenes.make("uniform", n=20_000).parts
    big = dict(big, h=(big["h"] * np.float32(6.0)))
    cams = small_orbit(3)
    rnd.load(p_small)
    rnd.set_colormap(scenes.ramp_palette())
    batch_render(rnd, torch_cuda, cams)
    rnd.load(big)                                    # same n, far larger discs
    got = batch_render(rnd, torch_cuda, cams)
    for cam, g in zip(cams, got):
        o = oracle.render(big, scenes.ramp_palette(), cam, {}, nthreads=os.cpu_count() or 1)
        B, _ = oracle.ambiguity(big, scenes.ramp_palette(), cam)
        assert rel_pixel_error(g, o, B) <= TOL32


def test_autotune_picks_valid_parameters(rnd, torch_cuda, scene):
    rnd.load(scene.parts)
    rnd.set_colormap(scene.palette)
    rnd.set_params()
    cams = small_orbit(4)
    imgs = [torch_cuda.empty((c["height"], c["width"], 3), device="cuda") for c in cams]
    best, ms = rnd.autotune(cams, imgs, reps=1)
    assert best["tile_px"] in (16, 32, 64) and ms > 0
    assert best["r_large"] >= best["r_small"] >= best["r_sml"]
    got = batch_render(rnd, torch_cuda, cams)       # with the tuned parameters
    for cam, g in zip(cams, got):
        o = oracle.render(scene.parts, scene.palette, cam, {}, nthreads=os.cpu_count() or 1)
        B, _ = oracle.ambiguity(scene.parts, scene.palette, cam)
        assert rel_pixel_error(g, o, B) <= TOL32
    rnd.set_params()


def test_orbit_full_size_sampled(rnd, torch_cuda):
    """20M clustered particles, 64 views (512/1024/2048), >= 1024 sampled pixels
    (whole tile-corner windows, the brightest and random pixels) of 4 views."""
    sc = scenes.make("orbit")
    rnd.load(sc.parts)
    rnd.set_colormap(sc.palette)
    rnd.set_params()
    got = batch_render(rnd, torch_cuda, sc.cams)
    for v in (0, 17, 34, 63):
        cam, g = sc.cams[v], got[v]
        assert np.isfinite(g).all()
        px, py = pick_pixels(g, n_windows=1, n_bright=64, n_random=256, seed=v)
        assert px.size >= 1024
        o = oracle.render_pixels(sc.parts, sc.palette, cam, {}, px, py, nthreads=os.cpu_count() or 1)
        M = np.abs(g).reshape(-1, 3).max(0)
        assert rel_pixel_error(g[py, px], o, M=M) <= TOL32
