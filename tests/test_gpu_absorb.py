"""GPU parity of the general absorption form (Eq. 1 with E_p != A_p): the CUDA
path (radix-sorted tile lists, front-to-back compositing, composition of
split tiles) against the FP64 oracle's mode 2, within the FP32 tolerance
after the oracle's ambiguity mass."""
import ctypes as C
import os

import numpy as np
import pytest

import oracle
from paper_1309_1114_gb300 import scenes
from tests._metrics import rel_pixel_error
from tests.test_gpu_parity import gpu_render, random_scene, sampled_check

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


def check(r, torch, parts, pal, cam, alpha, tol=TOL32, **params):
    g = gpu_render(r, torch, parts, pal, cam, mode=2, absorption=alpha, **params)
    q = {"mode": 2, "absorption": alpha}
    o = oracle.render(parts, pal, cam, q)
    B, _ = oracle.ambiguity(parts, pal, cam, q)
    assert np.isfinite(g).all()
    err = rel_pixel_error(g, o, B)
    assert err <= tol, f"max relative pixel error {err:.3e}"
    return g, o


@pytest.mark.parametrize("tile", [16, 32, 64])
@pytest.mark.parametrize("alpha", [0.3, 2.5])
def test_random_scenes_with_points(rnd, torch_cuda, tile, alpha):
    parts, cam = random_scene(11, 3000, 200, 150)
    rec = oracle.project(parts, scenes.ramp_palette(), cam)
    assert (rec["cls"] == 0).any() and (rec["cls"] == 1).any()
    check(rnd, torch_cuda, parts, scenes.ramp_palette(), cam, alpha, tile_px=tile)


@pytest.mark.parametrize("alpha", [0.5, 4.0])
def test_uniform_scene(rnd, torch_cuda, alpha):
    sc = scenes.make("uniform", n=200_000, width=256)
    check(rnd, torch_cuda, sc.parts, sc.palette, sc.cams[0], alpha)


def test_crowded_tiles_are_split_and_composed(rnd, torch_cuda):
    # halo cores put thousands of particles into a tile: several items per
    # tile, whose (C, T) partials are composed in depth order
    sc = scenes.make("clustered", n=300_000, width=384)
    cam = sc.cams[0]
    check(rnd, torch_cuda, sc.parts, sc.palette, cam, 1.5)
    st = rnd.stats()
    assert st["n_entries"][2] > 1024 * 50


def test_heavy_tailed_radii(rnd, torch_cuda):
    sc = scenes.make("pareto", n=150_000, width=384)
    check(rnd, torch_cuda, sc.parts, sc.palette, sc.cams[0], 0.8)


def test_clustered_full_size_sampled(rnd, torch_cuda):
    """The timed absorbing workload (10M clustered particles, 1024^2) at >= 1024
    sampled pixels, each pixel's particles sorted by FP64 depth by the oracle;
    the ambiguity mass covers near ties in depth."""
    sc = scenes.make("clustered")
    g, err = sampled_check(rnd, torch_cuda, sc, sc.cams[0], with_mass=True, mode=2,
                           absorption=1.0)
    assert err <= TOL32, err


def test_emission_equal_to_absorption_matches_the_ea_mode(rnd, torch_cuda):
    sc = scenes.make("uniform", n=100_000, width=192)
    cam = sc.cams[0]
    pal = np.full((1, 3), 0.75, dtype=np.float32)
    g = gpu_render(rnd, torch_cuda, sc.parts, pal, cam, mode=2, absorption=0.75)
    ea = gpu_render(rnd, torch_cuda, sc.parts, pal, cam, mode=1)
    M = np.abs(ea).reshape(-1, 3).max(0)
    assert rel_pixel_error(g, ea, M=M) <= 1e-5


def test_input_order_does_not_change_the_image(rnd, torch_cuda):
    sc = scenes.make("clustered", n=200_000, width=256)
    cam = sc.cams[0]
    base = gpu_render(rnd, torch_cuda, sc.parts, sc.palette, cam, mode=2, absorption=1.0)
    perm = np.random.default_rng(3).permutation(200_000)
    got = gpu_render(rnd, torch_cuda, {k: v[perm] for k, v in sc.parts.items()}, sc.palette, cam,
                     mode=2, absorption=1.0)
    M = np.abs(base).reshape(-1, 3).max(0)
    assert rel_pixel_error(got, base, M=M) <= 1e-6
    # a different order of the depths does change it
    flip = dict(sc.parts)
    flip["z"] = (1.0 - sc.parts["z"]).astype(np.float32)
    other = gpu_render(rnd, torch_cuda, flip, sc.palette, cam, mode=2, absorption=1.0)
    assert np.abs(other - base).max() > 1e-3


def test_absorption_mode_is_single_view_only(rnd, torch_cuda):
    from paper_1309_1114_gb300 import splotch as S
    parts, cam = random_scene(2, 50, 32, 32)
    rnd.load(parts)
    rnd.set_colormap(scenes.ramp_palette())
    rnd.set_camera(cam)
    rnd.set_params(mode=2, absorption=1.0)
    img = torch_cuda.zeros((32, 32, 3), device="cuda")
    with pytest.raises(S.SplotchError):
        rnd.render_batch([cam], [img])
    with pytest.raises(S.SplotchError):
        rnd.render_stream(parts, 10, img)
    for bad in (0.0, -1.0, float("nan")):
        with pytest.raises(S.SplotchError):
            rnd.set_params(mode=2, absorption=bad)
    rnd.set_params()
