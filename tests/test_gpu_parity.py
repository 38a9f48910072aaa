"""GPU parity: the CUDA path, called through the C ABI, against the FP64 oracle.

Tolerance: the FP32 path must stay within 1e-4 of the oracle under the error
metric of tests/_metrics.py (per-pixel relative error with a floor of 1e-3 of
the channel maximum, after subtracting the oracle's ambiguity mass).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1309_1114_gb300 import scenes
from tests._metrics import pick_pixels, rel_pixel_error

pytestmark = pytest.mark.gpu
TOL32 = 1e-4
HERE = os.path.dirname(os.path.abspath(__file__))


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


def gpu_render(r, torch, parts, pal, cam, fp16=None, h_log2_min=None, **params):
    r.load(parts, fp16, h_log2_min)
    r.set_colormap(pal)
    r.set_params(**params)
    r.set_camera(cam)
    img = torch.full((cam["height"], cam["width"], 3), float("nan"), device="cuda",
                     dtype=torch.float32)
    r.render(img)
    torch.cuda.synchronize()
    return img.cpu().numpy().astype(np.float64)


def oracle_params(params):
    keys = ("chi", "sigma_per_h", "s_box", "r_sml", "brightness", "mode", "absorption")
    return {k: v for k, v in params.items() if k in keys}


def check_image(r, torch, parts, pal, cam, tol=TOL32, **params):
    g = gpu_render(r, torch, parts, pal, cam, **params)
    op = oracle_params(params)
    o = oracle.render(parts, pal, cam, op, nthreads=os.cpu_count() or 1)
    B, _ = oracle.ambiguity(parts, pal, cam, op)
    assert np.isfinite(g).all()
    err = rel_pixel_error(g, o, B)
    assert err <= tol, f"max relative pixel error {err:.3e}"
    return g, o, err


def parts_of(rows):
    rows = np.asarray(rows, dtype=np.float64).reshape(-1, 6)
    return {k: rows[:, i].astype(np.float32) for i, k in enumerate(("x", "y", "z", "h", "I", "s"))}


def random_scene(seed, n, w, h, hmin=-7.0, hmax=-1.5, spread=0.3):
    rng = np.random.default_rng(seed)
    rows = np.column_stack([rng.uniform(-spread, 1 + spread, n), rng.uniform(-spread, 1 + spread, n),
                            rng.uniform(-1.3, 1.0, n), np.exp(rng.uniform(hmin, hmax, n)),
                            rng.random(n), rng.random(n)])
    cam = {"eye": (0.5, 0.5, -1.5), "target": (0.5, 0.5, 0.5), "up": (0.0, 1.0, 0.0),
           "fov_y_deg": 60.0, "width": w, "height": h, "z_near": 1e-3}
    return parts_of(rows), cam


# ------------------------------------------------------------- rasteriser
def test_raster_records_match_oracle(rnd, torch_cuda):
    sc = scenes.make("uniform", n=50000, width=256)
    cam = sc.cams[0]
    gpu_render(rnd, torch_cuda, sc.parts, sc.palette, cam)
    g = rnd.records(sc.n)
    o = oracle.project(sc.parts, sc.palette, cam)
    act = o["cls"] >= 0
    gcls = np.where(g["cls"] >= 0, np.minimum(g["cls"], 1), g["cls"])
    # class labels agree except within rounding of a threshold
    near = np.abs(o["r"] - 0.5) < 1e-5
    assert np.all((gcls == o["cls"]) | near)
    m = act & (g["cls"] >= 0)
    assert np.max(np.abs(g["xs"][m] - o["xs"][m])) < 2e-6
    assert np.max(np.abs(g["ys"][m] - o["ys"][m])) < 2e-6
    np.testing.assert_allclose(g["r"][m], o["r"][m], rtol=2e-6)
    np.testing.assert_allclose(g["e"][m], o["e"][m], rtol=2e-6, atol=1e-7)
    st = rnd.stats()
    assert st["n_active"] == int(np.sum(g["cls"] >= 0))


def test_stats_count_classes(rnd, torch_cuda):
    p, cam = random_scene(3, 3000, 200, 150, hmin=-8, hmax=-1)
    gpu_render(rnd, torch_cuda, p, scenes.ramp_palette(), cam, r_small=3.0, r_large=20.0)
    st = rnd.stats()
    g = rnd.records(3000)
    assert st["n_point"] == np.sum(g["cls"] == 0) > 0
    assert st["n_small"] == np.sum(g["cls"] == 1) > 0
    assert st["n_medium"] == np.sum(g["cls"] == 2) > 0
    assert st["n_large"] == np.sum(g["cls"] == 3) > 0
    assert st["n_active"] == st["n_point"] + st["n_small"] + st["n_medium"] + st["n_large"]


# ------------------------------------------------------------- full images
def test_golden_five_particles(rnd, torch_cuda):
    d = json.load(open(os.path.join(HERE, "golden", "five_particles.json")))
    rows = np.asarray(d["rows_xyzhIs"], dtype=np.float32)
    parts = {k: rows[:, i] for i, k in enumerate(("x", "y", "z", "h", "I", "s"))}
    pal = np.asarray(d["palette"], np.float32)
    g = gpu_render(rnd, torch_cuda, parts, pal, d["camera"])
    o = np.asarray(d["image"])
    B, _ = oracle.ambiguity(parts, pal, d["camera"])
    assert rel_pixel_error(g, o, B) <= TOL32


def test_uniform_scene_full_image(rnd, torch_cuda):
    sc = scenes.make("uniform")          # 200k particles, 256^2
    check_image(rnd, torch_cuda, sc.parts, sc.palette, sc.cams[0])


@pytest.mark.parametrize("seed,w,h", [(0, 37, 29), (1, 100, 61), (2, 129, 130), (3, 257, 96)])
def test_random_scenes_ragged_sizes(rnd, torch_cuda, seed, w, h):
    p, cam = random_scene(seed, 4000, w, h)
    check_image(rnd, torch_cuda, p, scenes.ramp_palette(), cam)


@pytest.mark.parametrize("tile", [16, 32, 64])
@pytest.mark.parametrize("r_small,r_large", [(0.5, 0.5), (4.0, 64.0), (1e6, 1e6), (2.0, 8.0)])
def test_thresholds_and_tile_size_do_not_change_the_image(rnd, torch_cuda, tile, r_small, r_large):
    # r_small / r_large / tile only choose how a particle is processed
    p, cam = random_scene(5, 3000, 150, 110, hmin=-8, hmax=-1.2)
    check_image(rnd, torch_cuda, p, scenes.ramp_palette(), cam, tile_px=tile, r_small=r_small,
                r_large=r_large)


def test_permutation_invariance(rnd, torch_cuda):
    p, cam = random_scene(9, 5000, 128, 128)
    pal = scenes.ramp_palette()
    a = gpu_render(rnd, torch_cuda, p, pal, cam)
    perm = np.random.default_rng(1).permutation(5000)
    b = gpu_render(rnd, torch_cuda, {k: v[perm] for k, v in p.items()}, pal, cam)
    M = np.abs(a).reshape(-1, 3).max(0)
    assert rel_pixel_error(b, a, M=M) < 1e-5


# ----------------------------------------------------- one class at a time
def test_point_particles_only(rnd, torch_cuda):
    rng = np.random.default_rng(4)
    n = 20000
    p, cam = random_scene(4, n, 96, 80, hmin=-12, hmax=-9)
    g, o, _ = check_image(rnd, torch_cuda, p, scenes.ramp_palette(), cam)
    assert rnd.stats()["n_point"] == rnd.stats()["n_active"]


def test_single_huge_splat_covers_image(rnd, torch_cuda):
    p = parts_of([0.5, 0.5, 0.5, 0.8, 1.0, 0.5])
    cam = scenes.camera(300, 200)
    g, o, _ = check_image(rnd, torch_cuda, p, scenes.ramp_palette(), cam)
    assert rnd.stats()["n_large"] == 1
    assert np.all(o[..., 0] > 0)   # the disc covers every pixel centre


def test_near_plane_and_off_screen_centres(rnd, torch_cuda):
    rows = [[0.5, 0.5, -1.4989, 0.001, 1.0, 0.2],   # just past the near plane: huge
            [0.5, 0.5, -1.6, 0.01, 1.0, 0.2],       # behind the eye
            [-0.9, 0.5, 0.0, 0.12, 1.0, 0.7],       # centre off screen, disc reaches in
            [0.5, 2.2, 0.0, 0.2, 1.0, 0.9],
            [0.51, 0.49, 0.3, 0.004, 1.0, 0.4]]
    cam = dict(scenes.camera(160, 120), z_near=1e-3)
    check_image(rnd, torch_cuda, parts_of(rows), scenes.ramp_palette(), cam)


def test_empty_and_tiny_particle_counts(rnd, torch_cuda):
    pal = scenes.ramp_palette()
    cam = scenes.camera(64, 48)
    empty = {k: np.zeros(0, np.float32) for k in ("x", "y", "z", "h", "I", "s")}
    g = gpu_render(rnd, torch_cuda, empty, pal, cam)
    assert np.all(g == 0.0)
    for n in (1, 3, 31, 33, 257):
        p, cam = random_scene(100 + n, n, 70, 50, hmin=-4, hmax=-2)
        check_image(rnd, torch_cuda, p, pal, cam)


def test_absorption_mode(rnd, torch_cuda):
    p, cam = random_scene(12, 3000, 120, 90)
    check_image(rnd, torch_cuda, p, scenes.ramp_palette(), cam, mode=1)


def test_render_host_equals_device(rnd, torch_cuda):
    p, cam = random_scene(13, 2000, 90, 70)
    g = gpu_render(rnd, torch_cuda, p, scenes.ramp_palette(), cam)
    h = rnd.render_host()
    # tile lists are filled with atomics, so the summation order (and the last
    # bits) can differ between two renders of the same frame
    M = np.abs(g).reshape(-1, 3).max(0)
    assert rel_pixel_error(h, g, M=M) < 1e-5


# ------------------------------------------------ clustered, larger sizes
def test_clustered_reduced_full_image(rnd, torch_cuda):
    sc = scenes.make("clustered", n=300_000, width=384)
    check_image(rnd, torch_cuda, sc.parts, sc.palette, sc.cams[0])


def sampled_check(r, torch, sc, cam, fp16=None, parts_oracle=None, h_log2_min=None,
                  n_windows=2, n_bright=64, n_random=448, with_mass=False, **params):
    """Full-size render, compared at sampled pixels computed one by one by the
    oracle: whole tile-corner windows (one at the brightest halo core), the
    brightest pixels and random pixels (tests/_metrics.pick_pixels), at least
    1024 in all.  with_mass subtracts the oracle's ambiguity mass (needed in
    mode 2, where particles closer in depth than an FP32 ulp may swap)."""
    g = gpu_render(r, torch, sc.parts, sc.palette, cam, fp16=fp16, h_log2_min=h_log2_min, **params)
    px, py = pick_pixels(g, tile=params.get("tile_px", 32), n_windows=n_windows,
                         n_bright=n_bright, n_random=n_random)
    assert px.size >= 1024
    src = sc.parts if parts_oracle is None else parts_oracle
    nt = os.cpu_count() or 1
    B = None
    if with_mass:
        o, B = oracle.render_pixels(src, sc.palette, cam, oracle_params(params), px, py,
                                    nthreads=nt, with_mass=True)
    else:
        o = oracle.render_pixels(src, sc.palette, cam, oracle_params(params), px, py, nthreads=nt)
    M = np.abs(g).reshape(-1, 3).max(0)
    err = rel_pixel_error(g[py, px], o, B, M=M)
    return g, err


def test_clustered_full_size_sampled(rnd, torch_cuda):
    sc = scenes.make("clustered")        # 10M particles, 1024^2
    g, err = sampled_check(rnd, torch_cuda, sc, sc.cams[0])
    assert err <= TOL32, err
    st = rnd.stats()
    assert st["n_active"] > 0.9 * sc.n


@pytest.mark.parametrize("w,h,tile", [(16384, 48, 32), (40, 16384, 64), (16384, 16384, 16)])
def test_extreme_image_sides(rnd, torch_cuda, w, h, tile):
    # the largest side the camera accepts and extreme aspect ratios: pixel and
    # tile indices far from the origin, ragged last tiles; a few thousand
    # particles keep the oracle quick
    parts, cam = random_scene(31 + w % 7, 4000, w, h, hmin=-9.0, hmax=-4.0)
    if w * h > 64_000_000:
        # the full 16384^2 image: compare sampled pixels and check the rest is finite
        g = gpu_render(rnd, torch_cuda, parts, scenes.ramp_palette(), cam, tile_px=tile)
        assert np.isfinite(g).all()
        ys, xs = np.nonzero(g[..., 0] > 0)
        rng = np.random.default_rng(0)
        pick = rng.choice(len(xs), min(256, len(xs)), replace=False)
        px, py = xs[pick].astype(np.int32), ys[pick].astype(np.int32)
        o = oracle.render_pixels(parts, scenes.ramp_palette(), cam, {}, px, py,
                                 nthreads=os.cpu_count() or 1)
        M = np.abs(g).reshape(-1, 3).max(0)
        assert rel_pixel_error(g[py, px], o, M=M) <= TOL32
        return
    check_image(rnd, torch_cuda, parts, scenes.ramp_palette(), cam, tile_px=tile)
