"""GPU parity of the colouring options (Sec. 2): per-particle colour
components in place of the palette, and logarithms of I and of s before
normalisation, against the FP64 oracle -- through the resident, streamed,
batched, allocation-free and absorbing paths."""
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


def coloured(parts, seed=0):
    rng = np.random.default_rng(seed)
    n = len(parts["x"])
    q = dict(parts)
    for k in ("cr", "cg", "cb"):
        q[k] = rng.random(n).astype(np.float32)
    return q


def check(r, torch, parts, pal, cam, oracle_par=None, tol=TOL32, **params):
    g = gpu_render(r, torch, parts, pal, cam, **params)
    op = dict(oracle_par or {})
    o = oracle.render(parts, pal, cam, op, nthreads=os.cpu_count() or 1)
    B, _ = oracle.ambiguity(parts, pal, cam, op)
    assert np.isfinite(g).all()
    err = rel_pixel_error(g, o, B)
    assert err <= tol, f"max relative pixel error {err:.3e}"
    return g


@pytest.mark.parametrize("tile", [16, 32, 64])
def test_colour_components(rnd, torch_cuda, tile):
    parts, cam = random_scene(21, 3000, 160, 128)
    check(rnd, torch_cuda, coloured(parts), scenes.ramp_palette(), cam, tile_px=tile)


def test_colour_components_uniform_scene_and_modes(rnd, torch_cuda):
    sc = scenes.make("uniform", n=200_000, width=256)
    p = coloured(sc.parts, 1)
    check(rnd, torch_cuda, p, sc.palette, sc.cams[0])
    check(rnd, torch_cuda, p, sc.palette, sc.cams[0], {"mode": 1}, mode=1)
    check(rnd, torch_cuda, p, sc.palette, sc.cams[0], {"mode": 2, "absorption": 1.5}, mode=2,
          absorption=1.5)


@pytest.mark.parametrize("flags", [1, 2, 3])
def test_logarithms(rnd, torch_cuda, flags):
    sc = scenes.make("uniform", n=200_000, width=256)
    p = dict(sc.parts)
    p["s"] = (10.0 ** (3.0 * p["s"])).astype(np.float32)        # log10(s) in [0, 3]
    p["I"] = (10.0 ** (1.0 + p["I"])).astype(np.float32)        # log10(I) in [1, 2]
    p["I"][::97] = 0.0                                            # inactive under the log
    rnd.set_colormap(sc.palette, 0.0, 3.0)
    g = None
    rnd.load(p)
    rnd.set_params(log_flags=flags)
    rnd.set_camera(sc.cams[0])
    cam = sc.cams[0]
    img = torch_cuda.empty((cam["height"], cam["width"], 3), device="cuda")
    rnd.render(img)
    torch_cuda.cuda.synchronize()
    g = img.cpu().numpy().astype(np.float64)
    q = {"log": flags, "s_min": 0.0, "s_max": 3.0}
    o = oracle.render(p, sc.palette, cam, q, nthreads=os.cpu_count() or 1)
    B, _ = oracle.ambiguity(p, sc.palette, cam, q)
    assert rel_pixel_error(g, o, B) <= TOL32
    rec = oracle.project(p, sc.palette, cam, q)
    assert rnd.stats()["n_active"] == int(np.sum(rec["cls"] >= 0))
    rnd.set_params()


def test_colour_components_streamed_batched_and_half_attributes(rnd, torch_cuda):
    sc = scenes.make("precision", n=300_000, width=256)
    p = coloured(sc.parts, 2)
    cam = sc.cams[0]
    base = gpu_render(rnd, torch_cuda, p, sc.palette, cam)
    M = np.abs(base).reshape(-1, 3).max(0)
    img = torch_cuda.empty_like(torch_cuda.from_numpy(base.astype(np.float32))).cuda()
    rnd.render_stream(p, 70_001, img)
    torch_cuda.cuda.synchronize()
    assert rel_pixel_error(img.cpu().numpy().astype(np.float64), base, M=M) <= 1e-5
    cams = [scenes.camera(256, azimuth_deg=a) for a in (0.0, 40.0)]
    imgs = [torch_cuda.empty((256, 256, 3), device="cuda") for _ in cams]
    rnd.load(p)
    rnd.render_batch(cams, imgs)
    torch_cuda.cuda.synchronize()
    assert rel_pixel_error(imgs[0].cpu().numpy().astype(np.float64), base, M=M) <= 1e-5
    # binary16 h, I, s with FP32 colour components, against the oracle on the widened values
    g = gpu_render(rnd, torch_cuda, p, sc.palette, cam, fp16=sc.fp16)
    wide = dict(scenes.widened(sc.parts, sc.fp16), cr=p["cr"], cg=p["cg"], cb=p["cb"])
    o = oracle.render(wide, sc.palette, cam, {}, nthreads=os.cpu_count() or 1)
    B, _ = oracle.ambiguity(wide, sc.palette, cam)
    assert rel_pixel_error(g, o, B) <= TOL32


def test_colour_components_without_allocation(rnd, torch_cuda):
    from paper_1309_1114_gb300 import splotch as S
    parts, cam = random_scene(22, 2000, 96, 80)
    p = coloured(parts, 3)
    base = gpu_render(rnd, torch_cuda, p, scenes.ramp_palette(), cam)
    dev = {k: torch_cuda.from_numpy(v).cuda() for k, v in p.items()}
    sp = S.spl_particles(len(parts["x"]), *[dev[k].data_ptr() for k in ("x", "y", "z", "h", "I", "s")],
                         S.SPL_ATTR_F32, S.SPL_MEM_DEVICE,
                         *[dev[k].data_ptr() for k in ("cr", "cg", "cb")])
    c = S.make_camera(cam)
    pal = np.ascontiguousarray(scenes.ramp_palette(), dtype=np.float32)
    img = torch_cuda.full((cam["height"], cam["width"], 3), float("nan"), device="cuda")
    rc = S.load_library().spl_render_noalloc(C.byref(sp), C.byref(c), None, pal.ctypes.data,
                                             pal.shape[0], 0.0, 1.0, img.data_ptr(), 0, None)
    assert rc == S.SPL_OK
    torch_cuda.cuda.synchronize()
    M = np.abs(base).reshape(-1, 3).max(0)
    assert rel_pixel_error(img.cpu().numpy().astype(np.float64), base, M=M) <= 1e-5


def test_partial_colour_components_are_rejected(rnd, torch_cuda):
    from paper_1309_1114_gb300 import splotch as S
    parts, cam = random_scene(23, 10, 16, 16)
    p = coloured(parts)
    h = [np.ascontiguousarray(p[k]) for k in ("x", "y", "z", "h", "I", "s", "cr")]
    sp = S.spl_particles(10, *[a.ctypes.data for a in h[:6]], S.SPL_ATTR_F32, S.SPL_MEM_HOST,
                         h[6].ctypes.data, None, None)
    assert S.load_library().spl_load_particles(rnd._h, C.byref(sp)) == S.SPL_EINVAL
    with pytest.raises(S.SplotchError):
        rnd.set_params(log_flags=4)
