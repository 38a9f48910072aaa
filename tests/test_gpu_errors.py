"""Error paths of the C ABI on a GPU: argument checks, call order, and the
policy for bad particle data (non-finite inputs or a negative smoothing
length make a particle inactive on both the GPU and the oracle)."""
import ctypes as C
import os

import numpy as np
import pytest

import oracle
from paper_1309_1114_gb300 import scenes
from tests._metrics import rel_pixel_error
from tests.test_gpu_parity import gpu_render

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def test_call_order_and_argument_checks(torch_cuda):
    from paper_1309_1114_gb300 import splotch as S
    lib = S.load_library()
    h = C.c_void_p()
    assert lib.spl_create(C.byref(h), 0, None) == S.SPL_OK
    img = torch_cuda.zeros((8, 8, 3), device="cuda")
    try:
        assert lib.spl_render(h, img.data_ptr(), None) == S.SPL_ESTATE      # nothing loaded
        assert lib.spl_create(C.byref(C.c_void_p()), 999, None) == S.SPL_EINVAL
        bad = [dict(scenes.camera(8), width=0), dict(scenes.camera(8), fov_y_deg=0.0),
               dict(scenes.camera(8), z_near=0.0),
               dict(scenes.camera(8), up=(0.0, 0.0, 1.0), target=(0.5, 0.5, 5.0)),
               dict(scenes.camera(8), width=20000)]
        for cam in bad:
            c = S.make_camera(cam)
            assert lib.spl_set_camera(h, C.byref(c)) == S.SPL_EINVAL
        for kw in ({"tile_px": 48}, {"r_small": 0.1}, {"r_large": 1.0, "r_small": 4.0},
                   {"chi": -1.0}, {"mode": 7}, {"sched": 9}):
            q = S.default_params(**kw)
            assert lib.spl_set_params(h, C.byref(q)) == S.SPL_EINVAL
        pal = np.array([[0, 0, 0], [np.nan, 1, 1]], np.float32)
        assert lib.spl_set_colormap(h, pal.ctypes.data, 2, 0.0, 1.0) == S.SPL_EINVAL
        assert lib.spl_set_colormap(h, pal.ctypes.data, 0, 0.0, 1.0) == S.SPL_EINVAL
        p = S.spl_particles(10, None, None, None, None, None, None, S.SPL_ATTR_F32, S.SPL_MEM_HOST)
        assert lib.spl_load_particles(h, C.byref(p)) == S.SPL_EINVAL
        n = C.c_int64(0)
        assert lib.spl_get_samples(h, None, None, 0, C.byref(n)) == S.SPL_ESTATE
        assert lib.spl_render_batch(h, None, 1, None, None) == S.SPL_EINVAL
    finally:
        assert lib.spl_destroy(h) == S.SPL_OK


def test_bad_particles_are_inactive(torch_cuda):
    from paper_1309_1114_gb300.splotch import Renderer
    sc = scenes.make("uniform", n=5000, width=96)
    parts = {k: v.copy() for k, v in sc.parts.items()}
    rng = np.random.default_rng(0)
    for k, bad in (("x", np.nan), ("z", np.inf), ("h", np.nan), ("h", -0.01), ("I", np.inf),
                   ("s", np.nan)):
        parts[k][rng.integers(0, 5000, 40)] = bad
    cam = sc.cams[0]
    r = Renderer(0)
    try:
        g = gpu_render(r, torch_cuda, parts, sc.palette, cam)
        assert np.isfinite(g).all()
        o = oracle.render(parts, sc.palette, cam, {}, nthreads=os.cpu_count() or 1)
        B, _ = oracle.ambiguity(parts, sc.palette, cam)
        assert rel_pixel_error(g, o, B) <= 1e-4
        rec = oracle.project(parts, sc.palette, cam)
        assert r.stats()["n_active"] == int(np.sum(rec["cls"] >= 0)) < 5000
    finally:
        r.close()
