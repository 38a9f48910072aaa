"""spl_render_noalloc: the render for callers that cannot allocate device memory.

Some callers cannot let a library call cudaMalloc: an application whose device
memory comes from its own allocator or is held to a fixed budget, or a host
program that passes only its own buffers and wants no hidden device
allocation.  For them the library has one entry point that takes the caller's
device particle arrays and output image and keeps every scratch buffer in a
fixed file-scope device array.  This test calls it through the C ABI twice in
a row and checks each image against the ordinary entry point, spl_render,
within the tolerance the other GPU-vs-GPU comparisons use (1e-5 per-pixel
relative, since the tile lists are filled with atomics and the summation order
may differ).  It also checks that sizes beyond the fixed maximum are rejected
with SPL_ELIMIT -- before binning (particles, tiles) and after it (list
entries) -- after which the entry point still renders correctly, and that the
call refuses a stream that is being captured into a CUDA graph (it waits on
the host mid-way, which capture forbids).

The file name makes pytest collect it last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1309_1114_gb300 import scenes
from tests._metrics import rel_pixel_error

pytestmark = pytest.mark.gpu


def _scene():
    rng = np.random.default_rng(21)
    n = 60000
    parts = {"x": rng.random(n, dtype=np.float32), "y": rng.random(n, dtype=np.float32),
             "z": rng.random(n, dtype=np.float32),
             "h": np.exp(np.log(0.004) + 0.7 * rng.standard_normal(n)).astype(np.float32),
             "I": rng.random(n, dtype=np.float32), "s": rng.random(n, dtype=np.float32)}
    cam = scenes.camera(320, 240)
    return parts, cam, scenes.ramp_palette()


def test_noalloc_render_matches_spl_render_twice():
    import torch
    from paper_1309_1114_gb300 import splotch as S

    parts, cam, pal = _scene()
    n = parts["x"].size
    r = S.Renderer(0)
    r.load(parts)
    r.set_colormap(pal)
    r.set_camera(cam)
    r.set_params()
    ref = torch.empty((cam["height"], cam["width"], 3), device="cuda", dtype=torch.float32)
    r.render(ref)
    torch.cuda.synchronize()
    ref_np = ref.cpu().numpy().astype(np.float64)
    r.close()
    assert np.isfinite(ref_np).all() and ref_np.max() > 0

    lib = S.load_library()
    dev = {k: torch.from_numpy(v).cuda() for k, v in parts.items()}
    p = S.spl_particles(n, *[dev[k].data_ptr() for k in ("x", "y", "z", "h", "I", "s")],
                        S.SPL_ATTR_F32, S.SPL_MEM_DEVICE)
    c = S.make_camera(cam)
    q = S.default_params()
    pal_c = np.ascontiguousarray(pal, dtype=np.float32)
    stream = torch.cuda.current_stream().cuda_stream
    M = np.abs(ref_np).reshape(-1, 3).max(0)
    for _ in range(2):
        out = torch.full_like(ref, float("nan"))
        rc = lib.spl_render_noalloc(C.byref(p), C.byref(c), C.byref(q), pal_c.ctypes.data,
                                    pal_c.shape[0], 0.0, 1.0, out.data_ptr(), 0, stream)
        assert rc == S.SPL_OK, lib.spl_error_string(rc)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        assert np.isfinite(got).all()
        assert rel_pixel_error(got, ref_np, M=M) < 1e-5


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_1309_1114_gb300 import splotch as S

    lib = S.load_library()
    n = 131073                                   # one more than the fixed maximum
    buf = torch.zeros(n, device="cuda", dtype=torch.float32)
    p = S.spl_particles(n, *([buf.data_ptr()] * 6), S.SPL_ATTR_F32, S.SPL_MEM_DEVICE)
    c = S.make_camera(scenes.camera(64, 64))
    pal = np.ascontiguousarray(scenes.ramp_palette())
    img = torch.zeros((64, 64, 3), device="cuda", dtype=torch.float32)
    rc = lib.spl_render_noalloc(C.byref(p), C.byref(c), None, pal.ctypes.data, pal.shape[0],
                                0.0, 1.0, img.data_ptr(), 0, None)
    assert rc == S.SPL_ELIMIT
    big = S.make_camera(scenes.camera(8192, 8192))   # 65536 tiles of 32 px
    p.n = 10
    rc = lib.spl_render_noalloc(C.byref(p), C.byref(big), None, pal.ctypes.data, pal.shape[0],
                                0.0, 1.0, img.data_ptr(), 0, None)
    assert rc == S.SPL_ELIMIT


def _noalloc(lib, S, parts_dev, n, cam, img, q=None, stream=None):
    p = S.spl_particles(n, *[parts_dev[k].data_ptr() for k in ("x", "y", "z", "h", "I", "s")],
                        S.SPL_ATTR_F32, S.SPL_MEM_DEVICE)
    c = S.make_camera(cam)
    pal = np.ascontiguousarray(scenes.ramp_palette())
    return lib.spl_render_noalloc(C.byref(p), C.byref(c), None if q is None else C.byref(q),
                                  pal.ctypes.data, pal.shape[0], 0.0, 1.0, img.data_ptr(), 0,
                                  stream)


def test_noalloc_rejects_lists_beyond_its_scratch_then_renders_again():
    import torch
    from paper_1309_1114_gb300 import splotch as S

    lib = S.load_library()
    # 131072 discs of radius ~40 px on a 2048^2 frame of 16 px tiles (16384
    # tiles): ~25 tile-list entries each, more than the 2^21 the scratch holds
    rng = np.random.default_rng(5)
    n = 131072
    big = {"x": rng.random(n, dtype=np.float32), "y": rng.random(n, dtype=np.float32),
           "z": rng.random(n, dtype=np.float32), "h": np.full(n, 0.015, np.float32),
           "I": rng.random(n, dtype=np.float32), "s": rng.random(n, dtype=np.float32)}
    dev = {k: torch.from_numpy(v).cuda() for k, v in big.items()}
    cam = scenes.camera(2048, 2048)
    img = torch.zeros((2048, 2048, 3), device="cuda", dtype=torch.float32)
    q = S.default_params(tile_px=16)
    rc = _noalloc(lib, S, dev, n, cam, img, q)
    assert rc == S.SPL_ELIMIT, lib.spl_error_string(rc)
    torch.cuda.synchronize()
    assert float(img.abs().max()) == 0.0          # nothing rendered

    parts, cam, pal = _scene()
    r = S.Renderer(0)
    r.load(parts)
    r.set_colormap(pal)
    r.set_camera(cam)
    ref = torch.empty((cam["height"], cam["width"], 3), device="cuda", dtype=torch.float32)
    r.render(ref)
    torch.cuda.synchronize()
    ref_np = ref.cpu().numpy().astype(np.float64)
    r.close()
    dev = {k: torch.from_numpy(v).cuda() for k, v in parts.items()}
    out = torch.full_like(ref, float("nan"))
    rc = _noalloc(lib, S, dev, parts["x"].size, cam, out)
    assert rc == S.SPL_OK, lib.spl_error_string(rc)
    torch.cuda.synchronize()
    M = np.abs(ref_np).reshape(-1, 3).max(0)
    assert rel_pixel_error(out.cpu().numpy().astype(np.float64), ref_np, M=M) < 1e-5


def test_noalloc_refuses_a_capturing_stream():
    import torch
    from paper_1309_1114_gb300 import splotch as S

    lib = S.load_library()
    parts, cam, pal = _scene()
    dev = {k: torch.from_numpy(v).cuda() for k, v in parts.items()}
    out = torch.zeros((cam["height"], cam["width"], 3), device="cuda", dtype=torch.float32)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side, capture_error_mode="thread_local"):
        rc = _noalloc(lib, S, dev, parts["x"].size, cam, out, stream=side.cuda_stream)
    assert rc == S.SPL_ESTATE
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0          # nothing was queued
