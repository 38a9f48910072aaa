"""The paper's MPI composition (Sec. 2) on the library: particle chunks are
rendered by the CUDA library into partial additive images, summed, and the
library's E = A map (spl_apply_ea) follows the sum.

Two forms: two contexts in one process on disjoint halves of the particles
(their images summed on the device), and two gloo ranks, each its own process
with its own context on the same GPU, composing through shard.render_frame.
The ranks' kernels never wait on one another (the all-reduce runs on the
host), so sharing one GPU is safe.  Bars: the composed frame equals the
single-context render within 1e-5 (summation order only) and the FP64
oracle within 1e-4."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1309_1114_gb300 import scenes, shard
from tests._metrics import rel_pixel_error

pytestmark = pytest.mark.gpu
TOL32 = 1e-4


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def scene():
    return scenes.make("clustered", n=300_000, width=320)


def whole_frame(torch, sc, mode):
    from paper_1309_1114_gb300.splotch import Renderer
    cam = sc.cams[0]
    r = Renderer(0)
    r.load(sc.parts)
    r.set_colormap(sc.palette)
    r.set_camera(cam)
    r.set_params(mode=mode)
    img = torch.empty((cam["height"], cam["width"], 3), device="cuda")
    r.render(img)
    torch.cuda.synchronize()
    r.close()
    return img.cpu().numpy().astype(np.float64)


def test_two_contexts_on_disjoint_halves_compose_to_the_frame(torch_cuda):
    from paper_1309_1114_gb300.splotch import Renderer
    torch = torch_cuda
    sc = scene()
    cam = sc.cams[0]
    parts = []
    for rank in range(2):
        r = Renderer(0)
        r.set_colormap(sc.palette)
        r.set_camera(cam)
        r.set_params(mode=1)                   # the frame asks for the E = A map
        img = torch.empty((cam["height"], cam["width"], 3), device="cuda")
        ea = shard.render_partial(r, sc.parts, rank, 2, img)
        assert ea and r.get_params()["mode"] == 1     # restored after the partial render
        parts.append((r, img))
    total = parts[0][1] + parts[1][1]          # the all-reduce of two partial images
    torch.cuda.synchronize()
    add = total.cpu().numpy().astype(np.float64)
    parts[0][0].apply_ea(total)
    torch.cuda.synchronize()
    ea_img = total.cpu().numpy().astype(np.float64)
    for r, _ in parts:
        r.close()
    whole_add = whole_frame(torch, sc, 0)
    whole_ea = whole_frame(torch, sc, 1)
    M = np.abs(whole_add).reshape(-1, 3).max(0)
    assert rel_pixel_error(add, whole_add, M=M) <= 1e-5
    M = np.abs(whole_ea).reshape(-1, 3).max(0)
    assert rel_pixel_error(ea_img, whole_ea, M=M) <= 1e-5
    nt = os.cpu_count() or 1
    o = oracle.render(sc.parts, sc.palette, cam, {"mode": 1}, nthreads=nt)
    B, _ = oracle.ambiguity(sc.parts, sc.palette, cam, {"mode": 1})
    assert rel_pixel_error(ea_img, o, B) <= TOL32


def test_apply_ea_is_the_map_of_every_value(torch_cuda):
    from paper_1309_1114_gb300.splotch import Renderer
    torch = torch_cuda
    v = torch.linspace(0.0, 30.0, 100_003, device="cuda", dtype=torch.float32)
    r = Renderer(0)
    out = r.apply_ea(v.clone())
    torch.cuda.synchronize()
    r.close()
    ref = -np.expm1(-v.cpu().numpy().astype(np.float64))
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=4e-7, atol=0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    from paper_1309_1114_gb300.splotch import Renderer
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        sc = scene()
        cam = sc.cams[0]
        r = Renderer(0)
        r.set_colormap(sc.palette)
        r.set_camera(cam)
        r.set_params(mode=1)
        img = torch.empty((cam["height"], cam["width"], 3), device="cuda")
        shard.render_frame(r, sc.parts, img)
        torch.cuda.synchronize()
        np.save(f"{out}.{rank}.npy", img.cpu().numpy())
        r.close()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_render_and_compose_the_frame(torch_cuda, tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "frame")
    mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    sc = scene()
    whole = whole_frame(torch_cuda, sc, 1)
    M = np.abs(whole).reshape(-1, 3).max(0)
    for rank in range(2):
        got = np.load(f"{out}.{rank}.npy").astype(np.float64)
        assert rel_pixel_error(got, whole, M=M) <= 1e-5
