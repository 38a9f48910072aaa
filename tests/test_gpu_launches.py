"""The kernel count a render reports (spl_stats.launches) against the kernels
the CUDA profiling interface sees during the same call, for the eager path of
each mode and for the replayed graph of a batch."""
import numpy as np
import pytest

from paper_1309_1114_gb300 import scenes

pytestmark = pytest.mark.gpu


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


def profiled_kernels(torch, fn):
    """Kernels launched while fn runs, as the profiler records them (the
    first session of a process may come back empty while the profiling
    interface starts: one retry)."""
    from torch.profiler import ProfilerActivity, profile
    for _ in range(2):
        torch.cuda.synchronize()
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            fn()
            torch.cuda.synchronize()
        names = [e.name for e in prof.events()
                 if e.device_type == torch.autograd.DeviceType.CUDA and "emcpy" not in e.name
                 and "emset" not in e.name]
        if names:
            return names
    return names


@pytest.mark.parametrize("params", [{}, {"mode": 1}, {"mode": 2, "absorption": 1.0},
                                    {"sched": 1}])
def test_reported_launches_match_the_profiler(rnd, torch_cuda, params):
    sc = scenes.make("pareto", n=100_000, width=256)      # every size class, large items
    rnd.load(sc.parts)
    rnd.set_colormap(sc.palette)
    rnd.set_params(**params)
    rnd.set_camera(sc.cams[0])
    img = torch_cuda.empty((256, 256, 3), device="cuda")
    rnd.render(img)                                        # sizes the buffers
    names = profiled_kernels(torch_cuda, lambda: rnd.render(img))
    if not names:
        pytest.skip("the profiler recorded no kernels on this machine")
    st = rnd.stats()
    if params.get("mode") != 2:        # the absorbing path keeps one depth-sorted list per tile
        assert st["n_large"] > 0
    assert st["launches"] == len(names), names
    rnd.set_params()


def test_graph_replay_reports_its_kernel_nodes(rnd, torch_cuda):
    sc = scenes.make("clustered", n=200_000, width=192)
    rnd.load(sc.parts)
    rnd.set_colormap(sc.palette)
    rnd.set_params()
    cams = [scenes.camera(192, azimuth_deg=a) for a in (0.0, 30.0, 60.0)]
    imgs = [torch_cuda.empty((192, 192, 3), device="cuda") for _ in cams]
    rnd.render_batch(cams, imgs)          # eager, then the graph is captured
    rnd.render_batch(cams, imgs)          # replay
    names = profiled_kernels(torch_cuda, lambda: rnd.render_batch(cams, imgs))
    if not names:
        pytest.skip("the profiler recorded no kernels on this machine")
    assert rnd.stats()["launches"] == len(names), names
    assert np.isfinite(imgs[0].cpu().numpy()).all()
