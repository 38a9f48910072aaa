"""The tile-cost network and the scheduler it drives.

* the network's forward, gradient and Adam kernels (FP32, GPU) against the
  FP64 oracle in oracle/ (itself pinned by finite differences);
* the per-item features of single-item tiles against the oracle's tile
  features (bit-exact up to radius-bin ties);
* longest-first scheduling (count heuristic or network) never changes the
  image;
* trained on the renderer's own timings, the network predicts held-out item
  costs better than the count heuristic;
* on a heavy-tailed scene the longest work item is measured against its pass
  (since persistent CTAs take items from a queue, no order of the items can
  shorten a pass by more than that fraction), and the frame times under each
  schedule are measured: the asserted result is that neither longest-first
  schedule beats taking the items in image order (a negative result).
"""
import os

import numpy as np
import pytest

import oracle
from paper_1309_1114_gb300 import scenes
from tests._metrics import rel_pixel_error
from tests.test_gpu_parity import gpu_render

pytestmark = pytest.mark.gpu
NP = 2177


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


def random_net(seed, n=256):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0, 0.25, NP)
    x = rng.random((n, 32)) * 3
    t = rng.normal(10, 2, n)
    return theta, x, t


def test_forward_matches_oracle(torch_cuda):
    from paper_1309_1114_gb300 import splotch as S
    theta, x, t = random_net(0)
    th = torch_cuda.tensor(theta, dtype=torch_cuda.float32, device="cuda")
    xs = torch_cuda.tensor(x, dtype=torch_cuda.float32, device="cuda")
    y = torch_cuda.empty(len(t), device="cuda")
    assert S.load_library().spl_mlp_forward(th.data_ptr(), xs.data_ptr(), len(t), y.data_ptr(), None) == 0
    torch_cuda.cuda.synchronize()
    ref = oracle.mlp_forward(th.cpu().numpy().astype(np.float64), xs.cpu().numpy().astype(np.float64))
    np.testing.assert_allclose(y.cpu().numpy(), ref, rtol=1e-5, atol=1e-5)


def test_gradient_matches_oracle(torch_cuda):
    from paper_1309_1114_gb300 import splotch as S
    theta, x, t = random_net(1, n=3000)
    th = torch_cuda.tensor(theta, dtype=torch_cuda.float32, device="cuda")
    xs = torch_cuda.tensor(x, dtype=torch_cuda.float32, device="cuda")
    ts = torch_cuda.tensor(t, dtype=torch_cuda.float32, device="cuda")
    g = torch_cuda.empty(NP, device="cuda")
    loss = torch_cuda.empty(1, device="cuda")
    rc = S.load_library().spl_mlp_loss_grad(th.data_ptr(), xs.data_ptr(), ts.data_ptr(), len(t),
                                            g.data_ptr(), loss.data_ptr(), None)
    assert rc == 0
    ref_loss, ref_g = oracle.mlp_loss_grad(th.cpu().numpy().astype(np.float64),
                                           xs.cpu().numpy().astype(np.float64),
                                           ts.cpu().numpy().astype(np.float64))
    assert loss.item() == pytest.approx(ref_loss, rel=1e-5)
    gg = g.cpu().numpy().astype(np.float64)
    scale = np.abs(ref_g).max()
    assert np.max(np.abs(gg - ref_g)) <= 1e-5 * scale


def test_adam_step_matches_oracle(torch_cuda):
    from paper_1309_1114_gb300 import splotch as S
    rng = np.random.default_rng(2)
    th0, g0 = rng.normal(0, 1, NP), rng.normal(0, 1, NP)
    th = torch_cuda.tensor(th0, dtype=torch_cuda.float32, device="cuda")
    g = torch_cuda.tensor(g0, dtype=torch_cuda.float32, device="cuda")
    m = torch_cuda.zeros(NP, device="cuda")
    v = torch_cuda.zeros(NP, device="cuda")
    ref_th = th.cpu().numpy().astype(np.float64)
    ref_m, ref_v = np.zeros(NP), np.zeros(NP)
    for step in (1, 2, 3):
        assert S.load_library().spl_mlp_adam(th.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(),
                                             NP, step, 1e-2, 0.9, 0.999, 1e-8, None) == 0
        oracle.adam_step(ref_th, g.cpu().numpy().astype(np.float64), ref_m, ref_v, step, lr=1e-2)
    torch_cuda.cuda.synchronize()
    np.testing.assert_allclose(th.cpu().numpy(), ref_th, rtol=1e-5, atol=1e-6)


def test_item_features_match_oracle_tile_features(rnd, torch_cuda):
    # few enough particles that no tile is split (small particles in their own
    # list, which holds twice as many entries per item); no large class
    sc = scenes.make("uniform", n=20_000, width=320)
    cam = sc.cams[0]
    rnd.load(sc.parts)
    rnd.set_colormap(sc.palette)
    rnd.set_params(r_small=4.0, r_large=1e9)
    rnd.set_camera(cam)
    rnd.set_recording(True)
    img = torch_cuda.empty((cam["height"], cam["width"], 3), device="cuda")
    rnd.render(img)
    f = torch_cuda.empty((4096, 32), device="cuda")
    t = torch_cuda.empty((4096,), device="cuda")
    n = rnd.samples(f, t)
    rnd.set_recording(False)
    st = rnd.stats()
    assert 0 < n <= st["n_tiles"] and n < 4096
    ref = oracle.tile_features(sc.parts, sc.palette, cam, {}, 32, area_scale=32 * 32)
    got = f[:n].cpu().numpy().astype(np.float64)
    # match each item to its tile through its feature vector: the item order
    # is the tile order of the non-empty tiles
    nonempty = np.where(ref[:, :16].sum(1) > 0)[0]
    assert len(nonempty) == n
    # counts and box areas per radius bin; the binning's 1e-3 px safety margin
    # and radius-bin ties may move a particle in or out of a tile or bin
    cg, cr = np.expm1(got[:, :16]), np.expm1(ref[nonempty][:, :16])
    ag, ar = np.expm1(got[:, 16:]) * 1024, np.expm1(ref[nonempty][:, 16:]) * 1024
    assert np.abs(cg - cr).sum() <= 2 + 0.002 * cr.sum()
    assert np.abs(ag - ar).sum() <= 0.002 * ar.sum()
    assert np.mean(np.abs(got - ref[nonempty]) < 1e-4) > 0.99
    assert np.all(np.isfinite(t[:n].cpu().numpy())) and t[:n].min().item() > 0
    rnd.set_params()


@pytest.mark.parametrize("sched", [1, 2])
def test_schedule_does_not_change_the_image(rnd, torch_cuda, sched):
    sc = scenes.make("pareto", n=300_000, width=512)
    cam = sc.cams[0]
    base = gpu_render(rnd, torch_cuda, sc.parts, sc.palette, cam)
    if sched == 2:
        from paper_1309_1114_gb300 import scheduler
        rnd.set_model(scheduler.init_theta(7, bias=10.0))
    got = gpu_render(rnd, torch_cuda, sc.parts, sc.palette, cam, sched=sched)
    M = np.abs(base).reshape(-1, 3).max(0)
    assert rel_pixel_error(got, base, M=M) < 1e-5
    o = oracle.render(sc.parts, sc.palette, cam, {}, nthreads=os.cpu_count() or 1)
    B, _ = oracle.ambiguity(sc.parts, sc.palette, cam)
    assert rel_pixel_error(got, o, B) <= 1e-4


def test_network_predicts_better_and_schedule_gain_is_bounded(rnd, torch_cuda):
    from paper_1309_1114_gb300 import scheduler
    # training samples from clustered, precision-like and orbit-like renders
    feats, logcs = [], []
    for name, n, w in (("clustered", 2_000_000, 1024), ("precision", 2_000_000, 1024),
                       ("orbit", 1_000_000, 2048)):
        sc = scenes.make(name, n=n, width=w)
        rnd.load(sc.parts)
        rnd.set_colormap(sc.palette)
        rnd.set_params()
        f, t = scheduler.collect(rnd, torch_cuda, sc.cams[:6])
        feats.append(f)
        logcs.append(t)
    f = torch_cuda.cat(feats)
    t = torch_cuda.cat(logcs)
    perm = torch_cuda.randperm(f.shape[0], generator=torch_cuda.Generator().manual_seed(0)).cuda()
    f, t = f[perm], t[perm]
    ntr = int(0.8 * f.shape[0])
    theta, losses = scheduler.train(f[:ntr], t[:ntr], steps=2000, lr=3e-3)
    assert losses[-1] < 0.5 * losses[0]
    heur = scheduler.fit_count_heuristic(f[:ntr], t[:ntr])
    te = t[ntr:].cpu().numpy()
    err_mlp = scheduler.rmse(scheduler.predict(theta, f[ntr:], torch_cuda).cpu().numpy(), te)
    cnt = np.log1p(scheduler.entries_of(f[ntr:]))
    err_cnt = scheduler.rmse(heur[0] + heur[1] * cnt, te)
    print(f"held-out RMSE of log(cycles): network {err_mlp:.3f}, count heuristic {err_cnt:.3f}, "
          f"{f.shape[0]} samples")
    assert err_mlp < err_cnt
    # the schedule on a heavy-tailed scene: what any order of the work items
    # can gain is bounded by the longest item against its pass (persistent CTAs
    # take items from a queue, so a pass ends at most one item after the ideal
    # finish); record every item's SM cycles without a schedule, then time the
    # frame under each schedule
    sc = scenes.make("pareto", n=4_000_000, width=1024)
    cam = sc.cams[0]
    rnd.load(sc.parts)
    rnd.set_colormap(sc.palette)
    rnd.set_model(theta, heur)
    rnd.set_camera(cam)
    img = torch_cuda.empty((cam["height"], cam["width"], 3), device="cuda")
    rnd.set_params()
    rnd.set_timing(True)
    for _ in range(3):
        rnd.render(img)
    st = rnd.stats()
    rnd.set_timing(False)
    pass_ms = st["sum_ms"][2] / max(st["timed_frames"], 1) + st["sum_ms"][3] / max(st["timed_frames"], 1)
    f, logc = scheduler.collect(rnd, torch_cuda, [cam])
    cycles = np.exp(logc.cpu().numpy().astype(np.float64))
    clock_hz = 2.07e9                          # SM clock under load (sm_max_mhz)
    bound = cycles.max() / (pass_ms * 1e-3 * clock_hz)
    times = {}
    for sched in (0, 1, 2):
        rnd.set_params(sched=sched)
        rnd.render(img)
        rnd.set_timing(True)
        for _ in range(5):
            rnd.render(img)
        st = rnd.stats()
        rnd.set_timing(False)
        times[sched] = st["sum_ms"][5] / max(st["timed_frames"], 1)
    print(f"longest item / tile + large passes: {bound:.4f} ({cycles.size} items); "
          f"frame ms by scheduler (none, count, network): {times}")
    rnd.set_params()
    # the measured result: the better prediction does not turn into a faster
    # frame -- taking the items in image order keeps neighbouring items on shared
    # records in L2, the heavy items already start early enough that the tail
    # the bound allows is not lost, and the network's features cost their own
    # kernels; neither schedule beats the in-order items by more than timing noise
    assert 0.0 < bound < 1.0
    assert times[2] >= times[0] * 0.97
    assert times[1] >= times[0] * 0.97
