"""FP16 attribute storage: the precision form of the render.

Positions and all arithmetic stay FP32 (the camera transform in double-float
FP32); h, I and s are stored as binary16 (SPL_ATTR_F16, 18 B per particle) or
only I and s are (SPL_ATTR_F16_IS, 20 B per particle), and widened to FP32 on
load.  Two errors are checked per image:

* against the FP64 oracle run on the same stored values (the binary16 values
  widened exactly): the render's own arithmetic, held to the FP32 bound 1e-4;
* against the FP64 oracle run on the original FP32 attributes: the storage
  error as well.  h sits inside exp(-d^2/h^2), so its 2^-11 rounding moves a
  clip-edge weight by up to ~2 chi^2 2^-11; with h in binary16 the image
  error is ~3e-3 (bound asserted: 4e-3), with h kept in FP32 it stays under
  the 2e-3 target, and so it does with h as a 16-bit logarithmic code
  (SPL_ATTR_LOGH16, 18 B per particle: 1/4096-octave steps).
"""
import os

import numpy as np
import pytest

import oracle
from paper_1309_1114_gb300 import scenes
from tests._codes import log16_decoded, log16_h
from tests._metrics import rel_pixel_error
from tests.test_gpu_parity import gpu_render, sampled_check

pytestmark = pytest.mark.gpu
TOL32 = 1e-4
TOL16_IS = 2e-3      # target bound, met with h in FP32 or as a 16-bit log code
TOL16_ALL = 4e-3     # stated bound with h in binary16 as well
LOG2_MIN = -14.0     # h of code 0: 2^-14 < 1e-4, the generator's smallest h


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


@pytest.fixture(scope="module")
def scene():
    return scenes.make("precision", n=400_000, width=512)


@pytest.fixture(scope="module")
def oracle_images(scene):
    cam = scene.cams[0]
    nt = os.cpu_count() or 1
    o32 = oracle.render(scene.parts, scene.palette, cam, {}, nthreads=nt)
    B32, _ = oracle.ambiguity(scene.parts, scene.palette, cam)
    wide = scenes.widened(scene.parts, scene.fp16)
    o16 = oracle.render(wide, scene.palette, cam, {}, nthreads=nt)
    B16, _ = oracle.ambiguity(wide, scene.palette, cam)
    wide_is = dict(scene.parts, I=wide["I"], s=wide["s"])
    o16is = oracle.render(wide_is, scene.palette, cam, {}, nthreads=nt)
    B16is, _ = oracle.ambiguity(wide_is, scene.palette, cam)
    return {"o32": (o32, B32), "o16": (o16, B16), "o16is": (o16is, B16is)}


def test_fp16_all_attributes(rnd, torch_cuda, scene, oracle_images):
    g = gpu_render(rnd, torch_cuda, scene.parts, scene.palette, scene.cams[0], fp16=scene.fp16)
    o16, B16 = oracle_images["o16"]
    assert rel_pixel_error(g, o16, B16) <= TOL32            # arithmetic
    o32, B32 = oracle_images["o32"]
    err = rel_pixel_error(g, o32, B32)                     # storage + arithmetic
    assert err <= TOL16_ALL, err


def test_fp16_intensity_and_scalar(rnd, torch_cuda, scene, oracle_images):
    half = {k: scene.fp16[k] for k in ("I", "s")}
    g = gpu_render(rnd, torch_cuda, scene.parts, scene.palette, scene.cams[0], fp16=half)
    o16is, B16is = oracle_images["o16is"]
    assert rel_pixel_error(g, o16is, B16is) <= TOL32
    o32, B32 = oracle_images["o32"]
    err = rel_pixel_error(g, o32, B32)
    assert err <= TOL16_IS, err


def test_log16_smoothing_length_meets_the_target(rnd, torch_cuda, scene, oracle_images):
    codes = log16_h(scene.parts["h"], LOG2_MIN)
    half = {"h": codes, "I": scene.fp16["I"], "s": scene.fp16["s"]}
    g = gpu_render(rnd, torch_cuda, scene.parts, scene.palette, scene.cams[0], fp16=half,
                   h_log2_min=LOG2_MIN)
    stored = dict(scene.parts, h=log16_decoded(codes, LOG2_MIN),
                  I=scene.fp16["I"].astype(np.float32), s=scene.fp16["s"].astype(np.float32))
    cam = scene.cams[0]
    o, B = oracle.render(stored, scene.palette, cam, {}, nthreads=os.cpu_count() or 1), \
        oracle.ambiguity(stored, scene.palette, cam)[0]
    assert rel_pixel_error(g, o, B) <= TOL32                # arithmetic
    o32, B32 = oracle_images["o32"]
    err = rel_pixel_error(g, o32, B32)                     # storage + arithmetic
    assert err <= TOL16_IS, err


def test_fp16_against_fp32_gpu_path(rnd, torch_cuda, scene):
    cam = scene.cams[0]
    g32 = gpu_render(rnd, torch_cuda, scene.parts, scene.palette, cam)
    g16 = gpu_render(rnd, torch_cuda, scene.parts, scene.palette, cam, fp16=scene.fp16)
    assert 0 < rel_pixel_error(g16, g32) <= TOL16_ALL


def test_precision_full_size_sampled(rnd, torch_cuda):
    """100M particles, 2048^2, all three attribute layouts, at sampled pixels."""
    sc = scenes.make("precision")
    cam = sc.cams[0]
    wide = scenes.widened(sc.parts, sc.fp16)
    g, err = sampled_check(rnd, torch_cuda, sc, cam)
    assert err <= TOL32, err
    few = {"n_windows": 1, "n_bright": 32, "n_random": 96}      # >= 1024 pixels each
    g, err = sampled_check(rnd, torch_cuda, sc, cam, fp16=sc.fp16, parts_oracle=wide, **few)
    assert err <= TOL32, err
    half = {k: sc.fp16[k] for k in ("I", "s")}
    g, err = sampled_check(rnd, torch_cuda, sc, cam, fp16=half, **few)
    assert err <= TOL16_IS, err
    codes = log16_h(sc.parts["h"], LOG2_MIN)
    g, err = sampled_check(rnd, torch_cuda, sc, cam, fp16=dict(half, h=codes), h_log2_min=LOG2_MIN,
                           **few)
    assert err <= TOL16_IS, err


# ------------------------------------------------------- the library encoder
def test_library_encoder_writes_the_reference_codes(rnd, torch_cuda, scene):
    """spl_encode_attrs: binary16 values bit for bit as numpy rounds them, and
    the 16-bit log codes of h as the FP64 reference encoder gives them."""
    from paper_1309_1114_gb300 import splotch as S
    torch = torch_cuda
    dev = {k: torch.from_numpy(scene.parts[k]).cuda() for k in ("h", "I", "s")}
    for store in (S.SPL_ATTR_F32, S.SPL_ATTR_F16, S.SPL_ATTR_F16_IS, S.SPL_ATTR_LOGH16):
        out = rnd.encode_attrs(dev["h"], dev["I"], dev["s"], store, LOG2_MIN)
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in out.items()}
        half = {k: scene.parts[k].astype(np.float16).view(np.uint16) for k in ("h", "I", "s")}
        if store == S.SPL_ATTR_F32:
            for k in ("h", "I", "s"):
                assert np.array_equal(got[k].view(np.uint32), scene.parts[k].view(np.uint32))
            continue
        assert np.array_equal(got["I"].view(np.uint16), half["I"])
        assert np.array_equal(got["s"].view(np.uint16), half["s"])
        if store == S.SPL_ATTR_F16:
            assert np.array_equal(got["h"].view(np.uint16), half["h"])
        elif store == S.SPL_ATTR_F16_IS:
            assert np.array_equal(got["h"].view(np.uint32), scene.parts["h"].view(np.uint32))
        else:
            assert np.array_equal(got["h"].view(np.uint16), log16_h(scene.parts["h"], LOG2_MIN))


def test_load_as_log16_renders_the_coded_image(rnd, torch_cuda, scene):
    """FP32 attributes loaded with log-code storage render the image of the
    codes encoded beforehand (1e-5: summation order only), and keep the
    particles that no code can stand for inactive."""
    from paper_1309_1114_gb300 import splotch as S
    torch = torch_cuda
    cam = scene.cams[0]
    codes = log16_h(scene.parts["h"], LOG2_MIN)
    coded = gpu_render(rnd, torch, scene.parts, scene.palette, cam,
                       fp16={"h": codes, "I": scene.fp16["I"], "s": scene.fp16["s"]},
                       h_log2_min=LOG2_MIN)
    rnd.load(scene.parts, store_as=S.SPL_ATTR_LOGH16, h_log2_min=LOG2_MIN)
    img = torch.empty((cam["height"], cam["width"], 3), device="cuda")
    rnd.render(img)
    torch.cuda.synchronize()
    got = img.cpu().numpy().astype(np.float64)
    M = np.abs(coded).reshape(-1, 3).max(0)
    assert rel_pixel_error(got, coded, M=M) <= 1e-5
    # host arrays go through the same device encoder
    bad = {k: v[:1000].copy() for k, v in scene.parts.items()}
    bad["h"][:3] = [-1.0, np.nan, np.inf]
    active = []
    for store in (S.SPL_ATTR_F32, S.SPL_ATTR_LOGH16):
        rnd.load(bad, store_as=store, h_log2_min=LOG2_MIN)
        rnd.set_camera(cam)
        small = torch.empty((cam["height"], cam["width"], 3), device="cuda")
        rnd.render(small)
        recs = rnd.records(1000)
        assert np.all(recs["cls"][:3] == -2)
        active.append(int(np.sum(recs["cls"][3:] >= 0)))
    # the coded h moves a radius by < 1e-4 relative: the same particles stay active
    assert active[0] > 900 and abs(active[0] - active[1]) <= 2
    with pytest.raises(S.SplotchError):
        rnd.load(bad, store_as=S.SPL_ATTR_LOGH16, h_log2_min=float("nan"))
    with pytest.raises(S.SplotchError):
        rnd.load(bad, store_as=7)
