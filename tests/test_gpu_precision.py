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
    codes = scenes.log16_h(scene.parts["h"], LOG2_MIN)
    half = {"h": codes, "I": scene.fp16["I"], "s": scene.fp16["s"]}
    g = gpu_render(rnd, torch_cuda, scene.parts, scene.palette, scene.cams[0], fp16=half,
                   h_log2_min=LOG2_MIN)
    stored = dict(scene.parts, h=scenes.log16_decoded(codes, LOG2_MIN),
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
    g, err = sampled_check(rnd, torch_cuda, sc, cam, fp16=sc.fp16, parts_oracle=wide)
    assert err <= TOL32, err
    half = {k: sc.fp16[k] for k in ("I", "s")}
    g, err = sampled_check(rnd, torch_cuda, sc, cam, fp16=half)
    assert err <= TOL16_IS, err
    codes = scenes.log16_h(sc.parts["h"], LOG2_MIN)
    g, err = sampled_check(rnd, torch_cuda, sc, cam, fp16=dict(half, h=codes), h_log2_min=LOG2_MIN)
    assert err <= TOL16_IS, err
