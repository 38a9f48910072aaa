"""Pins for the oracle's colouring options (Sec. 2): per-particle colour
components in place of the palette (a vector quantity gives R, G, B
directly), and logarithms of the intensity and of the colour scalar before
normalisation."""
import numpy as np
import pytest

import oracle
from paper_1309_1114_gb300 import scenes
from tests.test_oracle_pins import axis_camera, parts_of, random_tiny_scene


def with_rgb(parts, rgb):
    q = dict(parts)
    rgb = np.asarray(rgb, dtype=np.float32).reshape(-1, 3)
    rgb = np.broadcast_to(rgb, (len(parts["x"]), 3))
    q["cr"], q["cg"], q["cb"] = (np.ascontiguousarray(rgb[:, k]) for k in range(3))
    return q


def test_components_on_a_pixel_centre_by_hand():
    # 65 x 65, fov 90: the axis point lands on the centre of pixel (32, 32)
    cam = axis_camera(65)
    p = with_rgb(parts_of([0.0, 0.0, 1.0, 2.0 / 32.5, 2.0, 0.3]), [0.25, 0.75, 0.125])
    img = oracle.render(p, scenes.ramp_palette(), cam)
    np.testing.assert_allclose(img[32, 32], [0.5, 1.5, 0.25], rtol=1e-12)


def test_components_equal_to_a_constant_palette():
    p, cam = random_tiny_scene(3, n=80)
    pal = np.array([[0.3, 0.6, 0.9]], dtype=np.float32)
    a = oracle.render(p, pal, cam)
    b = oracle.render(with_rgb(p, pal[0]), scenes.ramp_palette(), cam)
    np.testing.assert_allclose(b, a, rtol=1e-12, atol=1e-300)


def test_components_are_separate_channels():
    p, cam = random_tiny_scene(4, n=80)
    rng = np.random.default_rng(0)
    rgb = rng.random((80, 3)).astype(np.float32)
    full = oracle.render(with_rgb(p, rgb), scenes.ramp_palette(), cam)
    swapped = oracle.render(with_rgb(p, rgb[:, ::-1]), scenes.ramp_palette(), cam)
    np.testing.assert_allclose(swapped, full[..., ::-1], rtol=1e-12, atol=1e-300)
    red = oracle.render(with_rgb(p, rgb * [1, 0, 0]), scenes.ramp_palette(), cam)
    np.testing.assert_allclose(red[..., 0], full[..., 0], rtol=1e-12, atol=1e-300)
    assert np.all(red[..., 1:] == 0.0)


def test_log_of_the_colour_scalar_before_normalisation():
    # s = 1, 10, 100, 1000 with log10 and range [0, 3] equals s = 0, 1, 2, 3 with
    # range [0, 3] and no logarithm (powers of ten: exact in FP32 and in log10)
    p, cam = random_tiny_scene(5, n=120)
    k = np.arange(120) % 4
    lin = dict(p, s=k.astype(np.float32))
    log = dict(p, s=(10.0 ** k).astype(np.float32))
    pal = scenes.ramp_palette()
    a = oracle.render(lin, pal, cam, {"s_min": 0.0, "s_max": 3.0})
    b = oracle.render(log, pal, cam, {"s_min": 0.0, "s_max": 3.0, "log": 2})
    np.testing.assert_allclose(b, a, rtol=1e-12, atol=1e-300)


def test_log_of_the_intensity():
    p, cam = random_tiny_scene(6, n=120)
    k = 1 + np.arange(120) % 3
    a = oracle.render(dict(p, I=k.astype(np.float32)), scenes.ramp_palette(), cam)
    b = oracle.render(dict(p, I=(10.0 ** k).astype(np.float32)), scenes.ramp_palette(), cam, {"log": 1})
    np.testing.assert_allclose(b, a, rtol=1e-12, atol=1e-300)


def test_non_positive_values_under_logarithms_are_inactive():
    p = parts_of([[0.0, 0.0, 1.0, 0.05, 0.0, 0.5], [0.0, 0.0, 1.0, 0.05, 1.0, -1.0],
                  [0.0, 0.0, 1.0, 0.05, 10.0, 10.0]])
    cam = axis_camera(65)
    rec = oracle.project(p, scenes.ramp_palette(), cam, {"log": 3})
    assert list(rec["cls"]) == [-2, -2, 1]
    rec = oracle.project(p, scenes.ramp_palette(), cam, {"log": 1})
    assert list(rec["cls"]) == [-2, 1, 1]
    bad = with_rgb(p, [[np.nan, 0, 0], [0, 0, 0], [1, 1, 1]])
    assert list(oracle.project(bad, scenes.ramp_palette(), cam)["cls"]) == [-2, 1, 1]
