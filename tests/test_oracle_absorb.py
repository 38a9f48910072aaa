"""Pins for the oracle's general absorption form (Eq. 1 with E_p != A_p, mode 2).

Across particle p a ray's intensity becomes I exp(-tau) + (E/A)(1 - exp(-tau)),
tau = A w; particles are crossed from the farthest to the nearest.  The pins
fix this against values worked out by hand from Eq. 1 (two particles in front
of each other, both orders, and equal depths), against the E = A special case
(whose solution 1 - exp(-S) is order-free), against the optically thin limit
(small absorption gives the additive sum), against opacity (large absorption
gives the nearest source term), and against the pixel-major brute force.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1309_1114_gb300 import scenes
from tests.test_oracle_pins import axis_camera, parts_of, random_tiny_scene

RED_BLUE = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 1.0]], dtype=np.float32)


def absorb(parts, pal, cam, alpha=1.0, brute=False, **par):
    q = dict(par, mode=2, absorption=alpha)
    return (oracle.render_bruteforce if brute else oracle.render)(parts, pal, cam, q)


def two_on_axis(z_red, z_blue):
    # 65 x 65, fov 90: the axis lands on the centre of pixel (32, 32), where the
    # Gaussian weight is exactly 1; h gives sigma_s >= 2 px at both depths
    return parts_of([[0.0, 0.0, z_red, 0.2, 1.0, 0.0], [0.0, 0.0, z_blue, 0.2, 1.0, 1.0]])


def test_two_particles_front_and_back_by_hand():
    # tau = absorption * I * w = 1 at the centre pixel for both particles.
    # Red in front of blue: start at 0 behind blue, cross blue then red:
    #   I = (0, 0, 1)(1 - 1/e);  I = I/e + (1, 0, 0)(1 - 1/e)
    cam = axis_camera(65)
    g = 1.0 - math.exp(-1.0)
    front_red = absorb(two_on_axis(1.0, 2.0), RED_BLUE, cam)[32, 32]
    np.testing.assert_allclose(front_red, [g, 0.0, g * math.exp(-1.0)], rtol=1e-12)
    front_blue = absorb(two_on_axis(2.0, 1.0), RED_BLUE, cam)[32, 32]
    np.testing.assert_allclose(front_blue, [g * math.exp(-1.0), 0.0, g], rtol=1e-12)


def test_equal_depths_are_ordered_by_index():
    # equal keys: ascending (key, index) runs front to back, so particle 0 is in
    # front of particle 1
    cam = axis_camera(65)
    g = 1.0 - math.exp(-1.0)
    img = absorb(two_on_axis(1.5, 1.5), RED_BLUE, cam)[32, 32]
    np.testing.assert_allclose(img, [g, 0.0, g * math.exp(-1.0)], rtol=1e-12)
    p = two_on_axis(1.5, 1.5)
    swapped = {k: v[::-1].copy() for k, v in p.items()}
    img = absorb(swapped, RED_BLUE, cam)[32, 32]
    np.testing.assert_allclose(img, [g * math.exp(-1.0), 0.0, g], rtol=1e-12)


def test_single_particle_source_and_optical_depth():
    # one particle: I = (colour / absorption)(1 - exp(-absorption * I_p * w))
    cam = axis_camera(65)
    h = 2.0 / 32.5
    p = parts_of([0.0, 0.0, 1.0, h, 0.5, 0.0])
    pal = np.array([[1.0, 0.5, 0.25]], dtype=np.float32)
    s2 = (float(np.float32(h)) * 32.5) ** 2
    for alpha in (0.3, 2.0):
        img = absorb(p, pal, cam, alpha)
        for (j, i), d2 in (((32, 32), 0.0), ((32, 33), 1.0), ((33, 34), 5.0)):
            tau = alpha * 0.5 * math.exp(-d2 / s2)
            expect = pal[0].astype(np.float64) / alpha * (1 - math.exp(-tau))
            np.testing.assert_allclose(img[j, i], expect, rtol=1e-12)
        assert np.all(img[32, 40] == 0.0)                 # d = 8 px > r = 6 px


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_emission_equal_to_absorption_gives_the_ea_map(seed):
    # constant grey palette equal to the absorption coefficient: E_p = A_p in
    # every channel, and Eq. 1 gives 1 - exp(-S) whatever the order
    p, cam = random_tiny_scene(seed, n=80)
    for alpha in (0.5, 1.75):           # exact in the FP32 palette
        pal = np.full((1, 3), alpha, dtype=np.float32)
        np.testing.assert_allclose(absorb(p, pal, cam, alpha), oracle.render(p, pal, cam, {"mode": 1}),
                                   rtol=1e-12, atol=1e-15)


def test_small_absorption_gives_the_additive_sum():
    p, cam = random_tiny_scene(4, n=80)
    pal = scenes.ramp_palette()
    add = oracle.render(p, pal, cam)
    thin = absorb(p, pal, cam, 1e-9)
    np.testing.assert_allclose(thin, add, rtol=1e-7, atol=1e-12)


def test_large_absorption_shows_the_nearest_source():
    # opaque particles: a covered pixel takes the source term colour / absorption
    # of its nearest particle
    cam = axis_camera(65)
    img = absorb(two_on_axis(1.0, 2.0), RED_BLUE, cam, 1e3, brightness=1e3)
    np.testing.assert_allclose(img[32, 32], [1e-3, 0.0, 0.0], rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_particle_major_equals_pixel_major_bruteforce(seed):
    p, cam = random_tiny_scene(seed)
    pal = scenes.ramp_palette()
    rec = oracle.project(p, pal, cam)
    assert (rec["cls"] == 0).any() and (rec["cls"] == 1).any()
    for alpha in (0.4, 3.0):
        a = absorb(p, pal, cam, alpha)
        b = absorb(p, pal, cam, alpha, brute=True)
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-300)


def test_input_order_does_not_matter_and_dark_particles_are_invisible():
    p, cam = random_tiny_scene(5, n=120)
    pal = scenes.ramp_palette()
    base = absorb(p, pal, cam, 0.8)
    perm = np.random.default_rng(0).permutation(120)
    np.testing.assert_allclose(absorb({k: v[perm] for k, v in p.items()}, pal, cam, 0.8), base,
                               rtol=1e-12, atol=1e-300)
    dark = {k: np.concatenate([v, v[:30]]) for k, v in p.items()}
    dark["I"][120:] = 0.0
    dark["z"][120:] -= 0.05                       # in front of their bright twins
    np.testing.assert_allclose(absorb(dark, pal, cam, 0.8), base, rtol=1e-12, atol=1e-300)


def test_order_matters_when_sources_differ():
    p, cam = random_tiny_scene(6, n=120)
    pal = scenes.ramp_palette()
    base = absorb(p, pal, cam, 2.0)
    flipped = dict(p)
    flipped["z"] = (0.5 - (p["z"] - 0.5)).astype(np.float32)    # mirror the depths
    assert np.abs(absorb(flipped, pal, cam, 2.0) - base).max() > 1e-3


def test_absorption_must_be_positive():
    p, cam = random_tiny_scene(0, n=5)
    with pytest.raises(ValueError):
        absorb(p, scenes.ramp_palette(), cam, 0.0)
