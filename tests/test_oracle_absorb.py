"""Pins for the oracle's general absorption form (Eq. 1 with E_p != A_p, mode 2).

Across particle p a ray's intensity becomes I exp(-tau) + (E/A)(1 - exp(-tau)),
tau = A w; particles are crossed from the farthest to the nearest.  The pins
fix this against values worked out by hand from Eq. 1 (two particles in front
of each other, both orders, and equal depths), against the E = A special case
(whose solution 1 - exp(-S) is order-free), against the optically thin limit
(small absorption gives the additive sum), against opacity (large absorption
gives the nearest source term), and against the pixel-major brute force.
Particles are ordered by their FP64 depth (two depths closer than one FP32 ulp
are still crossed in their true order); the ambiguity mass gains every
contribution whose depth lies within two FP32 ulps of another contribution to
the same pixel, which bounds what a renderer ordering by an FP32 depth key may
legitimately do differently.  The sampled-pixel oracle equals the full image
(values and mass) at every pixel in every mode.
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


# ---------------------------------------------- FP64 depth order and near ties
def behind_eye_camera(w=65):
    # eye at z = -1 looking down +z: a particle at world z has z_c = z + 1, and
    # the axis lands on the centre of pixel (32, 32) of a 65 x 65, fov 90 image
    return {"eye": (0.0, 0.0, -1.0), "target": (0.0, 0.0, 0.0), "up": (0.0, 1.0, 0.0),
            "fov_y_deg": 90.0, "width": w, "height": w, "z_near": 1e-3}


def sub_ulp_pair():
    # particle 0 (blue) at world z = 1 + 2^-23, particle 1 (red) at z = 1: the
    # depths 2 + 2^-23 and 2 differ in FP64 but both round to 2.0f, so an FP32
    # depth key ties them and would put particle 0 in front by index
    z_blue = float(np.nextafter(np.float32(1.0), np.float32(2.0)))
    return parts_of([[0.0, 0.0, z_blue, 0.2, 1.0, 1.0], [0.0, 0.0, 1.0, 0.2, 1.0, 0.0]])


def test_depths_closer_than_a_float_ulp_are_crossed_in_true_order():
    p = sub_ulp_pair()
    assert np.float32(2.0 + 2.0 ** -23) == np.float32(2.0)   # the keys would tie in FP32
    cam = behind_eye_camera()
    g = 1.0 - math.exp(-1.0)
    # red (index 1) is nearer in FP64: blue is crossed first, then red
    want = [g, 0.0, g * math.exp(-1.0)]
    np.testing.assert_allclose(absorb(p, RED_BLUE, cam)[32, 32], want, rtol=1e-12)
    np.testing.assert_allclose(absorb(p, RED_BLUE, cam, brute=True)[32, 32], want, rtol=1e-12)
    px = np.array([32], np.int32)
    got = oracle.render_pixels(p, RED_BLUE, cam, {"mode": 2, "absorption": 1.0}, px, px)
    np.testing.assert_allclose(got[0], want, rtol=1e-12)


def test_near_tie_mass_covers_the_swapped_order():
    p = sub_ulp_pair()
    cam = behind_eye_camera()
    q = {"mode": 2, "absorption": 1.0}
    B, _ = oracle.ambiguity(p, RED_BLUE, cam, q)
    # both contributions at the centre: brightness * I * w * (largest palette
    # value) = 1 each; the other order differs by g (1 - 1/e) per channel
    np.testing.assert_allclose(B[32, 32], [2.0, 2.0, 2.0], rtol=1e-12)
    g = 1.0 - math.exp(-1.0)
    swapped = np.array([g * math.exp(-1.0), 0.0, g])
    assert np.all(np.abs(swapped - absorb(p, RED_BLUE, cam)[32, 32]) <= B[32, 32])
    # depths 1e-3 apart are never swapped: no mass at the centre (no clip edge there)
    far = dict(p)
    far["z"] = np.array([1.001, 1.0], np.float32)
    B2, _ = oracle.ambiguity(far, RED_BLUE, cam, q)
    assert np.all(B2[32, 32] == 0.0)
    # no mass where only one of the tied pair reaches the pixel: move the blue
    # particle sideways so that its disc misses the red one's far edge
    side = dict(p)
    side["x"] = np.array([-0.3, 0.0], np.float32)      # x_s of blue = 32.5 + 4.875 px
    Bs, _ = oracle.ambiguity(side, RED_BLUE, cam, q)
    rec = oracle.project(side, RED_BLUE, cam, q)
    reach = lambda k, i, j: ((i + 0.5 - rec["xs"][k]) ** 2 + (j + 0.5 - rec["ys"][k]) ** 2
                             <= rec["r"][k] ** 2)
    for i in range(65):
        both = reach(0, i, 32) and reach(1, i, 32)
        only = reach(0, i, 32) != reach(1, i, 32)
        if both:
            assert Bs[32, i, 0] > 0.0
        if only and not np.any(np.abs(np.hypot(i + 0.5 - rec["xs"], 0.0) - rec["r"]) < 1e-3):
            assert Bs[32, i, 0] == 0.0


def near_tie_scene(seed):
    # a tiny scene plus copies of some particles moved by one float ulp in z:
    # exact near ties in depth that share most of their pixels
    p, cam = random_tiny_scene(seed, n=60)
    k = np.arange(0, 60, 3)
    out = {key: np.concatenate([v, v[k]]) for key, v in p.items()}
    out["z"][60:] = np.nextafter(p["z"][k], np.float32(9.0))
    out["s"][60:] = 1.0 - p["s"][k]
    return out, cam


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_selected_pixels_equal_the_full_image_in_every_mode(seed):
    p, cam = near_tie_scene(seed)
    pal = scenes.ramp_palette()
    H, W = cam["height"], cam["width"]
    py, px = np.mgrid[0:H, 0:W]
    px, py = px.ravel().astype(np.int32), py.ravel().astype(np.int32)
    for q in ({}, {"mode": 1}, {"mode": 2, "absorption": 0.7}, {"mode": 2, "absorption": 3.0}):
        img = oracle.render(p, pal, cam, q)
        B, _ = oracle.ambiguity(p, pal, cam, q)
        vals, mass = oracle.render_pixels(p, pal, cam, q, px, py, nthreads=3, with_mass=True)
        np.testing.assert_allclose(vals, img.reshape(-1, 3), rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(mass, B.reshape(-1, 3), rtol=1e-12, atol=1e-300)
    # the near ties do put mass on pixels that no clip edge reaches
    q = {"mode": 2, "absorption": 0.7}
    assert oracle.ambiguity(p, pal, cam, q)[0].sum() > 10 * oracle.ambiguity(
        {k: v[:60] for k, v in p.items()}, pal, cam, q)[0].sum()


def test_selected_pixels_reject_pixels_off_the_image():
    p, cam = random_tiny_scene(0, n=5)
    with pytest.raises(ValueError):
        oracle.render_pixels(p, scenes.ramp_palette(), cam, {"mode": 2}, np.array([cam["width"]]),
                             np.array([0]))
