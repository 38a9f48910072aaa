"""Pins for the FP64 oracle: closed forms, invariants and brute force.

Each test fixes part of the oracle against something other than the oracle
itself -- a pinhole-camera value worked out by hand, the integral of Eq. 2,
the order independence that Sec. 2 derives from E_p = A_p, a symmetry, or the
pixel-major brute-force formulation -- so that a dropped term, a wrong sign,
a transposed operand or an off-by-one bounding box fails one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1309_1114_gb300 import scenes


def axis_camera(w, h=None, fov=90.0):
    """Eye at the origin looking down +z with +y up (right = -x)."""
    return {"eye": (0.0, 0.0, 0.0), "target": (0.0, 0.0, 1.0), "up": (0.0, 1.0, 0.0),
            "fov_y_deg": fov, "width": w, "height": w if h is None else h, "z_near": 1e-3}


def parts_of(rows):
    rows = np.asarray(rows, dtype=np.float64).reshape(-1, 6)
    return {k: rows[:, i].astype(np.float32) for i, k in enumerate(("x", "y", "z", "h", "I", "s"))}


CONST_PAL = np.array([[1.0, 0.5, 0.25]], dtype=np.float32)


# ---------------------------------------------------------------- projection
def test_projection_closed_form():
    # fov 90 deg, 64 px: f = 32.  world (0.1, 0.2, 1.0): x_c = -0.1, y_c = 0.2,
    # z_c = 1 -> x_s = 32 - 3.2 = 28.8, y_s = 32 - 6.4 = 25.6;
    # sigma_s = h f / z = 2 (h = 1/16), r = 3 sigma_s = 6 (Eq. 7).
    rec = oracle.project(parts_of([0.1, 0.2, 1.0, 1 / 16, 1.0, 0.0]), CONST_PAL, axis_camera(64))
    assert rec["cls"][0] == 1
    assert rec["xs"][0] == pytest.approx(28.8, abs=1e-6)
    assert rec["ys"][0] == pytest.approx(25.6, abs=1e-6)
    assert rec["sigma"][0] == pytest.approx(2.0, rel=1e-6)
    assert rec["r"][0] == pytest.approx(6.0, rel=1e-6)


def test_radius_scales_inversely_with_depth_and_linearly_with_pixels():
    # Eq. 7: r(p) is linear in sigma_p and in N_pix, and (through A(p)) in 1/z.
    p = parts_of([[0.0, 0.0, 1.0, 0.01, 1, 0], [0.0, 0.0, 2.0, 0.01, 1, 0],
                  [0.0, 0.0, 4.0, 0.02, 1, 0]])
    r64 = oracle.project(p, CONST_PAL, axis_camera(64))["r"]
    r128 = oracle.project(p, CONST_PAL, axis_camera(128))["r"]
    assert r64[0] / r64[1] == pytest.approx(2.0, rel=1e-6)
    assert r64[2] == pytest.approx(r64[1], rel=1e-6)
    np.testing.assert_allclose(r128 / r64, 2.0, rtol=1e-6)
    rc = oracle.project(p, CONST_PAL, axis_camera(64), {"chi": 2.0})["r"]
    np.testing.assert_allclose(rc / r64, 2.0 / 3.0, rtol=1e-12)


def test_axis_point_maps_to_image_centre_for_any_view():
    for az in (0.0, 37.0, 180.0, 290.0):
        cam = scenes.camera(200, 150, azimuth_deg=az)
        rec = oracle.project(parts_of([0.5, 0.5, 0.5, 0.01, 1, 0]), CONST_PAL, cam)
        assert rec["xs"][0] == pytest.approx(100.0, abs=1e-9)
        assert rec["ys"][0] == pytest.approx(75.0, abs=1e-9)


def test_look_at_basis_is_orthonormal():
    cam = scenes.camera(64, azimuth_deg=33.0)
    v = oracle.view_info(cam)
    B = np.stack([v["right"], v["up"], v["fwd"]])
    np.testing.assert_allclose(B @ B.T, np.eye(3), atol=1e-14)
    assert v["f"] == pytest.approx(32.0 / math.tan(math.radians(30.0)), rel=1e-14)


# ------------------------------------------------------------------ palette
def test_palette_nodes_midpoints_and_clamping():
    pal = np.array([[0, 0, 0], [1, 0.5, 0], [1, 1, 1]], dtype=np.float32)
    s = [0.0, 0.5, 1.0, 0.25, 0.75, -3.0, 7.0]
    rows = [[0.0, 0.0, 1.0, 0.01, 1.0, v] for v in s]
    e = oracle.project(parts_of(rows), pal, axis_camera(32))["e"]
    expect = [[0, 0, 0], [1, 0.5, 0], [1, 1, 1], [0.5, 0.25, 0], [1, 0.75, 0.5],
              [0, 0, 0], [1, 1, 1]]
    np.testing.assert_allclose(e, expect, atol=1e-7)


def test_palette_normalisation_range_and_intensity_scale():
    pal = np.array([[0, 0, 0], [1, 1, 1]], dtype=np.float32)
    rows = [[0.0, 0.0, 1.0, 0.01, 2.0, 15.0]]
    e = oracle.project(parts_of(rows), pal, axis_camera(32),
                       {"s_min": 10.0, "s_max": 20.0, "brightness": 3.0})["e"]
    np.testing.assert_allclose(e[0], [3.0, 3.0, 3.0], rtol=1e-12)   # 3 * 2 * 0.5


# ---------------------------------------------------------- single particle
def test_single_particle_on_pixel_centre():
    # 65 x 65, fov 90 deg: f = 32.5, the axis point lands on x_s = y_s = 32.5,
    # the centre of pixel (32, 32).  h chosen for sigma_s = 2, so r = 6.
    cam = axis_camera(65)
    h = 2.0 / 32.5
    img = oracle.render(parts_of([0.0, 0.0, 1.0, h, 0.5, 0.0]), CONST_PAL, cam)
    e = np.array([0.5, 0.25, 0.125])
    # sigma_s from the stored FP32 h (about 2 px)
    s2 = (float(np.float32(h)) * 32.5 / math.tan(math.radians(45.0))) ** 2
    assert s2 == pytest.approx(4.0, rel=1e-6)
    np.testing.assert_allclose(img[32, 32], e, rtol=1e-12)
    np.testing.assert_allclose(img[32, 33], e * math.exp(-1 / s2), rtol=1e-12)
    np.testing.assert_allclose(img[31, 32], e * math.exp(-1 / s2), rtol=1e-12)
    np.testing.assert_allclose(img[33, 33], e * math.exp(-2 / s2), rtol=1e-12)
    np.testing.assert_allclose(img[32, 37], e * math.exp(-25 / s2), rtol=1e-12)
    # (32+5, 32+4): d^2 = 41 > r^2 = 36 -> clipped; (32+4, 32+4): d^2 = 32 kept
    assert np.all(img[36, 37] == 0.0)
    np.testing.assert_allclose(img[36, 36], e * math.exp(-32 / s2), rtol=1e-12)
    yy, xx = np.mgrid[0:65, 0:65]
    d2 = (xx - 32) ** 2 + (yy - 32) ** 2
    assert np.all(img[d2 > 36.5] == 0.0)
    assert np.all(img[d2 < 35.5] > 0.0)


def test_integrated_gaussian_of_isolated_particle():
    # Integral of Eq. 2 over the clipped disc: e * pi sigma^2 (1 - exp(-chi^2)).
    cam = axis_camera(129)
    for sig in (2.5, 4.0, 7.0):
        h = sig / 64.5
        img = oracle.render(parts_of([0.013, -0.021, 1.0, h, 1.0, 0.0]), CONST_PAL, cam)
        total = img[..., 0].sum()
        expect = math.pi * sig * sig * (1 - math.exp(-9.0))
        # lattice-point discrepancy on the clip circle bounds the residual
        bound = 2 * math.pi * 3 * sig * math.exp(-9.0) / (math.pi * sig * sig) + 1e-6
        assert abs(total / expect - 1) < bound


def test_point_rule_deposits_emission_in_one_pixel():
    # r <= r_sml = 0.5: the location is all that is computed (Sec. 4.1)
    cam = axis_camera(64)                     # f = 32
    h = 0.4 / 3 / 32                          # r = 0.4 px
    img = oracle.render(parts_of([0.05, -0.07, 1.0, h, 0.5, 0.0]), CONST_PAL, cam)
    # x_s = 32 - 1.6 = 30.4, y_s = 32 + 2.24 = 34.24
    nz = np.argwhere(img[..., 0] != 0)
    assert nz.tolist() == [[34, 30]]
    np.testing.assert_allclose(img[34, 30], [0.5, 0.25, 0.125], rtol=1e-12)


def test_class_threshold_switches_between_point_and_splat():
    cam = axis_camera(64)
    h = 0.6 / 3 / 32                          # r = 0.6 px -> splat
    p = parts_of([0.0, 0.0, 1.0, h, 1.0, 0.0])
    assert oracle.project(p, CONST_PAL, cam)["cls"][0] == 1
    assert oracle.project(p, CONST_PAL, cam, {"r_sml": 0.7})["cls"][0] == 0


# ------------------------------------------------------------- activeness
def test_inactive_behind_camera_and_outside_view():
    cam = axis_camera(64)
    rows = [[0.0, 0.0, -1.0, 0.01, 1, 0],     # behind the eye
            [0.0, 0.0, 0.0005, 0.01, 1, 0],   # inside the near plane
            [5.0, 0.0, 1.0, 0.001, 1, 0]]     # far off screen, small
    rec = oracle.project(parts_of(rows), CONST_PAL, cam)
    assert list(rec["cls"]) == [-2, -2, -2]
    assert np.all(oracle.render(parts_of(rows), CONST_PAL, cam) == 0.0)


def test_particle_centred_off_screen_still_contributes():
    # Fig. 4 (particle 2): outside the field of view yet active, because its
    # disc reaches the image.
    cam = axis_camera(64)                     # f = 32
    rows = [[1.1, 0.0, 1.0, 0.1, 1.0, 0.0]]   # x_s = 32 - 35.2 = -3.2, r = 9.6
    rec = oracle.project(parts_of(rows), CONST_PAL, cam)
    assert rec["xs"][0] < 0 and rec["cls"][0] == 1
    img = oracle.render(parts_of(rows), CONST_PAL, cam)
    assert img[32, 0, 0] > 0 and img[32, 7, 0] == 0


# --------------------------------------------------------------- invariants
def random_tiny_scene(seed, n=60, w=32, h=24):
    rng = np.random.default_rng(seed)
    cam = {"eye": (0.5, 0.5, -1.5), "target": (0.5, 0.5, 0.5), "up": (0.0, 1.0, 0.0),
           "fov_y_deg": 60.0, "width": w, "height": h, "z_near": 1e-3}
    rows = np.column_stack([rng.uniform(-0.3, 1.3, n), rng.uniform(-0.3, 1.3, n),
                            rng.uniform(-1.4, 1.0, n), np.exp(rng.uniform(-6, -1.5, n)),
                            rng.random(n), rng.random(n)])
    return parts_of(rows), cam


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_particle_major_equals_pixel_major_bruteforce(seed):
    p, cam = random_tiny_scene(seed)
    pal = scenes.ramp_palette()
    rec = oracle.project(p, pal, cam)
    assert (rec["cls"] == 0).any() and (rec["cls"] == 1).any() and (rec["cls"] == -2).any()
    a = oracle.render(p, pal, cam)
    b = oracle.render_bruteforce(p, pal, cam)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-300)


def test_pixel_sample_equals_full_image_and_threads_agree():
    p, cam = random_tiny_scene(7, n=400, w=48, h=40)
    pal = scenes.ramp_palette()
    full = oracle.render(p, pal, cam)
    full4 = oracle.render(p, pal, cam, nthreads=4)
    np.testing.assert_allclose(full4, full, rtol=1e-12, atol=1e-300)
    rng = np.random.default_rng(3)
    px, py = rng.integers(0, 48, 50), rng.integers(0, 40, 50)
    vals = oracle.render_pixels(p, pal, cam, {}, px, py, nthreads=3)
    np.testing.assert_allclose(vals, full[py, px], rtol=1e-12, atol=1e-300)


def test_linearity_and_order_independence():
    # E_p = A_p makes the result independent of integration order (Sec. 2);
    # the additive image is then linear in the emission.
    p, cam = random_tiny_scene(11, n=300)
    pal = scenes.ramp_palette()
    full = oracle.render(p, pal, cam)
    half = {k: v[:150] for k, v in p.items()}
    rest = {k: v[150:] for k, v in p.items()}
    np.testing.assert_allclose(oracle.render(half, pal, cam) + oracle.render(rest, pal, cam),
                               full, rtol=1e-12, atol=1e-14)
    perm = np.random.default_rng(5).permutation(300)
    np.testing.assert_allclose(oracle.render({k: v[perm] for k, v in p.items()}, pal, cam),
                               full, rtol=1e-12, atol=1e-14)
    scaled = dict(p, I=(p["I"] * np.float32(0.5)))
    np.testing.assert_allclose(oracle.render(scaled, pal, cam), 0.5 * full, rtol=1e-12,
                               atol=1e-300)
    np.testing.assert_allclose(oracle.render(p, pal, cam, {"brightness": 3.0}), 3 * full,
                               rtol=1e-12, atol=1e-300)


def test_on_axis_particle_gives_symmetric_image():
    cam = axis_camera(64)                     # axis lands on x_s = y_s = 32
    img = oracle.render(parts_of([0.0, 0.0, 1.0, 3.3 / 32, 1.0, 0.0]), CONST_PAL, cam)
    np.testing.assert_array_equal(img, img[:, ::-1])
    np.testing.assert_array_equal(img, img[::-1, :])
    np.testing.assert_array_equal(img, img.transpose(1, 0, 2))
    assert img[..., 0].max() > 0


def test_constant_palette_separates_colour():
    p, cam = random_tiny_scene(2, n=200)
    img = oracle.render(p, CONST_PAL, cam)
    np.testing.assert_allclose(img[..., 1], 0.5 * img[..., 0], rtol=1e-12)
    np.testing.assert_allclose(img[..., 2], 0.25 * img[..., 0], rtol=1e-12)


def test_absorption_mode_is_pointwise_map_of_additive_sum():
    # Eq. 1 with E = A and I(0) = 0 integrates to I = 1 - exp(-sum).
    p, cam = random_tiny_scene(4, n=200)
    pal = scenes.ramp_palette()
    add = oracle.render(p, pal, cam)
    ea = oracle.render(p, pal, cam, {"mode": 1})
    np.testing.assert_allclose(ea, -np.expm1(-add), rtol=1e-12, atol=1e-300)


# ---------------------------------------------------------------- ambiguity
def test_ambiguity_marks_clip_edge_class_edge_and_integer_points():
    cam = axis_camera(65)                     # f = 32.5, axis on pixel centre 32
    # clip edge: sigma_s = 2, r = 6 -> pixel (38, 32) is on the circle
    B, n = oracle.ambiguity(parts_of([0.0, 0.0, 1.0, 2.0 / 32.5, 1.0, 0.0]), CONST_PAL, cam)
    assert B[32, 38, 0] > 0 and B[32, 26, 0] > 0 and B[32, 32, 0] == 0 and n == 0
    # point exactly on a pixel corner (x_s = 32 in a 64 px image): two pixels each way
    cam64 = axis_camera(64)
    B, n = oracle.ambiguity(parts_of([0.0, 0.0, 1.0, 0.3 / 3 / 32, 1.0, 0.0]), CONST_PAL, cam64)
    assert n == 1
    assert sorted(map(tuple, np.argwhere(B[..., 0] > 0).tolist())) == [
        (31, 31), (31, 32), (32, 31), (32, 32)]
    # class edge: r = r_sml exactly -> point pixel and the whole disc are marked
    B, n = oracle.ambiguity(parts_of([0.01, 0.013, 1.0, 0.5 / 3 / 32, 1.0, 0.0]),
                            CONST_PAL, cam64)
    assert n == 1 and (B[..., 0] > 0).sum() >= 1


# ----------------------------------------------------------- tile features
def test_tile_features_hand_counted():
    cam = axis_camera(64)                     # f = 32, 16 px tiles -> 4 x 4
    # sigma_s = 2, r = 6 at (28.8, 25.6): pixel-centre box i in [23, 34],
    # j in [20, 31] -> tiles (x 1..2, y 1): areas 9*12 and 3*12; radius bin
    # floor(log2(6 / 0.5)) = 3.
    f = oracle.tile_features(parts_of([0.1, 0.2, 1.0, 1 / 16, 1.0, 0.0]), CONST_PAL, cam, {}, 16)
    assert f.shape == (16, 32)
    nz = {t: f[t] for t in range(16) if f[t].any()}
    assert sorted(nz) == [5, 6]
    for t, a in ((5, 108.0), (6, 36.0)):
        assert nz[t][3] == pytest.approx(math.log1p(1.0))
        assert nz[t][16 + 3] == pytest.approx(math.log1p(a))
        assert np.count_nonzero(nz[t]) == 2


def test_tile_membership_needs_the_disc_not_just_the_box():
    cam = axis_camera(64)                     # f = 32, 16 px tiles -> 4 x 4
    # x_s = y_s = 8 (centre of tile 0), r = 9: the box reaches tiles 0, 1, 4, 5,
    # but the nearest pixel centre of tile 5, (16.5, 16.5), is 8.5 sqrt(2) > 9 away
    f = oracle.tile_features(parts_of([0.75, 0.75, 1.0, 9.0 / 96.0, 1.0, 0.0]), CONST_PAL, cam, {}, 16)
    assert sorted(np.nonzero(f[:, :16].sum(1))[0].tolist()) == [0, 1, 4]


def test_non_finite_or_negative_inputs_are_inactive():
    cam = axis_camera(64)
    nan, inf = float("nan"), float("inf")
    rows = [[nan, 0.0, 1.0, 0.01, 1, 0], [0.0, 0.0, inf, 0.01, 1, 0], [0.0, 0.0, 1.0, nan, 1, 0],
            [0.0, 0.0, 1.0, 0.01, inf, 0], [0.0, 0.0, 1.0, 0.01, 1, nan], [0.0, 0.0, 1.0, -0.01, 1, 0]]
    rec = oracle.project(parts_of(rows), CONST_PAL, cam)
    assert list(rec["cls"]) == [-2] * 6
    img = oracle.render(parts_of(rows + [[0.0, 0.0, 1.0, 0.05, 1.0, 0.0]]), CONST_PAL, cam)
    assert np.isfinite(img).all() and img.max() > 0
