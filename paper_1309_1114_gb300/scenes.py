"""Seeded synthetic particle scenes.

This module only draws inputs: particle arrays, cameras and a palette.  It
holds none of the render's arithmetic, and both the CUDA path and the CPU
oracle take their inputs from it.

The paper measures on a Gadget N-body/SPH snapshot of about 400M particles
(Sec. 5) that is not available here; the generators below stand in for its
shape: dense, clustered haloes over a diffuse background, with smoothing
lengths that shrink where the matter is dense.

Scenes (seed in brackets):

* ``uniform``   [1]  200k particles uniform in the unit cube, log-normal h
  (median 0.005, sigma 0.5), I and s uniform on [0, 1); 256^2 image.
* ``clustered`` [2]  10M particles: 70 % from 500 Plummer haloes (halo masses
  with dN/dM ~ M^-1.9 on [1, 1e3], particle count proportional to mass, scale
  radius mapped linearly from M^(1/3) onto [0.002, 0.05], centres uniform in
  [0.1, 0.9]^3), 30 % uniform background; h = clip(eta n^(-1/3), 1e-4, 0.05)
  with n the analytic number density (own halo + background) and
  eta = (3*64/(4 pi))^(1/3); 1024^2 image.
* ``precision`` [3]  100M particles from the clustered generator, attributes
  h, I, s also stored as FP16; 2048^2 image.
* ``orbit``     [4]  20M clustered particles, 64 views on an azimuth orbit of
  radius 2 about +y through the cube centre (step 5.625 deg), resolutions
  cycling 512, 1024, 2048.
* ``pareto``    [5]  400M clustered positions with heavy-tailed smoothing
  lengths h = h_m U^(-1/1.5) (Pareto alpha = 1.5), h_m chosen so that a
  particle at depth 2 has r = 0.5 px, h capped so that r at depth 2 stays
  below the image diagonal; 4096^2 image.

Every camera looks at the cube centre from distance 2 with a 60 deg vertical
field of view; the palette is a 256-entry black-red-yellow-white ramp.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

CUBE_CENTRE = (0.5, 0.5, 0.5)
ETA_SPH = (3.0 * 64.0 / (4.0 * math.pi)) ** (1.0 / 3.0)


def ramp_palette(n: int = 256) -> np.ndarray:
    """n x 3 float32 black -> red -> yellow -> white ramp."""
    t = np.arange(n, dtype=np.float64) / max(n - 1, 1)
    pal = np.stack([np.clip(3 * t, 0, 1), np.clip(3 * t - 1, 0, 1), np.clip(3 * t - 2, 0, 1)], 1)
    return pal.astype(np.float32)


def camera(width: int, height: int | None = None, azimuth_deg: float = 0.0,
           distance: float = 2.0, fov_y_deg: float = 60.0, z_near: float = 1e-3) -> dict:
    """Camera on the orbit about +y through the cube centre."""
    height = width if height is None else height
    a = math.radians(azimuth_deg)
    cx, cy, cz = CUBE_CENTRE
    eye = (cx + distance * math.sin(a), cy, cz - distance * math.cos(a))
    return {"eye": eye, "target": CUBE_CENTRE, "up": (0.0, 1.0, 0.0),
            "fov_y_deg": fov_y_deg, "width": int(width), "height": int(height),
            "z_near": z_near}


@dataclass
class Scene:
    name: str
    parts: dict            # x, y, z, h, I, s: float32 arrays of equal length
    cams: list             # one or more camera dicts
    palette: np.ndarray    # n x 3 float32
    params: dict = field(default_factory=dict)
    fp16: dict | None = None   # h, I, s as float16 when the scene stores them so

    @property
    def n(self) -> int:
        return int(self.parts["x"].shape[0])


def uniform_particles(n: int, seed: int, h_median: float = 0.005, h_sigma: float = 0.5) -> dict:
    rng = np.random.default_rng(seed)
    pos = rng.random((3, n), dtype=np.float32)
    h = np.exp(math.log(h_median) + h_sigma * rng.standard_normal(n)).astype(np.float32)
    inten = rng.random(n, dtype=np.float32)
    s = rng.random(n, dtype=np.float32)
    return {"x": pos[0].copy(), "y": pos[1].copy(), "z": pos[2].copy(), "h": h, "I": inten, "s": s}


def _halo_masses(rng, n_halo, slope=1.9, m0=1.0, m1=1e3):
    u = rng.random(n_halo)
    e = 1.0 - slope
    return (m0 ** e + u * (m1 ** e - m0 ** e)) ** (1.0 / e)


def clustered_positions(n: int, seed: int, n_halo: int = 500, halo_frac: float = 0.7,
                        chunk: int = 1 << 24):
    """Positions (3 x n float32) plus the analytic number density at each one."""
    rng = np.random.default_rng(seed)
    m = _halo_masses(rng, n_halo)
    a = 0.002 + (0.05 - 0.002) * (np.cbrt(m) - 1.0) / (np.cbrt(1e3) - 1.0)
    centres = 0.1 + 0.8 * rng.random((n_halo, 3))
    n_in_halos = int(round(halo_frac * n))
    n_bg = n - n_in_halos
    counts = rng.multinomial(n_in_halos, m / m.sum())
    n_bg_density = float(n_bg)          # background particles per unit volume
    pos = np.empty((3, n), dtype=np.float32)
    dens = np.empty(n, dtype=np.float32)
    # haloes: Plummer radii by inverse CDF, isotropic directions, redraw any
    # point that falls outside the unit cube
    halo_id = np.repeat(np.arange(n_halo, dtype=np.int32), counts)
    start = 0
    while start < n_in_halos:
        stop = min(start + chunk, n_in_halos)
        hid = halo_id[start:stop]
        todo = np.arange(stop - start)
        while todo.size:
            k = todo.size
            u = rng.uniform(0.0, 0.999, k)
            ah = a[hid[todo]]
            rad = ah / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
            cth = rng.uniform(-1.0, 1.0, k)
            phi = rng.uniform(0.0, 2.0 * math.pi, k)
            sth = np.sqrt(1.0 - cth * cth)
            c = centres[hid[todo]]
            p = np.stack([c[:, 0] + rad * sth * np.cos(phi), c[:, 1] + rad * sth * np.sin(phi),
                          c[:, 2] + rad * cth])
            ok = np.all((p >= 0.0) & (p < 1.0), axis=0)
            idx = start + todo[ok]
            pos[:, idx] = p[:, ok]
            nh = counts[hid[todo[ok]]].astype(np.float64)
            rho = 3.0 * nh / (4.0 * math.pi * ah[ok] ** 3) * (1.0 + (rad[ok] / ah[ok]) ** 2) ** -2.5
            dens[idx] = rho + n_bg_density
            todo = todo[~ok]
        start = stop
    pos[:, n_in_halos:] = rng.random((3, n_bg), dtype=np.float32)
    dens[n_in_halos:] = n_bg_density
    return pos, dens


def clustered_particles(n: int, seed: int) -> dict:
    pos, dens = clustered_positions(n, seed)
    rng = np.random.default_rng(seed + 1000)
    h = np.clip(ETA_SPH * np.cbrt(dens.astype(np.float64)) ** -1.0, 1e-4, 0.05).astype(np.float32)
    inten = rng.random(n, dtype=np.float32)
    s = rng.random(n, dtype=np.float32)
    return {"x": pos[0].copy(), "y": pos[1].copy(), "z": pos[2].copy(), "h": h, "I": inten, "s": s}


def pareto_particles(n: int, seed: int, width: int, chi: float = 3.0, alpha: float = 1.5,
                     fov_y_deg: float = 60.0, depth: float = 2.0) -> dict:
    pos, _ = clustered_positions(n, seed)
    rng = np.random.default_rng(seed + 1000)
    f = 0.5 * width / math.tan(math.radians(fov_y_deg) / 2.0)
    h_m = 0.5 * depth / (chi * f)                     # r = 0.5 px at depth 2
    h_cap = math.hypot(width, width) * depth / (chi * f)
    u = 1.0 - rng.random(n)                           # (0, 1]
    h = np.minimum(h_m * u ** (-1.0 / alpha), h_cap).astype(np.float32)
    inten = rng.random(n, dtype=np.float32)
    s = rng.random(n, dtype=np.float32)
    return {"x": pos[0].copy(), "y": pos[1].copy(), "z": pos[2].copy(), "h": h, "I": inten, "s": s}


def fp16_attrs(parts: dict) -> dict:
    """h, I, s rounded to nearest FP16 (as float16 arrays)."""
    return {k: parts[k].astype(np.float16) for k in ("h", "I", "s")}


def widened(parts: dict, f16: dict) -> dict:
    """The particle set as the FP16 path stores it, widened back to float32."""
    out = dict(parts)
    for k in ("h", "I", "s"):
        out[k] = f16[k].astype(np.float32)
    return out


def orbit_cameras(n_views: int = 64, step_deg: float = 5.625, sizes=(512, 1024, 2048)) -> list:
    return [camera(sizes[k % len(sizes)], azimuth_deg=k * step_deg) for k in range(n_views)]


def make(name: str, n: int | None = None, width: int | None = None,
         n_views: int | None = None) -> Scene:
    """Named scene; n, width and n_views shrink it for tests."""
    pal = ramp_palette()
    if name == "uniform":
        n = 200_000 if n is None else n
        w = 256 if width is None else width
        return Scene(name, uniform_particles(n, 1), [camera(w)], pal)
    if name == "clustered":
        n = 10_000_000 if n is None else n
        w = 1024 if width is None else width
        return Scene(name, clustered_particles(n, 2), [camera(w)], pal)
    if name == "precision":
        n = 100_000_000 if n is None else n
        w = 2048 if width is None else width
        parts = clustered_particles(n, 3)
        return Scene(name, parts, [camera(w)], pal, fp16=fp16_attrs(parts))
    if name == "orbit":
        n = 20_000_000 if n is None else n
        nv = 64 if n_views is None else n_views
        cams = orbit_cameras(nv)
        if width is not None:
            cams = [dict(c, width=max(8, c["width"] * width // 2048),
                         height=max(8, c["height"] * width // 2048)) for c in cams]
        return Scene(name, clustered_particles(n, 4), cams, pal)
    if name == "pareto":
        n = 400_000_000 if n is None else n
        w = 4096 if width is None else width
        return Scene(name, pareto_particles(n, 5, w), [camera(w)], pal)
    raise KeyError(name)
