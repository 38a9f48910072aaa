"""FP64 CPU oracle for the Splotch per-frame render -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``splotch_oracle.c`` (plain C,
double precision) through ctypes and shares no code with the CUDA library.

The rules it implements, with the paper passages they come from, are listed in
the header comment of ``splotch_oracle.c``.  Parity status per function:

* ``project``, ``render``, ``render_pixels``, ``render_bruteforce``: pinned by
  closed forms, invariants and brute force in ``tests/test_oracle_pins.py``.
* ``ambiguity``: pinned by constructed edge cases (clip edge, class edge,
  integer positions) in the same file.
* ``mlp_forward``, ``mlp_loss_grad``, ``adam_step``: pinned by finite
  differences, a closed-form one-unit case and a hand-stepped Adam update in
  ``tests/test_oracle_mlp.py``.
* ``tile_features``: pinned by hand-counted cases in
  ``tests/test_oracle_pins.py``.
* colouring options (per-particle components ``cr``, ``cg``, ``cb`` in the
  particle dict; ``par["log"]`` bit 1 = log10 of I, bit 2 = log10 of s):
  pinned by a hand value, the constant-palette equivalence, channel
  separation and exact powers of ten in ``tests/test_oracle_colour.py``.
* ``render`` / ``render_bruteforce`` / ``render_pixels`` with ``mode = 2`` (Eq. 1
  with independent emission and absorption over particles in FP64 depth order):
  pinned by hand-worked two-particle cases (both orders, equal depths, depths
  closer than one FP32 ulp), the E = A special case, the optically thin and
  opaque limits, input-order invariance, the pixel-major brute force and the
  full image at every pixel in ``tests/test_oracle_absorb.py``.
* ``ambiguity`` in mode 2 (near-tie mass of particles within two FP32 ulps in
  depth) and ``render_pixels(..., with_mass=True)``: pinned by the near-tie
  cases and by the full-image mass at every pixel in the same file.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "splotch_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


class _Camera(C.Structure):
    _fields_ = [("eye", C.c_double * 3), ("target", C.c_double * 3),
                ("up", C.c_double * 3), ("fov_y_deg", C.c_double),
                ("width", C.c_int), ("height", C.c_int), ("z_near", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("chi", C.c_double), ("sigma_per_h", C.c_double),
                ("s_box", C.c_double), ("r_sml", C.c_double),
                ("brightness", C.c_double), ("s_min", C.c_double),
                ("s_max", C.c_double), ("mode", C.c_int), ("absorption", C.c_double),
                ("log_flags", C.c_int), ("cr", C.c_void_p), ("cg", C.c_void_p),
                ("cb", C.c_void_p)]


def build(force: bool = False) -> str:
    """Compile splotch_oracle.c into liboracle.so (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            dp, fp, ip, lp = (C.POINTER(C.c_double), C.POINTER(C.c_float),
                              C.POINTER(C.c_int), C.POINTER(C.c_long))
            cam, par = C.POINTER(_Camera), C.POINTER(_Params)
            parts = [C.c_long, fp, fp, fp, fp, fp, fp, fp, C.c_int, cam, par]
            lib.orc_project.argtypes = parts + [dp, dp, dp, dp, dp, ip]
            lib.orc_render.argtypes = parts + [dp, C.c_int]
            lib.orc_render_pixels.argtypes = parts + [C.c_long, ip, ip, dp, C.c_void_p, C.c_int]
            lib.orc_render_bruteforce.argtypes = parts + [dp]
            lib.orc_ambiguity.argtypes = parts + [dp, lp]
            lib.orc_view_info.argtypes = [cam, dp]
            lib.orc_mlp_nparam.restype = C.c_int
            lib.orc_mlp_forward.argtypes = [dp, C.c_long, dp, dp]
            lib.orc_mlp_loss_grad.argtypes = [dp, C.c_long, dp, dp, dp]
            lib.orc_mlp_loss_grad.restype = C.c_double
            lib.orc_adam_step.argtypes = [dp, dp, dp, dp, C.c_long, C.c_long,
                                          C.c_double, C.c_double, C.c_double, C.c_double]
            lib.orc_tile_features.argtypes = parts + [C.c_int, C.c_double, dp]
            _lib = lib
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def _camera(cam: dict) -> _Camera:
    c = _Camera()
    c.eye[:] = [float(v) for v in cam["eye"]]
    c.target[:] = [float(v) for v in cam["target"]]
    c.up[:] = [float(v) for v in cam["up"]]
    c.fov_y_deg = float(cam["fov_y_deg"])
    c.width = int(cam["width"])
    c.height = int(cam["height"])
    c.z_near = float(cam.get("z_near", 1e-3))
    return c


def _params(par: dict | None) -> _Params:
    par = dict(par or {})
    q = _Params()
    q.chi = float(par.get("chi", 3.0))
    q.sigma_per_h = float(par.get("sigma_per_h", 1.0))
    q.s_box = float(par.get("s_box", 1.0))
    q.r_sml = float(par.get("r_sml", 0.5))
    q.brightness = float(par.get("brightness", 1.0))
    q.s_min = float(par.get("s_min", 0.0))
    q.s_max = float(par.get("s_max", 1.0))
    q.mode = int(par.get("mode", 0))
    q.absorption = float(par.get("absorption", 1.0))
    q.log_flags = int(par.get("log", 0))
    return q


def _args(parts: dict, palette, cam, par):
    """Marshal the particle arrays (x, y, z, h, I, s) and settings."""
    arrs = [_f32(parts[k]) for k in ("x", "y", "z", "h", "I", "s")]
    n = arrs[0].shape[0]
    for a in arrs:
        if a.shape != (n,):
            raise ValueError("particle arrays must be 1-D and of equal length")
    pal = _f32(palette).reshape(-1)
    if pal.size % 3 or pal.size == 0:
        raise ValueError("palette must hold n*3 floats")
    c, q = _camera(cam), _params(par)
    rgb = None
    if "cr" in parts:
        # per-particle colour components replace the palette (Sec. 2)
        rgb = [_f32(parts[k]) for k in ("cr", "cg", "cb")]
        if any(a.shape != (n,) for a in rgb):
            raise ValueError("colour components must be 1-D and of the particle count")
        q.cr, q.cg, q.cb = (a.ctypes.data for a in rgb)
    keep = (arrs, pal, c, q, rgb)
    args = [n] + [_ptr(a, C.c_float) for a in arrs] + [_ptr(pal, C.c_float), pal.size // 3,
                                                       C.byref(c), C.byref(q)]
    return n, keep, args


def view_info(cam: dict) -> dict:
    lib = _load()
    out = np.zeros(13)
    c = _camera(cam)
    if lib.orc_view_info(C.byref(c), _ptr(out, C.c_double)):
        raise ValueError("invalid camera")
    return {"right": out[0:3], "up": out[3:6], "fwd": out[6:9], "f": out[9],
            "half_w": out[10], "half_h": out[11], "z_near": out[12]}


def project(parts, palette, cam, par=None) -> dict:
    """Per-particle FP64 records: xs, ys, sigma, r, e (n x 3), cls."""
    lib = _load()
    n, keep, args = _args(parts, palette, cam, par)
    out = {k: np.zeros(n) for k in ("xs", "ys", "sigma", "r")}
    e = np.zeros((n, 3))
    cls = np.zeros(n, dtype=np.int32)
    rc = lib.orc_project(*args, *[_ptr(out[k], C.c_double) for k in ("xs", "ys", "sigma", "r")],
                         _ptr(e, C.c_double), _ptr(cls, C.c_int))
    if rc:
        raise ValueError(f"orc_project failed ({rc})")
    out["e"], out["cls"] = e, cls
    return out


def render(parts, palette, cam, par=None, nthreads: int = 1) -> np.ndarray:
    """Full H x W x 3 FP64 image, particle-major."""
    lib = _load()
    n, keep, args = _args(parts, palette, cam, par)
    img = np.zeros((int(cam["height"]), int(cam["width"]), 3))
    rc = lib.orc_render(*args, _ptr(img, C.c_double), int(nthreads))
    if rc:
        raise ValueError(f"orc_render failed ({rc})")
    return img


def render_pixels(parts, palette, cam, par, px, py, nthreads: int = 1, with_mass: bool = False):
    """Values (k x 3) of the pixels (px[k], py[k]), pixel-major; with_mass also
    returns their ambiguity mass (k x 3), equal to ``ambiguity``'s there.  Mode 2
    sorts every pixel's particles by FP64 depth and crosses them (Eq. 1)."""
    lib = _load()
    n, keep, args = _args(parts, palette, cam, par)
    px = np.ascontiguousarray(px, dtype=np.int32)
    py = np.ascontiguousarray(py, dtype=np.int32)
    out = np.zeros((px.size, 3))
    B = np.zeros((px.size, 3)) if with_mass else None
    rc = lib.orc_render_pixels(*args, px.size, _ptr(px, C.c_int), _ptr(py, C.c_int),
                               _ptr(out, C.c_double), None if B is None else B.ctypes.data,
                               int(nthreads))
    if rc:
        raise ValueError(f"orc_render_pixels failed ({rc})")
    return (out, B) if with_mass else out


def render_bruteforce(parts, palette, cam, par=None) -> np.ndarray:
    """Every pixel against every particle (tiny scenes only)."""
    lib = _load()
    n, keep, args = _args(parts, palette, cam, par)
    img = np.zeros((int(cam["height"]), int(cam["width"]), 3))
    rc = lib.orc_render_bruteforce(*args, _ptr(img, C.c_double))
    if rc:
        raise ValueError(f"orc_render_bruteforce failed ({rc})")
    return img


def ambiguity(parts, palette, cam, par=None):
    """(B image H x W x 3, number of class/pixel-ambiguous particles)."""
    lib = _load()
    n, keep, args = _args(parts, palette, cam, par)
    B = np.zeros((int(cam["height"]), int(cam["width"]), 3))
    cnt = C.c_long(0)
    rc = lib.orc_ambiguity(*args, _ptr(B, C.c_double), C.byref(cnt))
    if rc:
        raise ValueError(f"orc_ambiguity failed ({rc})")
    return B, int(cnt.value)


def tile_features(parts, palette, cam, par, tile: int, area_scale: float = 1.0) -> np.ndarray:
    """Per-tile 32-bin cost features (n_tiles x 32), FP64."""
    lib = _load()
    n, keep, args = _args(parts, palette, cam, par)
    ntx = (int(cam["width"]) + tile - 1) // tile
    nty = (int(cam["height"]) + tile - 1) // tile
    out = np.zeros((nty * ntx, 32))
    rc = lib.orc_tile_features(*args, int(tile), float(area_scale), _ptr(out, C.c_double))
    if rc:
        raise ValueError(f"orc_tile_features failed ({rc})")
    return out


# ---- tile-cost network ------------------------------------------------------
def mlp_nparam() -> int:
    return int(_load().orc_mlp_nparam())


def mlp_forward(theta, x) -> np.ndarray:
    lib = _load()
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 32)
    y = np.zeros(x.shape[0])
    lib.orc_mlp_forward(_ptr(theta, C.c_double), x.shape[0], _ptr(x, C.c_double),
                        _ptr(y, C.c_double))
    return y


def mlp_loss_grad(theta, x, t):
    lib = _load()
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 32)
    t = np.ascontiguousarray(t, dtype=np.float64)
    g = np.zeros_like(theta)
    loss = lib.orc_mlp_loss_grad(_ptr(theta, C.c_double), x.shape[0], _ptr(x, C.c_double),
                                 _ptr(t, C.c_double), _ptr(g, C.c_double))
    return float(loss), g


def adam_step(theta, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam update of float64 arrays theta, m, v."""
    lib = _load()
    for a in (theta, m, v):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise ValueError("theta, m, v must be contiguous float64")
    grad = np.ascontiguousarray(grad, dtype=np.float64)
    lib.orc_adam_step(_ptr(theta, C.c_double), _ptr(grad, C.c_double), _ptr(m, C.c_double),
                      _ptr(v, C.c_double), theta.size, int(t), lr, beta1, beta2, eps)
