"""ctypes binding of ``include/splotch.h`` (argument marshalling only).

Every function of the C ABI is exposed under its own name (``spl_create``,
``spl_render`` ...); ``Renderer`` is a small convenience wrapper that takes
torch tensors and numpy arrays.  All computation happens in the CUDA library
``lib/libsplotch.so``; if it is missing or cannot be loaded, importing the
library raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libsplotch.so")

SPL_OK, SPL_EINVAL, SPL_ENOMEM, SPL_ECUDA, SPL_ESTATE, SPL_EDEVICE, SPL_ELIMIT = range(7)
SPL_MEM_HOST, SPL_MEM_DEVICE = 0, 1
SPL_ATTR_F32, SPL_ATTR_F16, SPL_ATTR_F16_IS, SPL_ATTR_LOGH16 = 0, 1, 2, 3
SPL_MODE_ADDITIVE, SPL_MODE_EA, SPL_MODE_ABSORB = 0, 1, 2
SPL_LOG_I, SPL_LOG_S = 1, 2
SPL_SCHED_NONE, SPL_SCHED_COUNT, SPL_SCHED_MLP = 0, 1, 2
SPL_MLP_NPARAM = 2177


class spl_particles(C.Structure):
    _fields_ = [("n", C.c_int64), ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("h", C.c_void_p), ("I", C.c_void_p), ("s", C.c_void_p),
                ("attr_type", C.c_int32), ("mem_space", C.c_int32),
                ("cr", C.c_void_p), ("cg", C.c_void_p), ("cb", C.c_void_p),
                ("h_log2_min", C.c_float)]


class spl_camera(C.Structure):
    _fields_ = [("eye", C.c_double * 3), ("target", C.c_double * 3), ("up", C.c_double * 3),
                ("fov_y_deg", C.c_double), ("width", C.c_int32), ("height", C.c_int32),
                ("z_near", C.c_double)]


class spl_params(C.Structure):
    _fields_ = [("chi", C.c_double), ("sigma_per_h", C.c_double), ("s_box", C.c_double),
                ("r_sml", C.c_double), ("brightness", C.c_double), ("tile_px", C.c_int32),
                ("r_small", C.c_double), ("r_large", C.c_double), ("mode", C.c_int32),
                ("sched", C.c_int32), ("absorption", C.c_double), ("log_flags", C.c_int32)]


class spl_stats(C.Structure):
    _fields_ = [("n_particles", C.c_int64), ("n_active", C.c_int64), ("n_point", C.c_int64),
                ("n_small", C.c_int64), ("n_medium", C.c_int64), ("n_large", C.c_int64),
                ("n_entries", C.c_int64 * 4), ("n_tiles", C.c_int32), ("tile_px", C.c_int32),
                ("ms_raster", C.c_float), ("ms_bin", C.c_float), ("ms_tile", C.c_float),
                ("ms_large", C.c_float), ("ms_epilogue", C.c_float), ("ms_total", C.c_float),
                ("timed_frames", C.c_int64), ("sum_ms", C.c_double * 6), ("launches", C.c_int32)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["n_entries"] = list(self.n_entries)
        d["sum_ms"] = list(self.sum_ms)
        return d


_P = C.c_void_p
_SIGS = {
    "spl_create": [C.POINTER(C.c_void_p), C.c_int, _P],
    "spl_destroy": [_P],
    "spl_load_particles": [_P, C.POINTER(spl_particles)],
    "spl_load_particles_as": [_P, C.POINTER(spl_particles), C.c_int32, C.c_float],
    "spl_encode_attrs": [_P, _P, _P, _P, C.c_int64, C.c_int32, C.c_float, _P, _P, _P, _P],
    "spl_apply_ea": [_P, _P, C.c_int64, _P],
    "spl_set_camera": [_P, C.POINTER(spl_camera)],
    "spl_set_colormap": [_P, _P, C.c_int32, C.c_float, C.c_float],
    "spl_default_params": [C.POINTER(spl_params)],
    "spl_set_params": [_P, C.POINTER(spl_params)],
    "spl_get_params": [_P, C.POINTER(spl_params)],
    "spl_render": [_P, _P, _P],
    "spl_render_host": [_P, _P],
    "spl_render_stream": [_P, C.POINTER(spl_particles), C.c_int64, _P, _P],
    "spl_render_batch": [_P, C.POINTER(spl_camera), C.c_int32, C.POINTER(C.c_void_p), _P],
    "spl_get_stats": [_P, C.POINTER(spl_stats)],
    "spl_set_timing": [_P, C.c_int32],
    "spl_set_graph": [_P, C.c_int32],
    "spl_get_records": [_P, C.c_int64, _P, _P, _P, _P, _P],
    "spl_count_work": [_P, C.POINTER(C.c_int64)],
    "spl_set_model": [_P, _P, _P],
    "spl_set_recording": [_P, C.c_int32],
    "spl_get_samples": [_P, _P, _P, C.c_int64, C.POINTER(C.c_int64)],
    "spl_mlp_nparam": [],
    "spl_mlp_forward": [_P, _P, C.c_int64, _P, _P],
    "spl_mlp_loss_grad": [_P, _P, _P, C.c_int64, _P, _P, _P],
    "spl_mlp_adam": [_P, _P, _P, _P, C.c_int64, C.c_int64, C.c_float, C.c_float, C.c_float,
                     C.c_float, _P],
    "spl_mlp_train": [_P, _P, C.c_int64, _P, C.c_int32, C.c_float, _P, _P],
    "spl_autotune": [_P, C.POINTER(spl_camera), C.c_int32, C.POINTER(C.c_void_p), C.c_int32,
                     C.POINTER(spl_params), C.POINTER(C.c_float)],
    "spl_render_noalloc": [C.POINTER(spl_particles), C.POINTER(spl_camera), C.POINTER(spl_params),
                           _P, C.c_int32, C.c_float, C.c_float, _P, C.c_int32, _P],
    "spl_error_string": [C.c_int],
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libsplotch.so (raises OSError when it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise OSError(f"CUDA library not built: {path} (run __graft_entry__.build())")
        lib = C.CDLL(path)
        for name, args in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = C.c_char_p if name == "spl_error_string" else C.c_int
        _lib = lib
    return _lib


class SplotchError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = load_library().spl_error_string(code).decode()
        super().__init__(f"{where}: {msg} ({code})")


def check(code: int, where: str) -> None:
    if code != SPL_OK:
        raise SplotchError(code, where)


def _exported(name):
    def call(*args):
        return getattr(load_library(), name)(*args)
    call.__name__ = name
    return call


for _name in _SIGS:
    globals()[_name] = _exported(_name)


# ---------------------------------------------------------------- helpers
def make_camera(cam: dict) -> spl_camera:
    c = spl_camera()
    c.eye[:] = [float(v) for v in cam["eye"]]
    c.target[:] = [float(v) for v in cam["target"]]
    c.up[:] = [float(v) for v in cam["up"]]
    c.fov_y_deg = float(cam["fov_y_deg"])
    c.width = int(cam["width"])
    c.height = int(cam["height"])
    c.z_near = float(cam.get("z_near", 1e-3))
    return c


def default_params(**over) -> spl_params:
    q = spl_params()
    check(load_library().spl_default_params(C.byref(q)), "spl_default_params")
    for k, v in over.items():
        if not hasattr(q, k):
            raise KeyError(k)
        setattr(q, k, v)
    return q


def _ptr(t):
    """Address of a torch tensor or a numpy array."""
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data


class Renderer:
    """One library context on one device and stream.

    ``load`` takes a dict of six arrays (x, y, z, h, I, s); numpy arrays are
    copied from host memory, CUDA tensors from device memory.  ``render``
    writes into a caller-owned CUDA float32 tensor of shape (H, W, 3).
    """

    def __init__(self, device: int = 0, stream: int | None = None):
        lib = load_library()
        h = C.c_void_p()
        check(lib.spl_create(C.byref(h), int(device), stream), "spl_create")
        self._h = h
        self.device = device
        self._keep = None

    def close(self):
        if getattr(self, "_h", None):
            load_library().spl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @staticmethod
    def _particles(parts: dict, fp16: dict | None, h_log2_min: float | None = None):
        """spl_particles for parts (and the arrays it points to, kept alive by
        the caller).  fp16 (optional) holds binary16 arrays that replace parts'
        h, I and s (SPL_ATTR_F16), or only I and s (SPL_ATTR_F16_IS); with
        h_log2_min, fp16["h"] holds 16-bit logarithmic codes (SPL_ATTR_LOGH16)."""
        src = dict(parts)
        attr = SPL_ATTR_F32
        if fp16 is not None:
            src.update(fp16)
            attr = SPL_ATTR_F16 if "h" in fp16 else SPL_ATTR_F16_IS
            if h_log2_min is not None:
                if "h" not in fp16:
                    raise ValueError("logarithmic h codes go in fp16['h']")
                attr = SPL_ATTR_LOGH16
        arrs = [src[k] for k in ("x", "y", "z", "h", "I", "s")]
        on_dev = [hasattr(a, "is_cuda") and a.is_cuda for a in arrs]
        if any(on_dev) and not all(on_dev):
            raise ValueError("particle arrays must all be on the host or all on the device")
        n = int(arrs[0].shape[0])
        if not any(on_dev):
            arrs = [np.ascontiguousarray(a) for a in arrs]
            want_h = {SPL_ATTR_F16: np.float16, SPL_ATTR_LOGH16: np.uint16}.get(attr, np.float32)
            wants = [np.float32] * 3 + [want_h] + \
                [np.float16 if attr != SPL_ATTR_F32 else np.float32] * 2
            for a, want in zip(arrs, wants):
                if a.dtype != want or a.shape != (n,):
                    raise ValueError("particle arrays: wrong dtype or shape")
        p = spl_particles(n, *[_ptr(a) for a in arrs], attr,
                          SPL_MEM_DEVICE if any(on_dev) else SPL_MEM_HOST)
        if h_log2_min is not None:
            p.h_log2_min = float(h_log2_min)
        if "cr" in src:
            # per-particle colour components (FP32, same memory space as the rest)
            rgb = [src[k] for k in ("cr", "cg", "cb")]
            if any(hasattr(a, "is_cuda") and a.is_cuda for a in rgb) != any(on_dev):
                raise ValueError("colour components must live where the particles do")
            if not any(on_dev):
                rgb = [np.ascontiguousarray(a, dtype=np.float32) for a in rgb]
            if any(tuple(a.shape) != (n,) for a in rgb):
                raise ValueError("colour components: wrong shape")
            p.cr, p.cg, p.cb = (_ptr(a) for a in rgb)
            arrs = arrs + rgb
        return p, arrs

    def load(self, parts: dict, fp16: dict | None = None, h_log2_min: float | None = None,
             store_as: int | None = None):
        """Load particles (host or device arrays; see _particles for fp16).  With
        store_as (an SPL_ATTR_* layout) the FP32 attributes of parts are
        converted by the library (spl_load_particles_as; h_log2_min for
        SPL_ATTR_LOGH16)."""
        if store_as is not None:
            if fp16 is not None:
                raise ValueError("store_as converts FP32 attributes: no fp16 arrays")
            p, keep = self._particles(parts, None)
            check(load_library().spl_load_particles_as(
                self._h, C.byref(p), int(store_as),
                float(h_log2_min if h_log2_min is not None else 0.0)), "spl_load_particles_as")
            del keep
            return
        p, keep = self._particles(parts, fp16, h_log2_min)
        check(load_library().spl_load_particles(self._h, C.byref(p)), "spl_load_particles")
        del keep

    def encode_attrs(self, h, I, s, store_as: int, h_log2_min: float = 0.0, stream=None) -> dict:
        """Library conversion of FP32 CUDA tensors h, I, s into the storage
        layout store_as; returns new CUDA tensors {"h", "I", "s"} (float32,
        float16 or int16 holding the uint16 codes)."""
        import torch
        n = int(h.numel())
        for t in (h, I, s):
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.numel() == n):
                raise ValueError("encode_attrs: contiguous float32 CUDA tensors of equal size")
        f16 = store_as != SPL_ATTR_F32
        dt_h = {SPL_ATTR_F16: torch.float16, SPL_ATTR_LOGH16: torch.int16}.get(store_as, torch.float32)
        out = {"h": torch.empty(n, dtype=dt_h, device=h.device),
               "I": torch.empty(n, dtype=torch.float16 if f16 else torch.float32, device=h.device),
               "s": torch.empty(n, dtype=torch.float16 if f16 else torch.float32, device=h.device)}
        check(load_library().spl_encode_attrs(self._h, h.data_ptr(), I.data_ptr(), s.data_ptr(), n,
                                              int(store_as), float(h_log2_min), out["h"].data_ptr(),
                                              out["I"].data_ptr(), out["s"].data_ptr(), stream),
              "spl_encode_attrs")
        return out

    def apply_ea(self, image, stream=None):
        """E = A map 1 - exp(-v) of every value of a CUDA float32 tensor, in place."""
        if not (image.is_cuda and image.is_contiguous()) or image.dtype.itemsize != 4:
            raise ValueError("apply_ea: contiguous float32 CUDA tensor")
        check(load_library().spl_apply_ea(self._h, image.data_ptr(), int(image.numel()), stream),
              "spl_apply_ea")
        return image

    def get_params(self) -> dict:
        q = spl_params()
        check(load_library().spl_get_params(self._h, C.byref(q)), "spl_get_params")
        return {k: getattr(q, k) for k, _ in q._fields_}

    def render_stream(self, parts: dict, chunk: int, image, fp16: dict | None = None,
                      stream: int | None = None, h_log2_min: float | None = None):
        """Out-of-core render of host particle arrays (page-locked for overlap)
        in chunks of `chunk` particles into the device image (fp16 and
        h_log2_min as in load)."""
        p, keep = self._particles(parts, fp16, h_log2_min)
        check(load_library().spl_render_stream(self._h, C.byref(p), int(chunk), image.data_ptr(),
                                               stream), "spl_render_stream")
        del keep
        return image

    def set_camera(self, cam: dict):
        c = make_camera(cam)
        check(load_library().spl_set_camera(self._h, C.byref(c)), "spl_set_camera")
        self.cam = dict(cam)

    def set_colormap(self, pal, s_min: float = 0.0, s_max: float = 1.0):
        pal = np.ascontiguousarray(pal, dtype=np.float32).reshape(-1, 3)
        check(load_library().spl_set_colormap(self._h, pal.ctypes.data, pal.shape[0],
                                              float(s_min), float(s_max)), "spl_set_colormap")

    def set_params(self, **kw):
        q = default_params(**kw)
        check(load_library().spl_set_params(self._h, C.byref(q)), "spl_set_params")

    def set_timing(self, on: bool = True):
        check(load_library().spl_set_timing(self._h, int(bool(on))), "spl_set_timing")

    def set_graph(self, on: bool = True):
        check(load_library().spl_set_graph(self._h, int(bool(on))), "spl_set_graph")

    def render(self, image, stream: int | None = None):
        check(load_library().spl_render(self._h, image.data_ptr(), stream), "spl_render")
        return image

    def render_host(self, out: np.ndarray | None = None) -> np.ndarray:
        shape = (self.cam["height"], self.cam["width"], 3)
        if out is None:
            out = np.empty(shape, dtype=np.float32)
        if out.shape != shape or out.dtype != np.float32 or not out.flags.c_contiguous:
            raise ValueError("render_host: out must be a contiguous float32 (H, W, 3) array")
        check(load_library().spl_render_host(self._h, out.ctypes.data), "spl_render_host")
        return out

    def render_batch(self, cams: list, images: list, stream: int | None = None):
        arr = (spl_camera * len(cams))(*[make_camera(c) for c in cams])
        ptrs = (C.c_void_p * len(images))(*[im.data_ptr() for im in images])
        check(load_library().spl_render_batch(self._h, arr, len(cams), ptrs, stream),
              "spl_render_batch")
        return images

    def autotune(self, cams: list, images: list, reps: int = 2) -> tuple:
        arr = (spl_camera * len(cams))(*[make_camera(c) for c in cams])
        ptrs = (C.c_void_p * len(images))(*[im.data_ptr() for im in images])
        best = spl_params()
        ms = C.c_float(0.0)
        check(load_library().spl_autotune(self._h, arr, len(cams), ptrs, int(reps), C.byref(best),
                                          C.byref(ms)), "spl_autotune")
        return {k: getattr(best, k) for k, _ in best._fields_}, float(ms.value)

    def set_model(self, theta=None, heur=None):
        th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float32)
        hu = None if heur is None else np.ascontiguousarray(heur, dtype=np.float32)
        if th is not None and th.size != SPL_MLP_NPARAM:
            raise ValueError("theta must hold SPL_MLP_NPARAM floats")
        check(load_library().spl_set_model(self._h, None if th is None else th.ctypes.data,
                                           None if hu is None else hu.ctypes.data), "spl_set_model")

    def set_recording(self, on: bool = True):
        check(load_library().spl_set_recording(self._h, int(bool(on))), "spl_set_recording")

    def samples(self, feat, logc) -> int:
        """Copy the last render's item samples into CUDA tensors; returns the count."""
        n = C.c_int64(0)
        check(load_library().spl_get_samples(self._h, feat.data_ptr(), logc.data_ptr(),
                                             int(logc.numel()), C.byref(n)), "spl_get_samples")
        return int(n.value)

    def stats(self) -> dict:
        s = spl_stats()
        check(load_library().spl_get_stats(self._h, C.byref(s)), "spl_get_stats")
        return s.as_dict()

    def count_work(self) -> list:
        out = (C.c_int64 * 4)()
        check(load_library().spl_count_work(self._h, out), "spl_count_work")
        return list(out)

    def records(self, n: int) -> dict:
        xs = np.zeros(n)
        ys = np.zeros(n)
        r = np.zeros(n, np.float32)
        e = np.zeros((n, 3), np.float32)
        cls = np.zeros(n, np.int32)
        check(load_library().spl_get_records(self._h, n, xs.ctypes.data, ys.ctypes.data,
                                             r.ctypes.data, e.ctypes.data, cls.ctypes.data),
              "spl_get_records")
        return {"xs": xs, "ys": ys, "r": r, "e": e, "cls": cls}
