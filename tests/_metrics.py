"""Error metric for GPU images against the FP64 oracle.

Per channel c, with M_c = max over pixels of |o_c| (the oracle image), a
pixel's error is max(0, |g - o| - B) / max(|o|, 1e-3 M_c), where B is the
oracle's ambiguity mass (contributions whose clip test, class test or point
pixel may legitimately flip between FP32 and FP64).  The image error is the
maximum over pixels and channels.
"""
import numpy as np


def rel_pixel_error(g, o, B=None, M=None, floor=1e-3):
    g = np.asarray(g, dtype=np.float64).reshape(-1, 3)
    o = np.asarray(o, dtype=np.float64).reshape(-1, 3)
    if M is None:
        M = np.abs(o).max(0)
    M = np.asarray(M, dtype=np.float64)
    den = np.maximum(np.abs(o), floor * M)
    den = np.where(den > 0, den, 1e-300)
    diff = np.abs(g - o)
    if B is not None:
        diff = np.clip(diff - np.asarray(B, dtype=np.float64).reshape(-1, 3), 0, None)
    if diff.size == 0:
        return 0.0
    return float(np.max(diff / den))
