"""Reference encoder of the 16-bit logarithmic smoothing-length layout
(SPL_ATTR_LOGH16), written with numpy in FP64, used by the tests to check the
library's encoder (spl_encode_attrs) and to hand the oracle the smoothing
lengths that the codes stand for.

Code k of h: round_half_even(4096 (log2 h - log2_min)) clamped to [0, 65535];
the smoothing length of code k is 2^(log2_min + k / 4096), handed to the
oracle rounded to FP32 (the value the GPU's FP32 decode approximates).
"""
import numpy as np

LOG16_STEPS = 4096     # codes per octave


def log16_h(h, log2_min: float) -> np.ndarray:
    k = np.rint((np.log2(np.maximum(np.asarray(h, np.float64), 1e-300)) - log2_min) * LOG16_STEPS)
    return np.clip(k, 0, 65535).astype(np.uint16)


def log16_decoded(codes, log2_min: float) -> np.ndarray:
    return np.exp2(log2_min + codes.astype(np.float64) / LOG16_STEPS).astype(np.float32)
