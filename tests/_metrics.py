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


def pick_pixels(g, tile=32, n_windows=2, n_bright=64, n_random=448, seed=0):
    """Pixels of an H x W x 3 image g at which a full-size render is compared
    with the oracle, pixel by pixel:

    * whole tile-sized windows centred on a tile corner, so that each covers
      the seams between four tiles: the first at the corner nearest the
      brightest pixel (a halo core: crowded tiles split into many work items),
      the others at random corners;
    * the n_bright brightest pixels (by the sum of the channels);
    * n_random pixels drawn uniformly.

    Returns (px, py) as int32 arrays without repeats."""
    g = np.asarray(g)
    H, W = g.shape[:2]
    rng = np.random.default_rng(seed)
    lum = g.reshape(H * W, -1).sum(1)
    picks = []
    by, bx = divmod(int(np.argmax(lum)), W)
    corners = [(int(round(bx / tile)) * tile, int(round(by / tile)) * tile)]
    for _ in range(n_windows - 1):
        corners.append((int(rng.integers(0, W // tile + 1)) * tile,
                        int(rng.integers(0, H // tile + 1)) * tile))
    half = tile // 2
    for cx, cy in corners[:n_windows]:
        x0 = min(max(cx - half, 0), max(W - tile, 0))
        y0 = min(max(cy - half, 0), max(H - tile, 0))
        yy, xx = np.mgrid[y0:min(y0 + tile, H), x0:min(x0 + tile, W)]
        picks.append((yy * W + xx).ravel())
    if n_bright:
        picks.append(np.argsort(lum)[-n_bright:])
    if n_random:
        picks.append(rng.integers(0, H * W, n_random))
    idx = np.unique(np.concatenate(picks))
    return (idx % W).astype(np.int32), (idx // W).astype(np.int32)
