"""Writes the stored expected values under tests/golden/ (calls only oracle/).

Run from the repository root:  python tests/golden/make_golden.py
The inputs are literal numbers written here; the expected pixels come from
the FP64 oracle.  The paper prints no image values, so every stored value in
this folder is an oracle value for the literal inputs below.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

# Five particles in the spirit of Fig. 4: a splat straddling two tiles, a
# point-rule particle, one centred off screen whose disc reaches the image,
# one behind the camera and one large splat.  Rows: x, y, z, h, I, s.
ROWS = [
    [0.50, 0.50, 0.50, 0.010, 0.8, 0.30],
    [0.30, 0.62, 0.20, 0.0004, 1.0, 0.90],
    [2.05, 0.40, 0.60, 0.080, 0.6, 0.55],
    [0.40, 0.40, -2.00, 0.020, 1.0, 0.10],
    [0.70, 0.35, 0.70, 0.400, 0.3, 0.75],
]
CAM = {"eye": [0.5, 0.5, -1.5], "target": [0.5, 0.5, 0.5], "up": [0.0, 1.0, 0.0],
       "fov_y_deg": 60.0, "width": 48, "height": 40, "z_near": 1e-3}
PAL = [[0.0, 0.0, 0.0], [1.0, 0.2, 0.0], [1.0, 1.0, 0.3], [1.0, 1.0, 1.0]]


def main():
    rows = np.asarray(ROWS, dtype=np.float32)
    parts = {k: rows[:, i] for i, k in enumerate(("x", "y", "z", "h", "I", "s"))}
    pal = np.asarray(PAL, dtype=np.float32)
    img = oracle.render(parts, pal, CAM)
    rec = oracle.project(parts, pal, CAM)
    out = {
        "source": "oracle FP64 render of the literal inputs in make_golden.py",
        "rows_xyzhIs": ROWS, "camera": CAM, "palette": PAL, "params": {},
        "cls": rec["cls"].tolist(), "xs": rec["xs"].tolist(), "ys": rec["ys"].tolist(),
        "r": rec["r"].tolist(),
        "image": img.tolist(),
    }
    with open(os.path.join(HERE, "five_particles.json"), "w") as f:
        json.dump(out, f, indent=None, separators=(",", ":"))
        f.write("\n")


if __name__ == "__main__":
    main()
