"""Training and use of the tile-cost network that orders the render's work items.

The renderer records, per work item, 32 features (per radius bin: log1p of
its particle count and of the tile pixels inside their boxes) and the SM
clock cycles its CTA spent (``Renderer.set_recording``).  ``train`` fits the
network 32 -> 64 (ReLU) -> 1 to log(cycles) with the library's own GPU
kernels (``spl_mlp_train``: forward, back-propagation and Adam on the
device); ``fit_count_heuristic`` fits the fallback a + b log1p(entries), which
also serves as the yardstick of the network's prediction error.  Device
buffers are torch CUDA tensors; all arithmetic on them runs in the library.
"""
from __future__ import annotations

import ctypes as C
import json
import math

import numpy as np

from . import splotch as S

NFEAT, NHID = 32, 64


def collect(renderer, torch, cams: list, max_items: int = 1 << 20):
    """Render every camera once with recording on; returns (feat, logc) CUDA tensors."""
    feats, logcs = [], []
    renderer.set_recording(True)
    try:
        for cam in cams:
            renderer.set_camera(cam)
            img = torch.empty((cam["height"], cam["width"], 3), device="cuda")
            renderer.render(img)
            f = torch.empty((max_items, NFEAT), device="cuda")
            t = torch.empty((max_items,), device="cuda")
            n = renderer.samples(f, t)
            feats.append(f[:n].clone())
            logcs.append(t[:n].clone())
    finally:
        renderer.set_recording(False)
    return torch.cat(feats), torch.cat(logcs)


def entries_of(feat) -> np.ndarray:
    """Total particle count of each sample (the count bins hold log1p(count))."""
    f = feat.detach().cpu().numpy().astype(np.float64)
    return np.expm1(f[:, :16]).sum(1)


def fit_count_heuristic(feat, logc) -> np.ndarray:
    """Least-squares a, b of log(cycles) ~ a + b log1p(entries)."""
    x = np.log1p(entries_of(feat))
    y = logc.detach().cpu().numpy().astype(np.float64)
    A = np.stack([np.ones_like(x), x], 1)
    coef, *_ = np.linalg.lstsq(A, y, rcond=None)
    return coef.astype(np.float32)


def init_theta(seed: int = 0, bias: float = 0.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    th = np.zeros(S.SPL_MLP_NPARAM, dtype=np.float32)
    th[:NHID * NFEAT] = rng.normal(0.0, math.sqrt(2.0 / NFEAT), NHID * NFEAT)
    th[NHID * NFEAT + NHID:NHID * NFEAT + 2 * NHID] = rng.normal(0.0, math.sqrt(1.0 / NHID), NHID)
    th[-1] = bias
    return th


def train(feat, logc, steps: int = 3000, lr: float = 3e-3, seed: int = 0, stream=None):
    """Full-batch Adam on the GPU; returns (theta as float32 numpy, losses)."""
    x = feat.contiguous()
    t = logc.contiguous()
    theta = init_theta(seed, bias=float(t.mean().item()))
    losses = np.zeros(max(steps, 1), dtype=np.float32)
    S.check(S.load_library().spl_mlp_train(x.data_ptr(), t.data_ptr(), int(t.numel()),
                                           theta.ctypes.data, int(steps), float(lr),
                                           losses.ctypes.data, stream), "spl_mlp_train")
    return theta, losses[:steps]


def predict(theta, feat, torch, stream=None):
    """Network output for CUDA features (one kernel launch)."""
    th = torch.from_numpy(np.ascontiguousarray(theta, dtype=np.float32)).cuda()
    y = torch.empty((feat.shape[0],), device="cuda")
    S.check(S.load_library().spl_mlp_forward(th.data_ptr(), feat.contiguous().data_ptr(),
                                             int(feat.shape[0]), y.data_ptr(), stream),
            "spl_mlp_forward")
    torch.cuda.synchronize()
    return y


def rmse(pred, logc) -> float:
    p = np.asarray(pred, dtype=np.float64)
    y = np.asarray(logc, dtype=np.float64)
    return float(np.sqrt(np.mean((p - y) ** 2)))


def save(path: str, theta, heur) -> None:
    with open(path, "w") as f:
        json.dump({"nparam": int(S.SPL_MLP_NPARAM), "theta": np.asarray(theta, np.float32).tolist(),
                   "heur": np.asarray(heur, np.float32).tolist()}, f)


def load(path: str):
    with open(path) as f:
        d = json.load(f)
    if d.get("nparam") != S.SPL_MLP_NPARAM:
        raise ValueError("model file: wrong parameter count")
    return np.asarray(d["theta"], np.float32), np.asarray(d["heur"], np.float32)
