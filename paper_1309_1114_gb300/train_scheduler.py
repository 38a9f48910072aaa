"""Train the tile-cost network on the renderer's own item timings.

  python -m paper_1309_1114_gb300.train_scheduler [--out PATH] [--samples N] [--steps K]

Renders the clustered (10M, 1024^2), precision (100M, 2048^2, FP16
attributes) and orbit (20M, six views at 512/1024/2048) scenes with recording
on, draws N samples (default 10000) of (item features, log SM cycles), trains
the network with the library's GPU kernels, fits the count heuristic on the
same samples, and writes both to PATH (default models/tile_cost.json next to
this file) together with their held-out prediction errors.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "models", "tile_cost.json")


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--samples", type=int, default=10000)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=3e-3)
    args = ap.parse_args(argv)

    import torch
    from . import scenes, scheduler
    from .splotch import Renderer

    r = Renderer(0, torch.cuda.current_stream().cuda_stream)
    feats, logcs, sources = [], [], []
    for name, views in (("clustered", 1), ("precision", 1), ("orbit", 6)):
        sc = scenes.make(name)
        r.load(sc.parts, sc.fp16 if name == "precision" else None)
        r.set_colormap(sc.palette)
        r.set_params()
        f, t = scheduler.collect(r, torch, sc.cams[:views])
        feats.append(f)
        logcs.append(t)
        sources.append(f"{name}: {f.shape[0]} items")
        del sc
    f = torch.cat(feats)
    t = torch.cat(logcs)
    g = torch.Generator().manual_seed(0)
    idx = torch.randperm(f.shape[0], generator=g)[: min(args.samples, f.shape[0])].cuda()
    f, t = f[idx].contiguous(), t[idx].contiguous()
    ntr = int(0.8 * f.shape[0])
    theta, losses = scheduler.train(f[:ntr], t[:ntr], steps=args.steps, lr=args.lr)
    heur = scheduler.fit_count_heuristic(f[:ntr], t[:ntr])
    te = t[ntr:].cpu().numpy()
    err_mlp = scheduler.rmse(scheduler.predict(theta, f[ntr:], torch).cpu().numpy(), te)
    err_cnt = scheduler.rmse(heur[0] + heur[1] * np.log1p(scheduler.entries_of(f[ntr:])), te)
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    scheduler.save(args.out, theta, heur)
    with open(args.out) as fh:
        d = json.load(fh)
    d.update({"samples": int(f.shape[0]), "train": ntr, "sources": sources,
              "loss_first": float(losses[0]), "loss_last": float(losses[-1]),
              "heldout_rmse_network": err_mlp, "heldout_rmse_count": err_cnt})
    with open(args.out, "w") as fh:
        json.dump(d, fh)
    print(json.dumps({k: v for k, v in d.items() if k not in ("theta",)}))
    r.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
