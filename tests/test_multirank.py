"""Frames split over ranks (gloo, world size 2, CPU): the composition of
partial images that the paper's MPI version uses (Sec. 2) reproduces the
whole frame, and the timing reduction takes the slowest rank.  Here the
partial images come from the oracle (no GPU); tests/test_gpu_shard.py renders
them with the library and applies the library's E = A map after the sum."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

from paper_1309_1114_gb300 import scenes, shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc = scenes.make("uniform", n=3000, width=48)
        cam = dict(sc.cams[0], height=40)
        lo, hi = shard.partition(sc.n, world)[rank]
        part = {k: v[lo:hi] for k, v in sc.parts.items()}
        img = torch.from_numpy(oracle.render(part, sc.palette, cam))
        shard.allreduce_image(img)
        ea = -np.expm1(-img.numpy())          # the E = A map after the sum
        slowest = shard.max_over_ranks(10.0 + rank)
        if rank == 0:
            np.save(out + ".add.npy", img.numpy())
            np.save(out + ".ea.npy", ea)
            np.save(out + ".t.npy", np.array([slowest]))
    finally:
        dist.destroy_process_group()


def test_partition_covers_every_particle_once():
    for n, w in ((0, 1), (10, 3), (1001, 4), (7, 8)):
        parts = shard.partition(n, w)
        assert parts[0][0] == 0 and parts[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        sizes = [hi - lo for lo, hi in parts]
        assert max(sizes) - min(sizes) <= 1


def test_two_rank_partial_images_compose_to_the_frame(tmp_path):
    import oracle
    out = str(tmp_path / "r")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    sc = scenes.make("uniform", n=3000, width=48)
    cam = dict(sc.cams[0], height=40)
    full = oracle.render(sc.parts, sc.palette, cam)
    np.testing.assert_allclose(np.load(out + ".add.npy"), full, rtol=1e-12, atol=1e-14)
    full_ea = oracle.render(sc.parts, sc.palette, cam, {"mode": 1})
    np.testing.assert_allclose(np.load(out + ".ea.npy"), full_ea, rtol=1e-12, atol=1e-14)
    assert np.load(out + ".t.npy")[0] == 11.0
