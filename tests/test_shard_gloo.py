"""Sharding across ranks on CPU (gloo, world size 2): each rank computes its
slice's gradients (here with the FP64 oracle standing in for the device), the
scene-level sums are all-reduced, and the result equals the unsharded
gradients; per-point gradients are the slices of the unsharded ones."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2104_00359_gb300.shard import shard_range


def test_shard_range_covers_once():
    for n in (0, 1, 7, 1000, 262144):
        for w in (1, 2, 3, 8):
            spans = [shard_range(n, r, w) for r in range(w)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[i][1] == spans[i + 1][0] for i in range(w - 1))
            sizes = [e - b for b, e in spans]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_path):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    from oracle import shs_oracle as O
    from paper_2104_00359_gb300 import synthetic as S
    from paper_2104_00359_gb300.shard import sharded_backward
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc = S.random_scene(55, 301, 6, 3)
    dB = np.random.default_rng(2).normal(size=(301, 3))
    cfg = O.Config(n_bands=3)

    def local(begin, end):
        g = O.shade_backward(cfg, sc["points"][begin:end], sc["normals"][begin:end], sc["albedo"][begin:end],
                             sc["centers"], sc["radii"], sc["light"], dB[begin:end])
        return {k: torch.from_numpy(np.ascontiguousarray(g[k])) for k in
                ("d_light", "d_centers", "d_radii", "d_albedo", "d_points")}

    g = sharded_backward(local, 301, rank, world)
    torch.save({k: v.numpy() for k, v in g.items()}, f"{out_path}.{rank}")
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_scene_gradients_match_unsharded(tmp_path):
    from oracle import shs_oracle as O
    from paper_2104_00359_gb300 import synthetic as S
    world = 2
    out = str(tmp_path / "g")
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    sc = S.random_scene(55, 301, 6, 3)
    dB = np.random.default_rng(2).normal(size=(301, 3))
    full = O.shade_backward(O.Config(n_bands=3), sc["points"], sc["normals"], sc["albedo"], sc["centers"],
                            sc["radii"], sc["light"], dB)
    parts = [torch.load(f"{out}.{r}", weights_only=False) for r in range(world)]
    for r, g in enumerate(parts):
        for k in ("d_light", "d_centers", "d_radii"):
            np.testing.assert_allclose(g[k], full[k], rtol=1e-12, atol=1e-12)
        b, e = shard_range(301, r, world)
        np.testing.assert_allclose(g["d_albedo"], full["d_albedo"][b:e], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(g["d_points"], full["d_points"][b:e], rtol=1e-12, atol=1e-14)
