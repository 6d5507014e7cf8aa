"""Data-parallel sharding of one scene's shading points across ranks.

Shading points are independent (Sec. 3.2, Eq. 8 is per point), so each rank
shades a contiguous slice of the G-buffer with the scene (spheres, lighting)
replicated; the forward pass needs no exchange.  The adjoint's scene-level
gradients (lighting, sphere centres and radii) are sums over all points and
need one sum all-reduce of 3K + 4N floats; per-point gradients stay local.
"""

from __future__ import annotations

import torch


def shard_range(n_points: int, rank: int, world: int):
    """[begin, end) of this rank's contiguous slice (sizes differ by at most 1)."""
    base, extra = divmod(int(n_points), int(world))
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


SCENE_GRADS = ("d_light", "d_centers", "d_radii")


def sharded_backward(local_backward, n_points, rank, world, group=None):
    """Run ``local_backward(begin, end)`` on this rank's slice and sum the
    scene-level gradients over ranks (one all-reduce of a flat buffer).

    ``local_backward`` returns a dict with the gradient arrays (torch tensors)
    for its slice; per-point entries are returned unchanged."""
    import torch.distributed as dist
    begin, end = shard_range(n_points, rank, world)
    g = local_backward(begin, end)
    present = [k for k in SCENE_GRADS if g.get(k) is not None]
    if world > 1 and present:
        flat = torch.cat([g[k].reshape(-1) for k in present])
        dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
        off = 0
        for k in present:
            n = g[k].numel()
            g[k] = flat[off:off + n].view_as(g[k])
            off += n
    return g


def scene_backward_on_slice(scene, points, normals, albedo, d_radiance, saved_views=None, want=None):
    """A ``local_backward`` for the CUDA library: the slice [begin, end) of
    device tensors through ``Scene.backward`` (recomputing f on the slice)."""
    want = want or scene.ALL

    def run(begin, end):
        return scene.backward(points[begin:end], normals[begin:end], albedo[begin:end],
                              d_radiance[begin:end], saved=None, want=want)
    return run
