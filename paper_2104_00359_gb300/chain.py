"""Scene chain above the shading layer (Sec. 3.3.1 and Sec. 3.5): rigid pose
and a linear deformation model producing the vertices, normals and sphere
centres that the shading library consumes, differentiable through torch
autograd and the library's adjoint kernel.

The paper drives its mesh with an embedded graph attached to the spheres and
optimises the global rigid pose and the graph's per-sphere transforms with
the image loss.  Here the deformation is the linearised form used by the
mesh-deformation workload: vertices, normals and sphere centres are affine in
a parameter vector p (v = v0 + A_v p, n = n0 + A_n p, c = c0 + A_c p), then a
6-DoF pose (axis-angle w, translation t) maps them to each view.
"""

from __future__ import annotations

import torch

from .shade import Scene, shade


def rodrigues(w):
    """Rotation matrix exp([w]x) for an axis-angle vector w (3,), smooth at 0."""
    th2 = (w * w).sum()
    z = torch.zeros((), dtype=w.dtype, device=w.device)
    K = torch.stack([torch.stack([z, -w[2], w[1]]), torch.stack([w[2], z, -w[0]]),
                     torch.stack([-w[1], w[0], z])])
    if float(th2) < 1e-8:                     # series: exact to O(th^4)
        a = 1.0 - th2 / 6.0
        b = 0.5 - th2 / 24.0
    else:
        th = torch.sqrt(th2)
        a = torch.sin(th) / th
        b = (1.0 - torch.cos(th)) / th2
    return torch.eye(3, dtype=w.dtype, device=w.device) + a * K + b * (K @ K)


def pose(points, normals, centers, w, t):
    """Apply the rigid pose (w, t): x -> R x + t, n -> R n."""
    R = rodrigues(w)
    return points @ R.T + t, normals @ R.T, centers @ R.T + t


def affine_deform(base, basis, p):
    """base [M, 3] + basis [M, 3, D] @ p [D]."""
    return base + torch.einsum("mcd,d->mc", basis, p)


def render_views(p, poses, model, radii, light, albedo, scenes):
    """Radiance of every view: [V, P, 3].

    model: dict with v0, A_v, n0, A_n, c0, A_c (tensors on the device);
    poses: [V, 6] (axis-angle, translation); scenes: one Scene per view."""
    v = affine_deform(model["v0"], model["A_v"], p)
    n = affine_deform(model["n0"], model["A_n"], p)
    c = affine_deform(model["c0"], model["A_c"], p)
    out = []
    for i, sc in enumerate(scenes):
        pv, pn, pc = pose(v, n, c, poses[i, :3], poses[i, 3:])
        out.append(shade(pv, pn, albedo, pc, radii, light, sc))
    return torch.stack(out)


def make_view_scenes(n_views, centers, radii, light, config):
    """One resident Scene per view (each view's sphere centres differ)."""
    return [Scene(centers.detach(), radii.detach(), light.detach(), config) for _ in range(n_views)]
