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

import ctypes

import torch

from . import _lib
from ._lib import check, ptr
from .shade import Scene, shade


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, name):
    if not (t.is_cuda and t.dtype == torch.float32):
        raise TypeError(f"{name} must be a float32 CUDA tensor")
    return t.contiguous()


class DeformPose(torch.autograd.Function):
    """x = R(w) (base + basis p) + t (t dropped for directions), forward and
    adjoint in the library's chain kernels; gradients flow to p and the pose
    (base and basis are constants of the model)."""

    @staticmethod
    def forward(ctx, base, basis, p, pose, direction):
        lib = _lib.load()
        base, basis, p, pose = (_dev(t.detach(), n) for t, n in
                                ((base, "base"), (basis, "basis"), (p, "p"), (pose, "pose")))
        M, D = int(base.shape[0]), int(p.shape[0])
        if tuple(basis.shape) != (M, 3, D) or tuple(pose.shape) != (6,):
            raise ValueError(f"basis {tuple(basis.shape)} / pose {tuple(pose.shape)} do not match M={M}, D={D}")
        x = torch.empty((M, 3), dtype=torch.float32, device=base.device)
        check(lib.shs_chain_forward(ptr(base), ptr(basis), M, D, ptr(p), ptr(pose), int(direction), None, ptr(x),
                                    _stream()), "shs_chain_forward")
        ctx.save_for_backward(base, basis, p, pose)
        ctx.direction = int(direction)
        return x

    @staticmethod
    def backward(ctx, dx):
        lib = _lib.load()
        base, basis, p, pose = ctx.saved_tensors
        M, D = int(base.shape[0]), int(p.shape[0])
        dx = _dev(dx, "dx")
        d_p = torch.empty((D,), dtype=torch.float32, device=base.device)
        d_pose = torch.empty((6,), dtype=torch.float32, device=base.device)
        nbytes = int(lib.shs_chain_workspace_bytes(M, D))
        ws = torch.empty((max(nbytes, 16) + 3) // 4, dtype=torch.float32, device=base.device)
        check(lib.shs_chain_backward(ptr(base), ptr(basis), M, D, ptr(p), ptr(pose), ctx.direction, ptr(dx),
                                     ptr(d_p), ptr(d_pose), ptr(ws), ws.numel() * 4, _stream()),
              "shs_chain_backward")
        return None, None, d_p, d_pose, None


def deform_pose(base, basis, p, pose, direction=False):
    """R(w) (base + basis p) + t for pose = (w, t) [6]; direction drops t."""
    return DeformPose.apply(base, basis, p, pose, bool(direction))


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
    """Apply the rigid pose (w, t) to already deformed arrays: x -> R x + t,
    n -> R n (torch ops; the rendering path uses the fused chain kernels)."""
    R = rodrigues(w)
    return points @ R.T + t, normals @ R.T, centers @ R.T + t


def affine_deform(base, basis, p):
    """base [M, 3] + basis [M, 3, D] @ p [D] (torch ops, for set-up and
    checks; the rendering path uses the fused chain kernels)."""
    return base + torch.einsum("mcd,d->mc", basis, p)


def render_views(p, poses, model, radii, light, albedo, scenes):
    """Radiance of every view: [V, P, 3].

    model: dict with v0, A_v, n0, A_n, c0, A_c (tensors on the device);
    poses: [V, 6] (axis-angle, translation); scenes: one Scene per view."""
    out = []
    for i, sc in enumerate(scenes):
        q = poses[i]
        pv = deform_pose(model["v0"], model["A_v"], p, q)
        pn = deform_pose(model["n0"], model["A_n"], p, q, direction=True)
        pc = deform_pose(model["c0"], model["A_c"], p, q)
        out.append(shade(pv, pn, albedo, pc, radii, light, sc))
    return torch.stack(out)


def make_view_scenes(n_views, centers, radii, light, config):
    """One resident Scene per view (each view's sphere centres differ)."""
    return [Scene(centers.detach(), radii.detach(), light.detach(), config) for _ in range(n_views)]


class DeformPoseViews(torch.autograd.Function):
    """x[v] = R(w_v) (base + basis p) + t_v for every view v in one launch
    (the deformation computed once per row); adjoint to p and all poses."""

    @staticmethod
    def forward(ctx, base, basis, p, poses, direction):
        lib = _lib.load()
        base, basis, p, poses = (_dev(t.detach(), n) for t, n in
                                 ((base, "base"), (basis, "basis"), (p, "p"), (poses, "poses")))
        M, D, V = int(base.shape[0]), int(p.shape[0]), int(poses.shape[0])
        if tuple(basis.shape) != (M, 3, D) or tuple(poses.shape) != (V, 6):
            raise ValueError(f"basis {tuple(basis.shape)} / poses {tuple(poses.shape)} do not match M={M}, D={D}")
        x = torch.empty((V, M, 3), dtype=torch.float32, device=base.device)
        check(lib.shs_chain_forward_views(ptr(base), ptr(basis), M, D, ptr(p), ptr(poses), V, int(direction), None,
                                          ptr(x), _stream()), "shs_chain_forward_views")
        ctx.save_for_backward(base, basis, p, poses)
        ctx.direction = int(direction)
        return x

    @staticmethod
    def backward(ctx, dx):
        lib = _lib.load()
        base, basis, p, poses = ctx.saved_tensors
        M, D, V = int(base.shape[0]), int(p.shape[0]), int(poses.shape[0])
        dx = _dev(dx, "dx")
        d_p = torch.empty((D,), dtype=torch.float32, device=base.device)
        d_poses = torch.empty((V, 6), dtype=torch.float32, device=base.device)
        nbytes = int(lib.shs_chain_views_workspace_bytes(M, D, V))
        ws = torch.empty((max(nbytes, 16) + 3) // 4, dtype=torch.float32, device=base.device)
        check(lib.shs_chain_backward_views(ptr(base), ptr(basis), M, D, ptr(p), ptr(poses), V, ctx.direction,
                                           ptr(dx), ptr(d_p), ptr(d_poses), ptr(ws), ws.numel() * 4, _stream()),
              "shs_chain_backward_views")
        return None, None, d_p, d_poses, None


def deform_pose_views(base, basis, p, poses, direction=False):
    """[V, M, 3]: every view's pose applied to base + basis p."""
    return DeformPoseViews.apply(base, basis, p, poses, bool(direction))


class ViewBatch:
    """Resident state for shading V views of one model together: one Scene per
    view (the views' sphere centres differ), the saved per-point state of each
    view, and a batch context.  One shs_shade_batch call shades every view,
    one more runs every view's adjoint."""

    def __init__(self, n_views, n_points, centers, radii, light, config):
        from .shade import Scene
        self.lib = _lib.load()
        self.V, self.P = int(n_views), int(n_points)
        self.scenes = [Scene(centers.detach(), radii.detach(), light.detach(), config) for _ in range(self.V)]
        dev = centers.device
        self.saved = [sc.new_saved(self.P, dev) for sc in self.scenes]
        h = ctypes.c_void_p()
        check(self.lib.shs_batch_create(ctypes.byref(h)), "shs_batch_create")
        self.batch = h
        self.K = self.scenes[0].K
        self.N = self.scenes[0].n_spheres

    def close(self):
        for sc in self.scenes:
            sc.close()
        self.scenes = []
        if getattr(self, "batch", None):
            check(self.lib.shs_batch_destroy(self.batch), "shs_batch_destroy")
            self.batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, reqs):
        arr = (_lib.ShsRequest * len(reqs))(*reqs)
        check(self.lib.shs_shade_batch(self.batch, arr, len(reqs), _stream()), "shs_shade_batch")


class ShadeViews(torch.autograd.Function):
    """Radiance [V, P, 3] of V views that share albedo, radii and lighting
    (points, normals and sphere centres per view), forward in one batched
    launch, adjoint in another (Eq. 8 and its adjoint per view)."""

    @staticmethod
    def forward(ctx, points, normals, albedo, centers, radii, light, views):
        V, P = views.V, views.P
        pts, nrm = _dev(points.detach(), "points"), _dev(normals.detach(), "normals")
        alb, ctr = _dev(albedo.detach(), "albedo"), _dev(centers.detach(), "centers")
        rad_, lgt = _dev(radii.detach(), "radii"), _dev(light.detach(), "light")
        for v, sc in enumerate(views.scenes):
            sc.update(centers=ctr[v], radii=rad_, light=lgt)
        out = torch.empty((V, P, 3), dtype=torch.float32, device=pts.device)
        reqs = []
        for v, sc in enumerate(views.scenes):
            r = _lib.ShsRequest()
            r.scene, r.n_points = sc.handle.value, P
            r.points, r.normals, r.albedo = pts[v].data_ptr(), nrm[v].data_ptr(), alb.data_ptr()
            r.radiance, r.saved = out[v].data_ptr(), views.saved[v].data_ptr()
            reqs.append(r)
        views.run(reqs)
        ctx.save_for_backward(pts, nrm, alb)
        ctx.views = views
        return out

    @staticmethod
    def backward(ctx, dB):
        pts, nrm, alb = ctx.saved_tensors
        views = ctx.views
        V, P, N, K = views.V, views.P, views.N, views.K
        dev = pts.device
        dB = _dev(dB, "d_radiance")
        z = lambda *s: torch.empty(s, dtype=torch.float32, device=dev)
        g = dict(d_points=z(V, P, 3), d_normals=z(V, P, 3), d_albedo=z(V, P, 3), d_centers=z(V, max(N, 1), 3),
                 d_radii=z(V, max(N, 1)), d_light=z(V, 3, K))
        reqs = []
        for v, sc in enumerate(views.scenes):
            r = _lib.ShsRequest()
            r.scene, r.n_points = sc.handle.value, P
            r.points, r.normals, r.albedo = pts[v].data_ptr(), nrm[v].data_ptr(), alb.data_ptr()
            r.saved, r.d_radiance = views.saved[v].data_ptr(), dB[v].data_ptr()
            r.d_light, r.d_albedo = g["d_light"][v].data_ptr(), g["d_albedo"][v].data_ptr()
            r.d_points, r.d_normals = g["d_points"][v].data_ptr(), g["d_normals"][v].data_ptr()
            if N:
                r.d_centers, r.d_radii = g["d_centers"][v].data_ptr(), g["d_radii"][v].data_ptr()
            reqs.append(r)
        views.run(reqs)
        d_centers = g["d_centers"][:, :N] if N else None
        d_radii = g["d_radii"][:, :N].sum(0) if N else None
        return (g["d_points"], g["d_normals"], g["d_albedo"].sum(0), d_centers, d_radii, g["d_light"].sum(0), None)


def render_views_batched(p, poses, model, radii, light, albedo, views):
    """Radiance of every view, [V, P, 3], with one chain launch per array
    (all views) and one shading launch for all views, forward and adjoint."""
    pv = deform_pose_views(model["v0"], model["A_v"], p, poses)
    pn = deform_pose_views(model["n0"], model["A_n"], p, poses, direction=True)
    pc = deform_pose_views(model["c0"], model["A_c"], p, poses)
    return ShadeViews.apply(pv, pn, albedo, pc, radii, light, views)
