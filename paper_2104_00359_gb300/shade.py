"""PyTorch-facing wrapper of the shading library.

``Scene`` owns a resident scene (spheres + SH lighting) on the current CUDA
device; ``Scene.shade`` / ``Scene.backward`` call the C ABI on torch's current
stream; ``shade`` is a ``torch.autograd.Function`` whose backward is the
library's hand-written adjoint kernel.  PyTorch supplies device memory and
streams only.
"""

from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import ShsConfig, check, ptr


@dataclass
class Config:
    """Method constants, mirrored into ``shs_config``.  ``epsilon`` = 3 is the
    paper's softened-blocker exponent (Sec. 3.3.2, Eq. 13)."""
    n_bands: int = 4
    epsilon: float = 3.0
    exp_tau: float = 1.0
    exp_kmax: int = 16
    fixed_k: int = -1
    precision: int = _lib.SHS_FP32
    deterministic: bool = True
    horizon_cull: bool = False
    exp_mode: int = 0          # 0: scaling + squarings (Sec. 3.3.2); 1: projected exponential;
                               # 2: as 0 with a fitted optimal linear table (Scene.set_ol_table)
    ol_table: tuple | None = None  # exp_mode 2: (a, b, s_max), set on every Scene made with this config

    def to_c(self):
        return ShsConfig(int(self.n_bands), float(self.epsilon), float(self.exp_tau), int(self.exp_kmax),
                         int(self.fixed_k), int(self.precision), int(bool(self.deterministic)),
                         int(bool(self.horizon_cull)), int(self.exp_mode))


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev_f32(t, shape, name):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float32):
        raise TypeError(f"{name} must be a float32 CUDA tensor")
    t = t.contiguous()
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


class Scene:
    """A resident sphere set and SH lighting (Sec. 3.3.1-3.3.2)."""

    def __init__(self, centers, radii, light, config: Config | None = None):
        self.lib = _lib.load()
        self.config = config or Config()
        self.K = self.config.n_bands ** 2
        self.n_spheres = int(centers.shape[0]) if centers is not None else 0
        c = _dev_f32(centers, (self.n_spheres, 3), "centers") if self.n_spheres else None
        r = _dev_f32(radii, (self.n_spheres,), "radii") if self.n_spheres else None
        L = _dev_f32(light, (3, self.K), "light")
        h = ctypes.c_void_p()
        cfg = self.config.to_c()
        check(self.lib.shs_scene_create(ctypes.byref(cfg), self.n_spheres, ptr(c), ptr(r), ptr(L), _stream(),
                                        ctypes.byref(h)), "shs_scene_create")
        self.handle = h
        if self.config.exp_mode == 2 and self.config.ol_table is not None:
            self.set_ol_table(*self.config.ol_table)

    def update(self, centers=None, radii=None, light=None):
        c = _dev_f32(centers, (self.n_spheres, 3), "centers") if centers is not None and self.n_spheres else None
        r = _dev_f32(radii, (self.n_spheres,), "radii") if radii is not None and self.n_spheres else None
        L = _dev_f32(light, (3, self.K), "light") if light is not None else None
        check(self.lib.shs_scene_update(self.handle, ptr(c), ptr(r), ptr(L), _stream()), "shs_scene_update")

    def set_ol_table(self, a, b, s_max):
        """Optimal linear coefficients a(s), b(s) at the nodes s_i = i s_max / (m-1)
        (exp_mode 2); host arrays, copied into the scene."""
        a = np.asarray(a, np.float64).ravel()
        b = np.asarray(b, np.float64).ravel()
        if a.shape != b.shape:
            raise ValueError("a and b must have the same length")
        tab = np.ascontiguousarray(np.concatenate([a, b]), np.float32)
        check(self.lib.shs_scene_set_ol_table(self.handle, tab.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                              int(a.shape[0]), float(s_max)), "shs_scene_set_ol_table")

    def close(self):
        if getattr(self, "handle", None):
            check(self.lib.shs_scene_destroy(self.handle), "shs_scene_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def saved_bytes(self, n_points):
        return int(self.lib.shs_saved_bytes(self.handle, int(n_points)))

    def saved_views(self, saved, n_points):
        """(f [P, K] float32 view, k [P] int32 view) of a saved buffer, with the
        layout shs_shade writes: f as [K][P], then k 16-byte aligned."""
        P = int(n_points)
        off = (self.K * P * 4 + 15) // 16 * 16 // 4
        f = saved[: self.K * P].view(self.K, P).t()
        k = saved[off: off + P].view(torch.int32)
        return f, k

    def new_saved(self, n_points, device=None):
        nbytes = self.saved_bytes(n_points)
        return torch.empty(max(nbytes, 16) // 4, dtype=torch.float32, device=device or "cuda")

    def shade(self, points, normals, albedo, saved=None, out=None):
        P = int(points.shape[0])
        pts = _dev_f32(points, (P, 3), "points")
        nrm = _dev_f32(normals, (P, 3), "normals")
        alb = _dev_f32(albedo, (P, 3), "albedo")
        rad = out if out is not None else torch.empty((P, 3), dtype=torch.float32, device=pts.device)
        check(self.lib.shs_shade(self.handle, P, ptr(pts), ptr(nrm), ptr(alb), ptr(rad), ptr(saved), _stream()),
              "shs_shade")
        return rad

    def shade_tail(self, normals, albedo, saved, out=None):
        """Radiance from the log-visibility a shade() call saved for the same
        points and spheres: only the exponential and the shading run (the
        lighting or the albedo changed since, the geometry did not)."""
        P = int(normals.shape[0])
        nrm = _dev_f32(normals, (P, 3), "normals")
        alb = _dev_f32(albedo, (P, 3), "albedo")
        rad = out if out is not None else torch.empty((P, 3), dtype=torch.float32, device=nrm.device)
        check(self.lib.shs_shade_tail(self.handle, P, ptr(nrm), ptr(alb), ptr(saved), ptr(rad), _stream()),
              "shs_shade_tail")
        return rad

    def _grad_buffers(self, P, device, want):
        z = lambda *s: torch.empty(s, dtype=torch.float32, device=device)
        N = self.n_spheres
        return dict(
            d_light=z(3, self.K) if "light" in want else None,
            d_albedo=z(P, 3) if "albedo" in want else None,
            d_centers=z(N, 3) if "centers" in want else None,
            d_radii=z(N) if "radii" in want else None,
            d_points=z(P, 3) if "points" in want else None,
            d_normals=z(P, 3) if "normals" in want else None,
        )

    ALL = ("light", "albedo", "centers", "radii", "points", "normals")

    def backward(self, points, normals, albedo, d_radiance, saved=None, want=ALL):
        P = int(points.shape[0])
        pts = _dev_f32(points, (P, 3), "points")
        nrm = _dev_f32(normals, (P, 3), "normals")
        alb = _dev_f32(albedo, (P, 3), "albedo")
        dB = _dev_f32(d_radiance, (P, 3), "d_radiance")
        g = self._grad_buffers(P, pts.device, want)
        check(self.lib.shs_shade_backward(self.handle, P, ptr(pts), ptr(nrm), ptr(alb), ptr(saved), ptr(dB),
                                          ptr(g["d_light"]), ptr(g["d_albedo"]), ptr(g["d_centers"]),
                                          ptr(g["d_radii"]), ptr(g["d_points"]), ptr(g["d_normals"]),
                                          _stream()), "shs_shade_backward")
        return g

    def backward_l2(self, points, normals, albedo, radiance, target, saved=None, want=ALL):
        """Loss 1/2 |B - target|^2 and its gradients in one launch."""
        P = int(points.shape[0])
        pts = _dev_f32(points, (P, 3), "points")
        nrm = _dev_f32(normals, (P, 3), "normals")
        alb = _dev_f32(albedo, (P, 3), "albedo")
        rad = _dev_f32(radiance, (P, 3), "radiance")
        tgt = _dev_f32(target, (P, 3), "target")
        g = self._grad_buffers(P, pts.device, want)
        g["loss"] = torch.empty((), dtype=torch.float32, device=pts.device)
        check(self.lib.shs_shade_backward_l2(self.handle, P, ptr(pts), ptr(nrm), ptr(alb), ptr(saved), ptr(rad),
                                             ptr(tgt), ptr(g["loss"]), ptr(g["d_light"]), ptr(g["d_albedo"]),
                                             ptr(g["d_centers"]), ptr(g["d_radii"]), ptr(g["d_points"]),
                                             ptr(g["d_normals"]), _stream()), "shs_shade_backward_l2")
        return g

    def device_status(self):
        st = ctypes.c_int32(0)
        check(self.lib.shs_scene_device_status(self.handle, _stream(), ctypes.byref(st)), "shs_scene_device_status")
        return int(st.value)


class ShadeFunction(torch.autograd.Function):
    """B = shade(points, normals, albedo, centers, radii, light) on a Scene.

    Forward stores the per-point log-visibility (``saved`` state) so the
    adjoint kernel only recomputes the per-sphere terms."""

    @staticmethod
    def forward(ctx, points, normals, albedo, centers, radii, light, scene):
        scene.update(centers.detach(), radii.detach(), light.detach())
        saved = scene.new_saved(points.shape[0], points.device)
        B = scene.shade(points.detach(), normals.detach(), albedo.detach(), saved=saved)
        ctx.scene = scene
        ctx.save_for_backward(points, normals, albedo, saved)
        return B

    @staticmethod
    def backward(ctx, dB):
        points, normals, albedo, saved = ctx.saved_tensors
        names = ("points", "normals", "albedo", "centers", "radii", "light")
        want = tuple(n for n, need in zip(names, ctx.needs_input_grad[:6]) if need)
        g = ctx.scene.backward(points.detach(), normals.detach(), albedo.detach(), dB.contiguous(),
                               saved=saved, want=want)
        return (g["d_points"], g["d_normals"], g["d_albedo"], g["d_centers"], g["d_radii"], g["d_light"], None)


def shade(points, normals, albedo, centers, radii, light, scene: Scene):
    """Differentiable shaded radiance [P, 3] (Eq. 8) through the CUDA library."""
    return ShadeFunction.apply(points, normals, albedo, centers, radii, light, scene)
