"""Differentiable rasterisation of shaded vertices, I_R = R(B, P), through the
library's kernels (``shs_rasterize`` / ``shs_rasterize_backward``).

``rasterize`` is a ``torch.autograd.Function``: gradients flow to the vertex
radiance (exactly) and to the vertex positions (through the perspective-
correct barycentrics, each pixel's triangle held fixed), so an image-space L2
loss reaches the shading path and the geometry.
"""

from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import check, ptr


def _proj_host(proj):
    P = np.ascontiguousarray(np.asarray(proj.detach().cpu() if torch.is_tensor(proj) else proj,
                                        dtype=np.float32).reshape(16))
    return P, P.ctypes.data_as(ctypes.c_void_p)


def _workspace(lib, V, H, W, device):
    need = int(lib.shs_raster_workspace_bytes(int(V), int(H), int(W)))
    return torch.empty(max(need, 256) // 4, dtype=torch.float32, device=device), need


class Rasterize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vertices, radiance, faces, proj, height, width):
        lib = _lib.load()
        v = vertices.detach().contiguous().float()
        b = radiance.detach().contiguous().float()
        f = faces.contiguous().to(torch.int32)
        H, W = int(height), int(width)
        P, Pp = _proj_host(proj)
        image = torch.empty((H, W, 3), dtype=torch.float32, device=v.device)
        face_index = torch.empty((H, W), dtype=torch.int32, device=v.device)
        ws, need = _workspace(lib, v.shape[0], H, W, v.device)
        stream = ctypes.c_void_p(torch.cuda.current_stream(v.device).cuda_stream)
        check(lib.shs_rasterize(ptr(v), v.shape[0], ptr(f), f.shape[0], Pp, ptr(b), H, W, ptr(image),
                                ptr(face_index), ptr(ws), need, stream), "shs_rasterize")
        ctx.save_for_backward(v, b, f, face_index)
        ctx.P = P
        ctx.size = (H, W)
        ctx.mark_non_differentiable(face_index)
        return image, face_index

    @staticmethod
    def backward(ctx, d_image, _d_face_index):
        lib = _lib.load()
        v, b, f, face_index = ctx.saved_tensors
        H, W = ctx.size
        want_v, want_b = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        dv = torch.empty_like(v) if want_v else None
        db = torch.empty_like(b) if want_b else None
        if not (want_v or want_b):
            return None, None, None, None, None, None
        ws, need = _workspace(lib, v.shape[0], H, W, v.device)
        stream = ctypes.c_void_p(torch.cuda.current_stream(v.device).cuda_stream)
        P = ctx.P
        check(lib.shs_rasterize_backward(ptr(v), v.shape[0], ptr(f), f.shape[0], P.ctypes.data_as(ctypes.c_void_p),
                                         ptr(b), H, W, ptr(face_index), ptr(d_image.contiguous().float()),
                                         ptr(db), ptr(dv), ptr(ws), need, stream), "shs_rasterize_backward")
        return dv, db, None, None, None, None


def rasterize(vertices, radiance, faces, proj, height, width):
    """(image [H, W, 3], face_index [H, W]) of a mesh with vertex radiance
    seen through the 4 x 4 projection ``proj`` (row-major, host or device)."""
    return Rasterize.apply(vertices, radiance, faces, proj, height, width)
