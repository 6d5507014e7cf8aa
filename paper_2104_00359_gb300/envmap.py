"""SH lighting from an equirectangular HDR environment map (Eq. 9), computed
by the library's projection kernel (``shs_project_envmap``)."""

from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import check, ptr


def project_envmap(env, n_bands, out=None, workspace=None):
    """[3, n_bands^2] SH coefficients of a [H, W, 3] float32 CUDA radiance map
    (row r: polar angles [r, r+1] pi / H from +z; column c: azimuths
    [c, c+1] 2 pi / W).  Runs on torch's current stream."""
    if not (env.is_cuda and env.dtype == torch.float32 and env.dim() == 3 and env.shape[2] == 3):
        raise TypeError("env must be a [H, W, 3] float32 CUDA tensor")
    lib = _lib.load()
    env = env.contiguous()
    H, W = int(env.shape[0]), int(env.shape[1])
    K = int(n_bands) ** 2
    light = out if out is not None else torch.empty((3, K), dtype=torch.float32, device=env.device)
    need = int(lib.shs_envmap_workspace_bytes(H, W, int(n_bands)))
    if workspace is None or workspace.numel() * workspace.element_size() < need:
        workspace = torch.empty(max(need, 4) // 4, dtype=torch.float32, device=env.device)
    stream = ctypes.c_void_p(torch.cuda.current_stream(env.device).cuda_stream)
    check(lib.shs_project_envmap(ptr(env), H, W, int(n_bands), ptr(light), ptr(workspace),
                                 workspace.numel() * workspace.element_size(), stream), "shs_project_envmap")
    return light
