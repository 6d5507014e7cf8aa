"""shs_shade_backward_noalloc: the backward pass for callers that cannot
allocate device memory (their memory belongs to another allocator, or their
loop must not allocate after start-up).  It keeps its intermediates in a
static device array, so each case calls it twice in a row through the C ABI
and checks both results against the FP64 oracle (per-point k from the GPU's
forward pass) and against the scene-based shs_shade_backward, within the
tolerances the other parity tests use: 1e-4, and 3e-4 for 8-band gradients
(the adjoint runs back through k squarings, each doubling the relative
rounding of its operand).  From 6 bands this call takes the fused backward
kernel, which the scene path does not use there, and with saved = NULL it
recomputes the log-visibility.  This file is collected last."""

import ctypes

import numpy as np
import pytest

from oracle import shs_oracle as O
from paper_2104_00359_gb300 import synthetic as S

from gpu_helpers import FIELDS, grad_err

pytestmark = pytest.mark.gpu
NAMES = ("d_light", "d_albedo", "d_centers", "d_radii", "d_points", "d_normals")


def _noalloc(lib, cfg_c, T, P, N, K, saved, dB, stream):
    import torch
    from paper_2104_00359_gb300._lib import check, ptr
    dev = T["points"].device
    out = dict(d_light=torch.full((3, K), np.nan, device=dev), d_albedo=torch.full((P, 3), np.nan, device=dev),
               d_centers=torch.full((N, 3), np.nan, device=dev), d_radii=torch.full((N,), np.nan, device=dev),
               d_points=torch.full((P, 3), np.nan, device=dev), d_normals=torch.full((P, 3), np.nan, device=dev))
    check(lib.shs_shade_backward_noalloc(ctypes.byref(cfg_c), N, ptr(T["centers"]), ptr(T["radii"]),
                                         ptr(T["light"]), P, ptr(T["points"]), ptr(T["normals"]),
                                         ptr(T["albedo"]), ptr(saved), ptr(dB), ptr(out["d_light"]),
                                         ptr(out["d_albedo"]), ptr(out["d_centers"]), ptr(out["d_radii"]),
                                         ptr(out["d_points"]), ptr(out["d_normals"]), stream),
          "shs_shade_backward_noalloc")
    st = ctypes.c_int32(-1)
    check(lib.shs_noalloc_device_status(stream, ctypes.byref(st)), "shs_noalloc_device_status")
    assert st.value == 0
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("n,n_spheres,use_saved", [(4, 37, True), (4, 7, True), (4, 37, False),
                                                     (6, 23, True), (8, 19, True), (8, 19, False)])
def test_noalloc_backward_matches_oracle_and_scene_backward_twice(n, n_spheres, use_saved):
    import torch
    from paper_2104_00359_gb300 import Config, Scene, _lib
    lib = _lib.load()
    K = n * n
    tol = 3e-4 if n >= 7 else 1e-4
    P0 = 700 if n <= 6 else 300
    sc = S.random_scene(300 + 10 * n + n_spheres, P0, n_spheres, n, inside_fraction=0.1)
    P, N = sc["points"].shape[0], n_spheres
    dev = torch.device("cuda:0")
    T = {k: torch.from_numpy(sc[k]).to(dev) for k in FIELDS}
    cfg = Config(n_bands=n, deterministic=False)
    scene = Scene(T["centers"], T["radii"], T["light"], cfg)
    saved = scene.new_saved(P, dev)
    scene.shade(T["points"], T["normals"], T["albedo"], saved=saved)
    dB = torch.from_numpy(np.random.default_rng(7).normal(size=(P, 3)).astype(np.float32)).to(dev)
    ref_t = scene.backward(T["points"], T["normals"], T["albedo"], dB, saved=saved)
    torch.cuda.synchronize()
    scene_ref = {k: v.cpu().numpy() for k, v in ref_t.items()}
    k_gpu = scene.saved_views(saved, P)[1].cpu().numpy().astype(np.int64)
    scene.close()
    oracle = O.shade_backward(O.Config(n_bands=n), *[sc[x] for x in FIELDS], dB.cpu().numpy(), k=k_gpu)
    # the oracle's sums of absolute per-point terms set the rounding scale of the scene-level sums
    for name in ("d_light", "d_centers", "d_radii"):
        scene_ref["abs_" + name] = oracle["abs_" + name]

    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cfg_c = cfg.to_c()
    for call in range(2):
        got = _noalloc(lib, cfg_c, T, P, N, K, saved if use_saved else None, dB, stream)
        for name in NAMES:
            assert np.all(np.isfinite(got[name])), (call, name)
            err = grad_err(name, got[name], oracle)
            assert err.max() <= tol, f"call {call}: {name} vs oracle, max err {err.max():.3e}"
            err = grad_err(name, got[name], scene_ref)
            assert err.max() <= tol, f"call {call}: {name} vs shs_shade_backward, max err {err.max():.3e}"


def test_noalloc_rejects_sizes_beyond_its_limits():
    from paper_2104_00359_gb300 import _lib
    from paper_2104_00359_gb300._lib import ShsConfig
    lib = _lib.load()
    cfg = ShsConfig()
    lib.shs_config_default(ctypes.byref(cfg))
    cfg.deterministic = 0
    one = ctypes.c_void_p(16)
    st = lib.shs_shade_backward_noalloc(ctypes.byref(cfg), 1025, one, one, one, 10, one, one, one, None, one,
                                        None, None, None, None, None, None, None)
    assert st == 1 and b"limit" in lib.shs_last_error()
    cfg.deterministic = 1       # fixed-order sums need per-block partials the fixed array cannot hold
    st = lib.shs_shade_backward_noalloc(ctypes.byref(cfg), 3, one, one, one, 10, one, one, one, None, one,
                                        None, None, None, None, None, None, None)
    assert st == 2 and b"deterministic" in lib.shs_last_error()
