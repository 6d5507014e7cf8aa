"""shs_shade_backward_noalloc: the backward pass for callers that cannot
allocate device memory (their memory belongs to another allocator, or their
loop must not allocate after start-up).  It keeps its intermediates in a
static device array, so the test calls it twice in a row through the C ABI
and checks both results against the scene-based shs_shade_backward, within the
tolerance the other parity tests use.  This file is collected last."""

import ctypes

import numpy as np
import pytest

from oracle import shs_oracle as O
from paper_2104_00359_gb300 import synthetic as S

from gpu_helpers import FIELDS, grad_err

pytestmark = pytest.mark.gpu
TOL = 1e-4
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
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("n_spheres", [37, 7])
def test_noalloc_backward_matches_scene_backward_twice(n_spheres):
    import torch
    from paper_2104_00359_gb300 import Config, Scene, _lib
    lib = _lib.load()
    n = 4
    K = n * n
    sc = S.random_scene(300 + n_spheres, 700, n_spheres, n, inside_fraction=0.1)
    P, N = sc["points"].shape[0], n_spheres
    dev = torch.device("cuda:0")
    T = {k: torch.from_numpy(sc[k]).to(dev) for k in FIELDS}
    cfg = Config(n_bands=n)
    scene = Scene(T["centers"], T["radii"], T["light"], cfg)
    saved = scene.new_saved(P, dev)
    scene.shade(T["points"], T["normals"], T["albedo"], saved=saved)
    dB = torch.from_numpy(np.random.default_rng(7).normal(size=(P, 3)).astype(np.float32)).to(dev)
    ref_t = scene.backward(T["points"], T["normals"], T["albedo"], dB, saved=saved)
    torch.cuda.synchronize()
    ref = {k: v.cpu().numpy() for k, v in ref_t.items()}
    k_gpu = scene.saved_views(saved, P)[1].cpu().numpy().astype(np.int64)
    scene.close()
    # sums of absolute per-point terms set the rounding scale of the scene-level sums
    absref = O.shade_backward(O.Config(n_bands=n), *[sc[x] for x in FIELDS], dB.cpu().numpy(), k=k_gpu)
    for name in ("d_light", "d_centers", "d_radii"):
        ref["abs_" + name] = absref["abs_" + name]

    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cfg_c = cfg.to_c()
    for call in range(2):
        got = _noalloc(lib, cfg_c, T, P, N, K, saved, dB, stream)
        for name in NAMES:
            assert np.all(np.isfinite(got[name])), (call, name)
            err = grad_err(name, got[name], ref)
            assert err.max() <= TOL, f"call {call}: {name} max err {err.max():.3e}"


def test_noalloc_rejects_sizes_beyond_its_limits():
    from paper_2104_00359_gb300 import _lib
    from paper_2104_00359_gb300._lib import ShsConfig
    lib = _lib.load()
    cfg = ShsConfig()
    lib.shs_config_default(ctypes.byref(cfg))
    one = ctypes.c_void_p(16)
    st = lib.shs_shade_backward_noalloc(ctypes.byref(cfg), 1025, one, one, one, 10, one, one, one, None, one,
                                        None, None, None, None, None, None, None)
    assert st == 1 and b"limit" in lib.shs_last_error()
