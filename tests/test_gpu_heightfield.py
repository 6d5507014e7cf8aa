"""The 1024x1024 height field with 300 spheres at n = 8 (K = 64): forward and
backward at full size in one launch each, compared with the FP64 oracle on a
random sample of points (per-point outputs the oracle computes one by one)."""

import numpy as np
import pytest

from oracle import shs_oracle as O
from paper_2104_00359_gb300 import synthetic as S

from gpu_helpers import FIELDS, grad_err, oracle_k_consistent, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-4
# Gradients at 8 bands: the adjoint runs back through k ~ 4-5 squarings, each
# doubling the relative rounding error of its operand (as in the forward), so
# float32 per-point gradients carry ~2^k more rounding than the radiance.
TOL_GRAD_8 = 3e-4


def test_height_field_n8_full_size_sampled():
    import torch
    from paper_2104_00359_gb300 import Config, Scene
    sc = S.height_field_scene()
    dev = torch.device("cuda:0")
    T = {k: torch.from_numpy(sc[k]).to(dev) for k in FIELDS}
    scene = Scene(T["centers"], T["radii"], T["light"], Config(n_bands=8))
    P = sc["points"].shape[0]
    saved = scene.new_saved(P, dev)
    B = scene.shade(T["points"], T["normals"], T["albedo"], saved=saved)
    dB = torch.from_numpy(np.random.default_rng(9).normal(size=(P, 3)).astype(np.float32)).to(dev)
    g = scene.backward(T["points"], T["normals"], T["albedo"], dB, saved=saved,
                       want=("albedo", "points", "normals"))
    torch.cuda.synchronize()
    assert scene.device_status() == 0
    k = scene.saved_views(saved, P)[1].cpu().numpy().astype(np.int64)
    sel = np.sort(np.random.default_rng(1).choice(P, 256, replace=False))
    cfg = O.Config(n_bands=8)
    args = [sc[f][sel] if f in ("points", "normals", "albedo") else sc[f] for f in FIELDS]
    ref = O.shade_forward(cfg, *args)
    oracle_k_consistent(cfg, ref["f"], k[sel])
    ref = O.shade_forward(cfg, *args, k=k[sel])
    assert rel_err(B.cpu().numpy()[sel], ref["radiance"]).max() <= TOL
    gref = O.shade_backward(cfg, *args, dB.cpu().numpy()[sel], k=k[sel])
    for name in ("d_albedo", "d_points", "d_normals"):
        err = grad_err(name, g[name].cpu().numpy()[sel], gref)
        assert err.max() <= TOL_GRAD_8, f"{name}: {err.max():.3e}"
    scene.close()
