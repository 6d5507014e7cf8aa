"""The projected-exponential variant of the SH exponential (exp_mode = 1):
V = e0 P_n[exp(f^)] by the 2n x 4n quadrature, forward and adjoint, against the
FP64 oracle computing the same definition."""

import numpy as np
import pytest

from oracle import shs_oracle as O
from paper_2104_00359_gb300 import synthetic as S

from gpu_helpers import FIELDS, gpu_run, grad_err, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8])
def test_projected_exp_forward(n):
    sc = S.random_scene(600 + n, 421, 13, n, inside_fraction=0.1)
    cfg = O.Config(n_bands=n, exp_mode=1)
    B, k, f, _, status = gpu_run(sc, cfg)
    assert status == 0
    assert np.all(k == 0)
    ref = O.shade_forward(cfg, *[sc[x] for x in FIELDS])
    np.testing.assert_allclose(f, ref["f"], rtol=0, atol=2e-5 * max(1.0, np.abs(ref["f"]).max()))
    err = rel_err(B, ref["radiance"])
    assert err.max() <= TOL, f"radiance max err {err.max():.3e}"
    # a different method: the answers differ at the level of the two approximations
    B0, *_ = gpu_run(sc, O.Config(n_bands=n))
    if n > 1:
        assert rel_err(B0, ref["radiance"]).max() > 10 * TOL


@pytest.mark.parametrize("n,n_spheres", [(2, 9), (4, 40), (5, 9), (6, 12), (8, 10)])
def test_projected_exp_backward(n, n_spheres):
    sc = S.random_scene(700 + n, 300, n_spheres, n, inside_fraction=0.1)
    cfg = O.Config(n_bands=n, exp_mode=1)
    dB = np.random.default_rng(8).normal(size=sc["points"].shape).astype(np.float32)
    B, k, f, g, status = gpu_run(sc, cfg, dB=dB)
    assert status == 0
    ref = O.shade_backward(cfg, *[sc[x] for x in FIELDS], dB)
    for name in ("d_light", "d_albedo", "d_centers", "d_radii", "d_points", "d_normals"):
        err = grad_err(name, g[name], ref)
        assert err.max() <= TOL, f"{name}: max err {err.max():.3e}"


def test_projected_exp_rejected_with_fp16_operands():
    """exp(f^) spans more than the half-precision range: FP16 operands are
    refused for the projected exponential (BF16 and TF32 run it)."""
    import torch
    from paper_2104_00359_gb300 import Config, Scene, _lib
    dev = torch.device("cuda:0")
    light = torch.zeros((3, 64), device=dev)
    with pytest.raises(_lib.ShsError) as e:
        Scene(None, None, light, Config(n_bands=8, precision=_lib.SHS_FP16, exp_mode=1))
    assert e.value.status == 2
    for prec in (_lib.SHS_BF16, _lib.SHS_TF32):
        Scene(None, None, light, Config(n_bands=8, precision=prec, exp_mode=1)).close()


def test_projected_exp_with_horizon_cull_backward():
    """Both options together (the fused backward is compiled per combination)."""
    sc = S.random_scene(720, 300, 33, 4, inside_fraction=0.05)
    nh = sc["normals"].astype(np.float64)
    nh /= np.linalg.norm(nh, axis=1, keepdims=True)
    d = sc["centers"].astype(np.float64)[None] - sc["points"].astype(np.float64)[:, None]
    margin = np.einsum("pjc,pc->pj", d, nh) + sc["radii"].astype(np.float64)[None]
    keep = np.all(np.abs(margin) > 1e-4 * (1.0 + np.abs(d).sum(-1)), axis=1)
    for k in ("points", "normals", "albedo"):
        sc[k] = np.ascontiguousarray(sc[k][keep])
    cfg = O.Config(n_bands=4, exp_mode=1, horizon_cull=True)
    dB = np.random.default_rng(9).normal(size=sc["points"].shape).astype(np.float32)
    B, k, f, g, status = gpu_run(sc, cfg, dB=dB)
    assert status == 0
    ref = O.shade_backward(cfg, *[sc[x] for x in FIELDS], dB)
    assert rel_err(B, ref["forward"]["radiance"]).max() <= TOL
    for name in ("d_light", "d_albedo", "d_centers", "d_radii", "d_points", "d_normals"):
        err = grad_err(name, g[name], ref)
        assert err.max() <= TOL, f"{name}: max err {err.max():.3e}"
