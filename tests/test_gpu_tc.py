"""Tensor-core (tcgen05) paths.

1. Operand layouts and descriptors: a one-CTA D = A B^T through
   shs_tc_gemm_selftest against float64 numpy for every operand type the
   tails use (plain BF16: one rounding per operand; BF16 split in two parts;
   BF16 in three parts, TF32 and FP16 in two parts, the tails' types).
2. The 8-band reduced-precision tails (squarings, Eq. 7, and shading, Eq. 8,
   forward and adjoint) against the FP64 oracle, per output: radiance and
   every gradient within 2e-3 (the stated reduced-precision tolerance) for
   BF16, TF32 and FP16, with the per-point squaring counts k from the GPU.
   The float32 pair terms f and k must equal the FP32 path's bitwise.
3. The projected exponential (exp_mode 1, V = e0 P[exp(f^)] by the 2n x 4n
   rule) on the tensor cores, BF16 and TF32, forward and adjoint, against the
   oracle's projected exponential, every output within 2e-3."""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
TOL_TC = 2e-3
GRADS = ("d_light", "d_albedo", "d_centers", "d_radii", "d_points", "d_normals")


@pytest.mark.parametrize("n,k", [(64, 64), (256, 64), (192, 64), (16, 16), (48, 32)])
def test_tc_gemm_matches_numpy(n, k):
    import torch
    from paper_2104_00359_gb300 import _lib
    lib = _lib.load()
    rng = np.random.default_rng(n * 1000 + k)
    A = rng.normal(size=(128, k)).astype(np.float32)
    B = rng.normal(size=(n, k)).astype(np.float32)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    dev = torch.device("cuda:0")
    tA, tB = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    # mode: 0 BF16, 1 BF16 x2, 2 BF16 x3, 3 TF32 x2, 4 FP16 x2; 5-7 as 2-4 with A in tensor memory
    for mode, tol in ((0, 2e-2), (1, 1e-4), (2, 2e-6), (3, 2e-6), (4, 2e-6), (5, 2e-6), (6, 2e-6), (7, 2e-6)):
        D = torch.full((128, n), np.nan, device=dev)
        _lib.check(lib.shs_tc_gemm_selftest(_lib.ptr(tA), _lib.ptr(tB), n, k, mode, _lib.ptr(D), _lib.ptr(st),
                                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)),
                   "shs_tc_gemm_selftest")
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        got = D.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got)), mode
        err = np.abs(got - ref) / scale
        assert err.max() <= tol, (mode, err.max())


def _run(sc, prec, dB, saved=True, deterministic=True, target=None, exp_mode=0):
    import torch
    from paper_2104_00359_gb300 import Config, Scene
    from gpu_helpers import FIELDS
    dev = torch.device("cuda:0")
    T = {k: torch.from_numpy(np.ascontiguousarray(sc[k])).to(dev) for k in FIELDS}
    P = sc["points"].shape[0]
    scene = Scene(T["centers"], T["radii"], T["light"], Config(n_bands=8, precision=prec,
                                                               deterministic=deterministic, exp_mode=exp_mode))
    sv = scene.new_saved(P, dev)
    B = scene.shade(T["points"], T["normals"], T["albedo"], saved=sv)
    if target is not None:
        tg = torch.from_numpy(np.ascontiguousarray(target, np.float32)).to(dev)
        g = scene.backward_l2(T["points"], T["normals"], T["albedo"], B, tg, saved=sv if saved else None)
    else:
        g = scene.backward(T["points"], T["normals"], T["albedo"],
                           torch.from_numpy(np.ascontiguousarray(dB, np.float32)).to(dev),
                           saved=sv if saved else None)
    torch.cuda.synchronize()
    assert scene.device_status() == 0
    f, k = scene.saved_views(sv, P)
    out = dict(radiance=B.cpu().numpy(), f=f.cpu().numpy(), k=k.cpu().numpy().astype(np.int64))
    out.update({name: (v.cpu().numpy() if v is not None else None) for name, v in g.items()})
    scene.close()
    return out


def _errors(sc, got, dB, k, exp_mode=0):
    from oracle import shs_oracle as O
    from gpu_helpers import FIELDS, grad_err, rel_err
    args = [sc[x] for x in FIELDS]
    cfg = O.Config(n_bands=8, exp_mode=exp_mode)
    ref = O.shade_backward(cfg, *args, dB, k=k)
    errs = {"radiance": float(rel_err(got["radiance"], ref["forward"]["radiance"]).max())}
    for name in GRADS:
        errs[name] = float(grad_err(name, got[name], ref).max())
    return errs


def _sample_scene(which):
    from paper_2104_00359_gb300 import synthetic as S
    if which == "random":
        return S.random_scene(77, 700, 40, 8, inside_fraction=0.05)
    hf = S.height_field_scene(res=128)
    sel = np.sort(np.random.default_rng(1).choice(hf["points"].shape[0], 600, replace=False))
    out = dict(hf)
    for key in ("points", "normals", "albedo"):
        out[key] = np.ascontiguousarray(hf[key][sel])
    return out


@pytest.mark.parametrize("scene_kind", ["random", "heightfield"])
@pytest.mark.parametrize("prec_name", ["bf16", "tf32", "fp16"])
def test_tensor_core_tails_n8_against_oracle(prec_name, scene_kind):
    """Forward and adjoint tails on the tensor cores, every output vs FP64."""
    from paper_2104_00359_gb300._lib import SHS_BF16, SHS_FP16, SHS_FP32, SHS_TF32
    prec = dict(bf16=SHS_BF16, tf32=SHS_TF32, fp16=SHS_FP16)[prec_name]
    sc = _sample_scene(scene_kind)
    P = sc["points"].shape[0]
    dB = np.random.default_rng(5).normal(size=(P, 3))
    g32 = _run(sc, SHS_FP32, dB)
    gtc = _run(sc, prec, dB)
    np.testing.assert_array_equal(gtc["f"], g32["f"])
    np.testing.assert_array_equal(gtc["k"], g32["k"])
    e32 = _errors(sc, g32, dB, g32["k"])
    etc = _errors(sc, gtc, dB, g32["k"])
    print(f"{prec_name} {scene_kind}: " + ", ".join(f"{k} {v:.2e}" for k, v in etc.items()))
    print(f"fp32 {scene_kind}: " + ", ".join(f"{k} {v:.2e}" for k, v in e32.items()))
    assert e32["radiance"] <= 1e-4
    for name, v in etc.items():
        assert v <= TOL_TC, f"{prec_name} {scene_kind}: {name} max normalised error {v:.3e}"


def test_tensor_core_adjoint_modes():
    """BF16: recompute (no saved state) equals saved; the unordered (atomic)
    reduction agrees with the fixed-order one; the fused L2 adjoint."""
    from oracle import shs_oracle as O
    from paper_2104_00359_gb300._lib import SHS_BF16
    from gpu_helpers import FIELDS, grad_err
    from paper_2104_00359_gb300 import synthetic as S
    sc = S.random_scene(78, 333, 23, 8, inside_fraction=0.05)
    P = sc["points"].shape[0]
    dB = np.random.default_rng(6).normal(size=(P, 3))
    a = _run(sc, SHS_BF16, dB)
    b = _run(sc, SHS_BF16, dB, saved=False)
    c = _run(sc, SHS_BF16, dB, deterministic=False)
    for name in GRADS:
        np.testing.assert_allclose(b[name], a[name], rtol=0, atol=1e-6 * np.abs(a[name]).max())
    ref = O.shade_backward(O.Config(n_bands=8), *[sc[x] for x in FIELDS], dB, k=a["k"])
    for name in ("d_light", "d_centers", "d_radii"):
        assert grad_err(name, c[name], ref).max() <= TOL_TC, name
    tgt = S.perturb_scene(sc, 3)
    target = O.shade_forward(O.Config(n_bands=8), *[tgt[x] for x in FIELDS])["radiance"]
    d = _run(sc, SHS_BF16, None, target=target)
    dBl = d["radiance"].astype(np.float64) - target.astype(np.float32)
    ref = O.shade_backward(O.Config(n_bands=8), *[sc[x] for x in FIELDS], dBl, k=d["k"])
    assert abs(float(d["loss"]) - 0.5 * np.sum(dBl ** 2)) <= 1e-5 * np.sum(dBl ** 2)
    for name in GRADS:
        assert grad_err(name, d[name], ref).max() <= TOL_TC, name


@pytest.mark.parametrize("scene_kind", ["random", "heightfield"])
@pytest.mark.parametrize("prec_name", ["bf16", "tf32"])
def test_tensor_core_projected_exp_n8_against_oracle(prec_name, scene_kind):
    """exp_mode 1 on the tensor cores: the exp pass, shading and adjoint
    through the 16 x 32 rule, every output vs the oracle's projected
    exponential; the float32 CUDA-core variant is checked beside it."""
    from paper_2104_00359_gb300._lib import SHS_BF16, SHS_FP32, SHS_TF32
    prec = dict(bf16=SHS_BF16, tf32=SHS_TF32)[prec_name]
    sc = _sample_scene(scene_kind)
    P = sc["points"].shape[0]
    dB = np.random.default_rng(15).normal(size=(P, 3))
    g32 = _run(sc, SHS_FP32, dB, exp_mode=1)
    gtc = _run(sc, prec, dB, exp_mode=1)
    np.testing.assert_array_equal(gtc["f"], g32["f"])
    assert np.all(gtc["k"] == 0) and np.all(g32["k"] == 0)
    e32 = _errors(sc, g32, dB, None, exp_mode=1)
    etc = _errors(sc, gtc, dB, None, exp_mode=1)
    print(f"{prec_name} projexp {scene_kind}: " + ", ".join(f"{k} {v:.2e}" for k, v in etc.items()))
    print(f"fp32 projexp {scene_kind}: " + ", ".join(f"{k} {v:.2e}" for k, v in e32.items()))
    assert e32["radiance"] <= 1e-4
    for name, v in etc.items():
        assert v <= TOL_TC, f"{prec_name} projexp {scene_kind}: {name} max normalised error {v:.3e}"


def test_tensor_core_projected_exp_modes():
    """BF16 projected exponential: recompute (no saved state) equals saved,
    the fused L2 adjoint against the oracle, and the re-shading tail."""
    import torch
    from oracle import shs_oracle as O
    from paper_2104_00359_gb300 import Config, Scene, synthetic as S
    from paper_2104_00359_gb300._lib import SHS_BF16
    from gpu_helpers import FIELDS, grad_err, rel_err
    sc = S.random_scene(79, 301, 17, 8, inside_fraction=0.05)
    P = sc["points"].shape[0]
    dB = np.random.default_rng(16).normal(size=(P, 3))
    a = _run(sc, SHS_BF16, dB, exp_mode=1)
    b = _run(sc, SHS_BF16, dB, saved=False, exp_mode=1)
    for name in GRADS:
        np.testing.assert_allclose(b[name], a[name], rtol=0, atol=1e-6 * np.abs(a[name]).max())
    cfg = O.Config(n_bands=8, exp_mode=1)
    tgt = S.perturb_scene(sc, 4)
    target = O.shade_forward(cfg, *[tgt[x] for x in FIELDS])["radiance"]
    d = _run(sc, SHS_BF16, None, target=target, exp_mode=1)
    dBl = d["radiance"].astype(np.float64) - target.astype(np.float32)
    ref = O.shade_backward(cfg, *[sc[x] for x in FIELDS], dBl)
    assert abs(float(d["loss"]) - 0.5 * np.sum(dBl ** 2)) <= 1e-5 * np.sum(dBl ** 2)
    for name in GRADS:
        assert grad_err(name, d[name], ref).max() <= TOL_TC, name
    # shs_shade_tail from the saved pair terms under new lighting
    dev = torch.device("cuda:0")
    T = {k: torch.from_numpy(np.ascontiguousarray(sc[k])).to(dev) for k in FIELDS}
    scene = Scene(T["centers"], T["radii"], T["light"], Config(n_bands=8, precision=SHS_BF16, exp_mode=1))
    sv = scene.new_saved(P, dev)
    scene.shade(T["points"], T["normals"], T["albedo"], saved=sv)
    light2 = np.random.default_rng(17).normal(scale=0.3, size=sc["light"].shape).astype(np.float32)
    light2[:, 0] = 1.0
    scene.update(light=torch.from_numpy(light2).to(dev))
    B2 = scene.shade_tail(T["normals"], T["albedo"], sv).cpu().numpy()
    assert scene.device_status() == 0
    scene.close()
    args = [sc[x] for x in FIELDS]
    args[FIELDS.index("light")] = light2
    ref2 = O.shade_forward(cfg, *args)["radiance"]
    assert rel_err(B2, ref2).max() <= TOL_TC
