"""Tensor-core (tcgen05) operand layouts and descriptors: a one-CTA
D = A B^T through shs_tc_gemm_selftest against float64 numpy, in plain BF16
(error of one BF16 rounding per operand) and in split precision (three MMAs,
about 16 significant bits per operand)."""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


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
    for split, tol in ((0, 2e-2), (1, 1e-4)):
        D = torch.full((128, n), np.nan, device=dev)
        _lib.check(lib.shs_tc_gemm_selftest(_lib.ptr(tA), _lib.ptr(tB), n, k, split, _lib.ptr(D), _lib.ptr(st),
                                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)),
                   "shs_tc_gemm_selftest")
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        got = D.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
        err = np.abs(got - ref) / scale
        assert err.max() <= tol, (split, err.max())


@pytest.mark.parametrize("prec,tol", [("fp16", 2e-3), ("bf16", 5e-3)])
def test_tensor_core_tail_n8_against_oracle(prec, tol):
    """8 bands, split 16-bit tensor-core squarings and shading contraction:
    radiance against the FP64 oracle (k from the GPU), and bitwise agreement
    of the float32 pair terms f with the FP32 path."""
    import torch
    from oracle import shs_oracle as O
    from paper_2104_00359_gb300 import Config, Scene, synthetic as S
    from paper_2104_00359_gb300._lib import SHS_BF16, SHS_FP16
    from gpu_helpers import FIELDS, rel_err
    sc = S.random_scene(77, 700, 40, 8, inside_fraction=0.05)
    dev = torch.device("cuda:0")
    T = {k: torch.from_numpy(sc[k]).to(dev) for k in FIELDS}
    P = sc["points"].shape[0]
    out = {}
    for name, p in (("fp32", 0), (prec, SHS_FP16 if prec == "fp16" else SHS_BF16)):
        scene = Scene(T["centers"], T["radii"], T["light"], Config(n_bands=8, precision=p))
        sv = scene.new_saved(P, dev)
        B = scene.shade(T["points"], T["normals"], T["albedo"], saved=sv)
        torch.cuda.synchronize()
        assert scene.device_status() == 0
        f, k = scene.saved_views(sv, P)
        out[name] = (B.cpu().numpy(), f.cpu().numpy(), k.cpu().numpy().astype(np.int64))
        scene.close()
    np.testing.assert_array_equal(out[prec][1], out["fp32"][1])
    np.testing.assert_array_equal(out[prec][2], out["fp32"][2])
    ref = O.shade_forward(O.Config(n_bands=8), *[sc[x] for x in FIELDS], k=out["fp32"][2])["radiance"]
    e32 = rel_err(out["fp32"][0], ref).max()
    etc = rel_err(out[prec][0], ref).max()
    print(f"{prec}: max normalised radiance error {etc:.2e} (fp32 path {e32:.2e})")
    assert e32 <= 1e-4
    assert etc <= tol
