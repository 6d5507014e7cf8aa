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
