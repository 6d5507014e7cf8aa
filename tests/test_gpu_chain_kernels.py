"""The scene-chain kernels (shs_chain_forward / shs_chain_backward: linear
deformation and rigid pose, Sec. 3.3.1 and Sec. 3.5) against the FP64 chain
oracle, element by element, including the mesh-deformation workload's full
size (50,000 rows x 60 parameters)."""

import ctypes

import numpy as np
import pytest

from oracle import chain_oracle as C

pytestmark = pytest.mark.gpu


def _case(M, D, wscale, seed):
    rng = np.random.default_rng(seed)
    base = rng.normal(size=(M, 3)).astype(np.float32)
    basis = rng.normal(0.0, 0.01, size=(M, 3, D)).astype(np.float32)
    p = rng.normal(size=D).astype(np.float32)
    ax = rng.normal(size=3)
    ax /= np.linalg.norm(ax)
    pose = np.concatenate([ax * wscale, rng.normal(0.0, 0.1, 3)]).astype(np.float32)
    g = rng.normal(size=(M, 3)).astype(np.float32)
    return base, basis, p, pose, g


def _run(base, basis, p, pose, g, direction):
    import torch
    from paper_2104_00359_gb300 import _lib
    from paper_2104_00359_gb300._lib import check, ptr
    lib = _lib.load()
    dev = torch.device("cuda:0")
    T = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (base, basis, p, pose, g)]
    M, D = base.shape[0], p.shape[0]
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    x = torch.full((M, 3), np.nan, dtype=torch.float32, device=dev)
    xr = torch.full((M, 3), np.nan, dtype=torch.float32, device=dev)
    check(lib.shs_chain_forward(ptr(T[0]), ptr(T[1]), M, D, ptr(T[2]), ptr(T[3]), int(direction), ptr(xr), ptr(x), s),
          "forward")
    nbytes = lib.shs_chain_workspace_bytes(M, D)
    ws = torch.empty(max(nbytes, 16) // 4, dtype=torch.float32, device=dev)
    d_p = torch.full((D,), np.nan, dtype=torch.float32, device=dev)
    d_pose = torch.full((6,), np.nan, dtype=torch.float32, device=dev)
    check(lib.shs_chain_backward(ptr(T[0]), ptr(T[1]), M, D, ptr(T[2]), ptr(T[3]), int(direction), ptr(T[4]),
                                 ptr(d_p), ptr(d_pose), ptr(ws), ws.numel() * 4, s), "backward")
    torch.cuda.synchronize()
    return x.cpu().numpy(), xr.cpu().numpy(), d_p.cpu().numpy(), d_pose.cpu().numpy()


def _sum_err(got, ref, aref):
    scale = np.maximum(np.maximum(np.abs(ref), 1e-3 * max(np.abs(ref).max(), 1e-30)), 1e-2 * aref)
    return (np.abs(got - ref) / scale).max()


@pytest.mark.parametrize("M,D,wscale", [(1, 1, 0.0), (37, 5, 1e-5), (1000, 60, 0.7), (5003, 256, 3.0),
                                        (50000, 60, 2.2)])
@pytest.mark.parametrize("direction", [False, True])
def test_chain_kernels_match_oracle(M, D, wscale, direction):
    base, basis, p, pose, g = _case(M, D, wscale, seed=M + D)
    x, xr, d_p, d_pose = _run(base, basis, p, pose, g, direction)
    rx, rxr = C.deform_pose(base, basis, p, pose, direction)
    assert np.abs(xr - rxr).max() <= 1e-5 * np.abs(rxr).max()
    assert np.abs(x - rx).max() <= 1e-5 * np.abs(rx).max()
    ref = C.deform_pose_backward(base, basis, p, pose, g, direction)
    assert _sum_err(d_p, ref["d_p"], ref["abs_d_p"]) <= 1e-4
    assert _sum_err(d_pose, ref["d_pose"], ref["abs_d_pose"]) <= 1e-4
    if direction:
        assert np.all(d_pose[3:] == 0)


def test_chain_empty_and_invalid():
    import torch
    from paper_2104_00359_gb300 import _lib
    from paper_2104_00359_gb300._lib import ptr
    lib = _lib.load()
    dev = torch.device("cuda:0")
    p = torch.ones(4, device=dev)
    pose = torch.zeros(6, device=dev)
    d_p = torch.full((4,), 7.0, device=dev)
    d_pose = torch.full((6,), 7.0, device=dev)
    ws = torch.empty(1024, device=dev)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.shs_chain_forward(None, None, 0, 4, ptr(p), ptr(pose), 0, None, None, s) == 0
    assert lib.shs_chain_backward(None, None, 0, 4, ptr(p), ptr(pose), 0, None, ptr(d_p), ptr(d_pose), ptr(ws),
                                  4096, s) == 0
    torch.cuda.synchronize()
    assert torch.all(d_p == 0) and torch.all(d_pose == 0)
    base = torch.zeros((2, 3), device=dev)
    basis = torch.zeros((2, 3, 300), device=dev)
    x = torch.zeros((2, 3), device=dev)
    big = torch.ones(300, device=dev)
    assert lib.shs_chain_forward(ptr(base), ptr(basis), 2, 300, ptr(big), ptr(pose), 0, None, ptr(x), s) == 1
    assert lib.shs_chain_forward(ptr(base), ptr(basis), 2, 4, ptr(p), ptr(pose), 2, None, ptr(x), s) == 1
    assert lib.shs_chain_backward(ptr(base), ptr(basis), 2, 4, ptr(p), ptr(pose), 0, ptr(x), ptr(d_p), ptr(d_pose),
                                  ptr(ws), 8, s) == 1


def test_autograd_function_matches_oracle():
    import torch
    from paper_2104_00359_gb300.chain import deform_pose
    base, basis, p, pose, g = _case(777, 12, 1.3, seed=3)
    dev = torch.device("cuda:0")
    tp = torch.from_numpy(p).to(dev).requires_grad_(True)
    tq = torch.from_numpy(pose).to(dev).requires_grad_(True)
    x = deform_pose(torch.from_numpy(base).to(dev), torch.from_numpy(basis).to(dev), tp, tq)
    (x * torch.from_numpy(g).to(dev)).sum().backward()
    ref = C.deform_pose_backward(base, basis, p, pose, g)
    assert _sum_err(tp.grad.cpu().numpy(), ref["d_p"], ref["abs_d_p"]) <= 1e-4
    assert _sum_err(tq.grad.cpu().numpy(), ref["d_pose"], ref["abs_d_pose"]) <= 1e-4


@pytest.mark.parametrize("M,D,V", [(1, 3, 1), (333, 17, 5), (50000, 60, 16), (2000, 100, 32)])
@pytest.mark.parametrize("direction", [False, True])
def test_chain_views_match_oracle_per_view(M, D, V, direction):
    """shs_chain_forward_views / shs_chain_backward_views: every view against
    the oracle's single-pose chain; d_p is the sum over views of the oracle's,
    d_poses[v] view v's."""
    import torch
    from paper_2104_00359_gb300 import _lib
    from paper_2104_00359_gb300._lib import check, ptr
    rng = np.random.default_rng(M + 7 * V)
    base, basis, p, _, _ = _case(M, D, 0.0, seed=M + D + V)
    poses = np.concatenate([rng.normal(0.0, 0.8, (V, 3)), rng.normal(0.0, 0.2, (V, 3))], 1).astype(np.float32)
    g = rng.normal(size=(V, M, 3)).astype(np.float32)
    lib = _lib.load()
    dev = torch.device("cuda:0")
    T = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (base, basis, p, poses, g)]
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    x = torch.full((V, M, 3), np.nan, dtype=torch.float32, device=dev)
    check(lib.shs_chain_forward_views(ptr(T[0]), ptr(T[1]), M, D, ptr(T[2]), ptr(T[3]), V, int(direction), None,
                                      ptr(x), s), "forward views")
    nbytes = lib.shs_chain_views_workspace_bytes(M, D, V)
    ws = torch.empty(max(nbytes, 16) // 4, dtype=torch.float32, device=dev)
    d_p = torch.full((D,), np.nan, dtype=torch.float32, device=dev)
    d_poses = torch.full((V, 6), np.nan, dtype=torch.float32, device=dev)
    check(lib.shs_chain_backward_views(ptr(T[0]), ptr(T[1]), M, D, ptr(T[2]), ptr(T[3]), V, int(direction), ptr(T[4]),
                                       ptr(d_p), ptr(d_poses), ptr(ws), ws.numel() * 4, s), "backward views")
    torch.cuda.synchronize()
    x, d_p, d_poses = x.cpu().numpy(), d_p.cpu().numpy(), d_poses.cpu().numpy()
    ref_dp, abs_dp = np.zeros(D), np.zeros(D)
    for v in range(V):
        rx, _ = C.deform_pose(base, basis, p, poses[v], direction)
        assert np.abs(x[v] - rx).max() <= 1e-5 * max(np.abs(rx).max(), 1e-30), v
        ref = C.deform_pose_backward(base, basis, p, poses[v], g[v], direction)
        assert _sum_err(d_poses[v], ref["d_pose"], ref["abs_d_pose"]) <= 1e-4, v
        ref_dp += ref["d_p"]
        abs_dp += ref["abs_d_p"]
    assert _sum_err(d_p, ref_dp, abs_dp) <= 1e-4
    # more views than the limit: refused before any launch
    assert lib.shs_chain_forward_views(ptr(T[0]), ptr(T[1]), M, D, ptr(T[2]), ptr(T[3]), 33, 0, None, ptr(T[4]),
                                       s) == 1
