"""Mesh-deformation batch through the library's autograd Function: gradients
with respect to the deformation parameters and each view's 6-DoF pose.

The reference chain rule runs in float64 on the oracle's adjoint (d_points,
d_normals, d_centers per view); it is itself pinned by central finite
differences of the oracle's forward pass on a reduced mesh.  The CUDA result
(float32, torch autograd over the library's adjoint) is compared with it at
the reduced size and at the full 16 views x 50,000 vertices x 200 spheres."""

import multiprocessing as mp
import os

import numpy as np
import pytest

from oracle import shs_oracle as O
from paper_2104_00359_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _rot(w):
    th = np.linalg.norm(w)
    K = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    if th < 1e-8:
        return np.eye(3) + K
    return np.eye(3) + np.sin(th) / th * K + (1 - np.cos(th)) / th ** 2 * (K @ K)


def _posed(m, p, pose):
    v = m["v0"].astype(np.float64) + m["A_v"].astype(np.float64) @ p
    n = m["n0"].astype(np.float64) + m["A_n"].astype(np.float64) @ p
    c = m["c0"].astype(np.float64) + m["A_c"].astype(np.float64) @ p
    R = _rot(pose[:3])
    return v @ R.T + pose[3:], n @ R.T, c @ R.T + pose[3:], v, n, c, R


def _view_grad(args):
    """Oracle adjoint of one view (optionally a chunk of its points) and the
    float64 chain rule to (p, pose).  Returns gradient and |term| sums."""
    m, p, pose, w, k, idx, cfg = args
    pv, pn, pc, v, n, c, R = _posed(m, p, pose)
    if idx is None:
        idx = np.arange(pv.shape[0])
    g = O.shade_backward(cfg, pv[idx], pn[idx], m["albedo"][idx], pc, m["radii"], m["light"], w[idx], k=k[idx])
    gv, gn, gc = g["d_points"], g["d_normals"], g["d_centers"]
    Av, An, Ac = (m[x].astype(np.float64) for x in ("A_v", "A_n", "A_c"))
    tv = np.einsum("mc,mcd->md", gv @ R, Av[idx])
    tn = np.einsum("mc,mcd->md", gn @ R, An[idx])
    tc = np.einsum("jc,jcd->jd", gc @ R, Ac)
    dp = tv.sum(0) + tn.sum(0) + tc.sum(0)
    adp = np.abs(tv).sum(0) + np.abs(tn).sum(0) + np.abs(tc).sum(0)
    dt = gv.sum(0) + gc.sum(0)
    adt = np.abs(gv).sum(0) + np.abs(gc).sum(0)
    dR = gv.T @ v[idx] + gn.T @ n[idx] + gc.T @ c
    adR = np.abs(gv).T @ np.abs(v[idx]) + np.abs(gn).T @ np.abs(n[idx]) + np.abs(gc).T @ np.abs(c)
    dw, adw = np.zeros(3), np.zeros(3)
    h = 1e-7
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        dRdw = (_rot(pose[:3] + e) - _rot(pose[:3] - e)) / (2 * h)
        dw[a] = np.sum(dR * dRdw)
        adw[a] = np.sum(adR * np.abs(dRdw))
    return dp, adp, np.concatenate([dw, dt]), np.concatenate([adw, adt])


def _gpu(m, p0, poses0, wts, cfg_kw, batched=False):
    """Gradients to p and the poses through the library: one chain and one
    shading call per view, or (batched) all views in one chain launch per
    array and one shading launch per pass."""
    import torch
    from paper_2104_00359_gb300 import Config, chain
    dev = torch.device("cuda:0")
    T = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in m.items() if k != "n_bands"}
    p = torch.from_numpy(p0.astype(np.float32)).to(dev).requires_grad_(True)
    poses = torch.from_numpy(poses0.astype(np.float32)).to(dev).requires_grad_(True)
    cfg = Config(n_bands=m["n_bands"], **cfg_kw)
    c0 = chain.affine_deform(T["c0"], T["A_c"], p.detach())
    scenes = chain.make_view_scenes(poses.shape[0], c0, T["radii"], T["light"], cfg)
    W = torch.from_numpy(wts.astype(np.float32)).to(dev)
    if batched:
        views = chain.ViewBatch(poses.shape[0], T["v0"].shape[0], c0, T["radii"], T["light"], cfg)
        B = chain.render_views_batched(p, poses, T, T["radii"], T["light"], T["albedo"], views)
        (B * W).sum().backward()
        torch.cuda.synchronize()
        for sc in views.scenes:
            assert sc.device_status() == 0
        views.close()
    else:
        B = chain.render_views(p, poses, T, T["radii"], T["light"], T["albedo"], scenes)
        (B * W).sum().backward()
    # per-point squaring counts of every view, for the oracle
    ks = []
    with torch.no_grad():
        for i, sc in enumerate(scenes):
            q = poses[i].detach()
            pv = chain.deform_pose(T["v0"], T["A_v"], p.detach(), q)
            pn = chain.deform_pose(T["n0"], T["A_n"], p.detach(), q, direction=True)
            pc = chain.deform_pose(T["c0"], T["A_c"], p.detach(), q)
            sc.update(pc, T["radii"], T["light"])
            sv = sc.new_saved(pv.shape[0], dev)
            sc.shade(pv, pn, T["albedo"], saved=sv)
            ks.append(sc.saved_views(sv, pv.shape[0])[1].cpu().numpy().astype(np.int64))
    torch.cuda.synchronize()
    for sc in scenes:
        sc.close()
    return p.grad.cpu().numpy(), poses.grad.cpu().numpy(), ks


def _check(got, ref, aref, name):
    scale = np.maximum(np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max()), 1e-2 * aref)
    err = np.abs(got - ref) / scale
    assert err.max() <= TOL, f"{name}: {err.max():.3e}"


@pytest.mark.parametrize("batched", [False, True])
def test_chain_reduced_against_finite_differences(batched):
    m = S.mesh_deformation_scene(seed=5, n_theta=30, n_phi=20, n_spheres=30, n_params=8, n_views=2)
    rng = np.random.default_rng(6)
    p0 = rng.normal(0, 0.5, 8)
    poses0 = m["poses"].astype(np.float64)
    wts = rng.normal(size=(2, m["v0"].shape[0], 3))
    cfg = O.Config(n_bands=4, fixed_k=3)
    # the reference chain rule against central differences of the oracle forward
    args = [(m, p0, poses0[i], wts[i], np.full(m["v0"].shape[0], 3), None, cfg) for i in range(2)]
    parts = [_view_grad(a) for a in args]
    dp = sum(x[0] for x in parts)
    dpose = np.stack([x[2] for x in parts])

    def loss(p, poses):
        tot = 0.0
        for i in range(2):
            pv, pn, pc, *_ = _posed(m, p, poses[i])
            tot += np.sum(wts[i] * O.shade_forward(cfg, pv, pn, m["albedo"], pc, m["radii"], m["light"])["radiance"])
        return tot

    h = 1e-6
    for d in range(8):
        e = np.zeros(8)
        e[d] = h
        fd = (loss(p0 + e, poses0) - loss(p0 - e, poses0)) / (2 * h)
        assert abs(fd - dp[d]) <= 1e-6 * max(1.0, abs(fd)), (d, fd, dp[d])
    for i in range(2):
        for d in range(6):
            e = np.zeros_like(poses0)
            e[i, d] = h
            fd = (loss(p0, poses0 + e) - loss(p0, poses0 - e)) / (2 * h)
            assert abs(fd - dpose[i, d]) <= 1e-6 * max(1.0, abs(fd)), (i, d, fd, dpose[i, d])
    # the CUDA path against the reference
    gp, gpose, _ = _gpu(m, p0, poses0, wts, dict(fixed_k=3), batched=batched)
    _check(gp, dp, sum(x[1] for x in parts), "d_p")
    _check(gpose, dpose, np.stack([x[3] for x in parts]), "d_pose")


def test_chain_full_size_16_views():
    """16 views x 50,000 vertices x 200 spheres, 60 deformation parameters."""
    m = S.mesh_deformation_scene()
    rng = np.random.default_rng(7)
    p0 = rng.normal(0, 0.5, 60)
    poses0 = m["poses"].astype(np.float64)
    V, M = poses0.shape[0], m["v0"].shape[0]
    wts = rng.normal(size=(V, M, 3))
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(processes=max(1, min(16, os.cpu_count() or 1)))
    try:
        gp, gpose, ks = _gpu(m, p0, poses0, wts, {})
        gpb, gposeb, _ = _gpu(m, p0, poses0, wts, {}, batched=True)
        cfg = O.Config(n_bands=4)
        chunks = np.array_split(np.arange(M), 4)
        tasks = [(m, p0, poses0[i], wts[i], ks[i], c, cfg) for i in range(V) for c in chunks]
        parts = pool.map(_view_grad, tasks)
    finally:
        pool.close()
        pool.join()
    dp = sum(x[0] for x in parts)
    adp = sum(x[1] for x in parts)
    dpose = np.stack([sum(parts[i * 4 + c][2] for c in range(4)) for i in range(V)])
    adpose = np.stack([sum(parts[i * 4 + c][3] for c in range(4)) for i in range(V)])
    _check(gp, dp, adp, "d_p")
    _check(gpose, dpose, adpose, "d_pose")
    _check(gpb, dp, adp, "d_p (batched views)")
    _check(gposeb, dpose, adpose, "d_pose (batched views)")
