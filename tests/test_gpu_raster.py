"""Rasterisation of shaded vertices (shs_rasterize / shs_rasterize_backward)
against the FP64 brute-force rasteriser of oracle/raster_oracle.py.

float32 and float64 may assign a pixel whose centre lies on a shared edge (or
two triangles at nearly equal depth) differently; such pixels must be rare
and lie on an edge, and the colours and gradients are compared on the GPU's
own assignment (the oracle's adjoint takes the face map as input)."""

import numpy as np
import pytest

from oracle import raster_oracle as R
from oracle import shs_oracle as O
from paper_2104_00359_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


def _mesh(n_theta=20, n_phi=24, seed=2):
    m = S.mesh_deformation_scene(seed=seed, n_theta=n_theta, n_phi=n_phi, n_spheres=8, n_params=4, n_views=2)
    return m, S.uv_grid_faces(n_theta, n_phi)


def _gpu(v, faces, P, B, H, W, dI=None):
    import torch
    from paper_2104_00359_gb300.raster import rasterize
    dev = torch.device("cuda:0")
    vt = torch.from_numpy(np.ascontiguousarray(v, np.float32)).to(dev).requires_grad_(dI is not None)
    bt = torch.from_numpy(np.ascontiguousarray(B, np.float32)).to(dev).requires_grad_(dI is not None)
    ft = torch.from_numpy(np.ascontiguousarray(faces, np.int32)).to(dev)
    img, fi = rasterize(vt, bt, ft, P, H, W)
    out = dict(image=img.detach().cpu().numpy(), face_index=fi.cpu().numpy().astype(np.int64))
    if dI is not None:
        (img * torch.from_numpy(np.ascontiguousarray(dI, np.float32)).to(dev)).sum().backward()
        out["d_vertices"] = vt.grad.cpu().numpy()
        out["d_radiance"] = bt.grad.cpu().numpy()
    torch.cuda.synchronize()
    return out


def _edge_distance(v, faces, P, face_idx):
    """Smallest screen-space barycentric of each pixel in its (oracle) face."""
    clip = R.project(v, P)
    q = R.pixel_centres(*face_idx.shape)
    out = np.full(face_idx.shape, np.inf)
    for r, c in zip(*np.nonzero(face_idx >= 0)):
        ids = faces[face_idx[r, c]]
        n = clip[ids, :2] / clip[ids, 3:4]
        E = np.array(R._edges(n[0], n[1], n[2], q[r, c]))
        out[r, c] = (E / E.sum()).min()
    return out


@pytest.mark.parametrize("H,W", [(48, 48), (37, 61)])
def test_forward_matches_oracle(H, W):
    m, faces = _mesh()
    P = S.look_at_perspective((2.5, 1.0, 1.2), aspect=W / H)
    B = m["albedo"]
    got = _gpu(m["v0"], faces, P, B, H, W)
    ref_img, ref_fi = R.rasterize(m["v0"], faces, P, B, H, W)
    diff = got["face_index"] != ref_fi
    assert diff.mean() < 0.01, diff.mean()
    if diff.any():
        # disagreements sit on edges of the oracle's (or the GPU's) triangle
        d_ref = _edge_distance(m["v0"], faces, P, np.where(diff, ref_fi, -1))
        d_got = _edge_distance(m["v0"], faces, P, np.where(diff, got["face_index"], -1))
        near = np.minimum(np.abs(d_ref), np.abs(d_got))      # background side: inf
        assert np.all(near[diff] < 1e-4), near[diff].max()
    same = ~diff
    # colours on the GPU's assignment
    ref_same = R.shade_pixels(m["v0"], faces, P, B, got["face_index"])
    err = np.abs(got["image"] - ref_same).max()
    assert err <= 1e-5 * np.abs(ref_same).max(), err
    assert np.array_equal(got["image"][same & (ref_fi < 0)], np.zeros(((same & (ref_fi < 0)).sum(), 3)))


def test_backward_matches_oracle():
    m, faces = _mesh()
    H = W = 40
    P = S.look_at_perspective((2.2, -1.0, 1.5))
    B = m["albedo"]
    dI = np.random.default_rng(3).normal(size=(H, W, 3))
    got = _gpu(m["v0"], faces, P, B, H, W, dI=dI)
    ref = R.rasterize_backward(m["v0"], faces, P, B, got["face_index"], dI)
    for name in ("d_radiance", "d_vertices"):
        r, g = ref[name], got[name]
        err = np.abs(g - r) / np.maximum(np.abs(r), 1e-2 * np.abs(r).max())
        assert err.max() <= 1e-3, f"{name}: {err.max():.3e}"


def test_empty_and_culled_inputs():
    import torch
    from paper_2104_00359_gb300.raster import rasterize
    dev = torch.device("cuda:0")
    v = torch.tensor([[-1.0, -1.0, -3.0], [1.0, -1.0, -3.0], [0.0, 1.0, 1.0]], device=dev)   # one vertex behind
    b = torch.ones((3, 3), device=dev)
    P = S.look_at_perspective((0.0, 0.0, 0.0), target=(0.0, 0.0, -1.0), up=(0.0, 1.0, 0.0))
    img, fi = rasterize(v, b, torch.tensor([[0, 1, 2]], dtype=torch.int32, device=dev), P, 8, 8)
    assert torch.all(fi == -1) and torch.all(img == 0)
    img, fi = rasterize(v, b, torch.zeros((0, 3), dtype=torch.int32, device=dev), P, 5, 7)
    assert img.shape == (5, 7, 3) and torch.all(fi == -1)


def test_image_loss_reaches_the_lighting():
    """Closing the loop: image-space L2 (Sec. 3.5's objective) through the
    rasteriser and the shading path to the SH lighting, against the oracle
    chain (raster adjoint -> shading adjoint) on the GPU's face map."""
    import torch
    from paper_2104_00359_gb300 import Config, Scene, shade
    from paper_2104_00359_gb300.raster import rasterize
    m, faces = _mesh(16, 20, seed=4)
    H = W = 32
    P = S.look_at_perspective((2.4, 0.8, 1.0))
    dev = torch.device("cuda:0")
    T = {k: torch.from_numpy(np.ascontiguousarray(m[k])).to(dev) for k in ("v0", "n0", "albedo", "c0", "radii", "light")}
    light = T["light"].clone().requires_grad_(True)
    scene = Scene(T["c0"], T["radii"], light.detach(), Config(n_bands=4))
    Bv = shade(T["v0"], T["n0"], T["albedo"], T["c0"], T["radii"], light, scene)
    img, fi = rasterize(T["v0"], Bv, torch.from_numpy(faces).to(dev), P, H, W)
    target = torch.from_numpy(np.random.default_rng(5).uniform(0, 1, (H, W, 3)).astype(np.float32)).to(dev)
    loss = 0.5 * ((img - target) ** 2).sum()
    loss.backward()
    scene.close()
    cfg = O.Config(n_bands=4)
    args = [m[k] for k in ("v0", "n0", "albedo", "c0", "radii", "light")]
    fw = O.shade_forward(cfg, *args)
    fimap = fi.cpu().numpy().astype(np.int64)
    ref_img = R.shade_pixels(m["v0"], faces, P, fw["radiance"], fimap)
    dB = R.rasterize_backward(m["v0"], faces, P, fw["radiance"], fimap,
                              ref_img - target.cpu().numpy())["d_radiance"]
    g = O.shade_backward(cfg, *args, dB)
    ref, a = g["d_light"], g["abs_d_light"]
    got = light.grad.cpu().numpy()
    err = np.abs(got - ref) / np.maximum(np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max()), 1e-2 * a)
    assert err.max() <= 1e-3, err.max()
