"""The oracle's hand-written adjoint against central finite differences of its
own forward pass (pins the reverse-mode steps, not the forward)."""

import numpy as np
import pytest

from oracle import shs_oracle as O
from paper_2104_00359_gb300 import synthetic as S


def _scene(seed, P, N, n, inside=0.0):
    sc = S.random_scene(seed, P, N, n, inside_fraction=inside)
    out = {k: sc[k].astype(np.float64) for k in ("points", "normals", "albedo", "centers", "radii", "light")}
    # keep every pair away from the singular tangency D = r (FD across it is
    # meaningless); points strictly inside stay (clamped cap, zero d/d cos a)
    D = np.linalg.norm(out["centers"][None] - out["points"][:, None], axis=-1)
    gap = np.abs(D - out["radii"][None]) / out["radii"][None]
    keep = np.all(gap > 0.05, axis=1)
    for k in ("points", "normals", "albedo"):
        out[k] = out[k][keep]
    return out


ORDER = ("points", "normals", "albedo", "centers", "radii", "light")


@pytest.mark.parametrize("n,fixed_k,inside", [(4, 2, 0.0), (3, 0, 0.3), (5, 3, 0.2)])
def test_adjoint_matches_central_differences(n, fixed_k, inside):
    sc = _scene(30 + n, 10, 5, n, inside)
    cfg = O.Config(n_bands=n, fixed_k=fixed_k)
    rng = np.random.default_rng(31)
    dB = rng.normal(size=sc["points"].shape)
    g = O.shade_backward(cfg, *[sc[k] for k in ORDER], dB)
    grads = dict(points=g["d_points"], normals=g["d_normals"], albedo=g["d_albedo"],
                 centers=g["d_centers"], radii=g["d_radii"], light=g["d_light"])

    def loss(arrs):
        return float(np.sum(dB * O.shade_forward(cfg, *[arrs[k] for k in ORDER])["radiance"]))

    h = 1e-6
    for name in ORDER:
        base = sc[name]
        fd = np.zeros_like(base)
        it = np.nditer(base, flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            plus = dict(sc)
            minus = dict(sc)
            plus[name] = base.copy()
            minus[name] = base.copy()
            plus[name][idx] += h
            minus[name][idx] -= h
            fd[idx] = (loss(plus) - loss(minus)) / (2 * h)
        scale = max(np.abs(fd).max(), 1e-3)
        np.testing.assert_allclose(grads[name], fd, atol=2e-7 * scale + 1e-9, err_msg=name)


def test_adjoint_with_free_k_away_from_boundaries():
    """Per-point k (no override): small perturbations keep every k, so the
    adjoint still matches FD (k is piecewise constant, its gradient is 0)."""
    sc = _scene(40, 12, 6, 4)
    cfg = O.Config(n_bands=4, exp_tau=0.5)
    fw = O.shade_forward(cfg, *[sc[k] for k in ORDER])
    assert fw["k"].max() >= 2
    dB = np.random.default_rng(41).normal(size=sc["points"].shape)
    g = O.shade_backward(cfg, *[sc[k] for k in ORDER], dB)
    h = 1e-6
    for j in range(sc["centers"].shape[0]):
        for c in range(3):
            p = dict(sc)
            m = dict(sc)
            p["centers"] = sc["centers"].copy()
            m["centers"] = sc["centers"].copy()
            p["centers"][j, c] += h
            m["centers"][j, c] -= h
            fp = O.shade_forward(cfg, *[p[k] for k in ORDER])
            fm = O.shade_forward(cfg, *[m[k] for k in ORDER])
            assert np.array_equal(fp["k"], fw["k"]) and np.array_equal(fm["k"], fw["k"])
            fd = np.sum(dB * (fp["radiance"] - fm["radiance"])) / (2 * h)
            assert abs(fd - g["d_centers"][j, c]) < 2e-7 * max(1.0, abs(fd))


def test_adjoint_with_horizon_cull():
    """Horizon culling is a per-pair selection with no gradient: away from its
    boundary the adjoint still matches central differences."""
    sc = _scene(44, 10, 6, 4)
    cfg = O.Config(n_bands=4, fixed_k=2, horizon_cull=True)
    nh = sc["normals"] / np.linalg.norm(sc["normals"], axis=1, keepdims=True)
    margin = np.einsum("pjc,pc->pj", sc["centers"][None] - sc["points"][:, None], nh) + sc["radii"][None]
    assert (margin < 0).any() and (margin > 0).any()           # some pairs culled, some kept
    keep = np.all(np.abs(margin) > 1e-3, axis=1)
    for k in ("points", "normals", "albedo"):
        sc[k] = sc[k][keep]
    dB = np.random.default_rng(45).normal(size=sc["points"].shape)
    g = O.shade_backward(cfg, *[sc[k] for k in ORDER], dB)
    h = 1e-6
    for name, grad in (("centers", g["d_centers"]), ("radii", g["d_radii"]), ("points", g["d_points"])):
        base = sc[name]
        it = np.nditer(base, flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            p, m = dict(sc), dict(sc)
            p[name], m[name] = base.copy(), base.copy()
            p[name][idx] += h
            m[name][idx] -= h
            fd = np.sum(dB * (O.shade_forward(cfg, *[p[k] for k in ORDER])["radiance"]
                              - O.shade_forward(cfg, *[m[k] for k in ORDER])["radiance"])) / (2 * h)
            assert abs(fd - grad[idx]) < 2e-7 * max(1.0, abs(fd)), (name, idx, fd, grad[idx])


def test_adjoint_of_projected_exponential():
    """The projected-exponential variant's adjoint against central differences."""
    sc = _scene(46, 8, 5, 4)
    cfg = O.Config(n_bands=4, exp_mode=1)
    dB = np.random.default_rng(47).normal(size=sc["points"].shape)
    g = O.shade_backward(cfg, *[sc[k] for k in ORDER], dB)
    grads = dict(points=g["d_points"], normals=g["d_normals"], albedo=g["d_albedo"],
                 centers=g["d_centers"], radii=g["d_radii"], light=g["d_light"])
    h = 1e-6
    for name in ("centers", "radii", "points", "normals", "light"):
        base = sc[name]
        fd = np.zeros_like(base)
        it = np.nditer(base, flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            p, m = dict(sc), dict(sc)
            p[name], m[name] = base.copy(), base.copy()
            p[name][idx] += h
            m[name][idx] -= h
            fd[idx] = np.sum(dB * (O.shade_forward(cfg, *[p[k] for k in ORDER])["radiance"]
                                   - O.shade_forward(cfg, *[m[k] for k in ORDER])["radiance"])) / (2 * h)
        scale = max(np.abs(fd).max(), 1e-3)
        np.testing.assert_allclose(grads[name], fd, atol=2e-7 * scale + 1e-9, err_msg=name)


def test_adjoint_of_fitted_table_step():
    """exp_mode 2 with the stored fitted table: adjoint against central
    differences (through a(s), b(s) and their slopes)."""
    import os
    from oracle import fit_ol_table as F
    tab = F.read_table(os.path.join(os.path.dirname(__file__), "golden", "ol_table_n4.txt"))
    sc = _scene(48, 8, 5, 4)
    cfg = O.Config(n_bands=4, exp_mode=2, ol_table=tab)
    dB = np.random.default_rng(49).normal(size=sc["points"].shape)
    g = O.shade_backward(cfg, *[sc[k] for k in ORDER], dB)
    grads = dict(points=g["d_points"], normals=g["d_normals"], albedo=g["d_albedo"],
                 centers=g["d_centers"], radii=g["d_radii"], light=g["d_light"])
    h = 1e-6
    for name in ("centers", "radii", "points", "normals", "light"):
        base = sc[name]
        fd = np.zeros_like(base)
        it = np.nditer(base, flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            p, m = dict(sc), dict(sc)
            p[name], m[name] = base.copy(), base.copy()
            p[name][idx] += h
            m[name][idx] -= h
            fd[idx] = np.sum(dB * (O.shade_forward(cfg, *[p[k] for k in ORDER])["radiance"]
                                   - O.shade_forward(cfg, *[m[k] for k in ORDER])["radiance"])) / (2 * h)
        scale = max(np.abs(fd).max(), 1e-3)
        np.testing.assert_allclose(grads[name], fd, atol=2e-7 * scale + 1e-9, err_msg=name)
