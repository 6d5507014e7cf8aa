"""The fitted optimal linear step of the SH exponential (exp_mode = 2, Sec.
3.3.2's optimal linear setting with tabulated a(s), b(s)): forward and adjoint
against the FP64 oracle on the same table, which the committed fit script
wrote from the oracle alone."""

import os

import numpy as np
import pytest

from oracle import fit_ol_table as F
from oracle import shs_oracle as O
from paper_2104_00359_gb300 import synthetic as S

from gpu_helpers import FIELDS, gpu_run, grad_err, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-4
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cfg(n, **kw):
    """The 8-band table at 8 bands, the 4-band one otherwise (any table is a
    valid input).  The library takes the table as float32, like every other
    input, so the oracle is given the same float32 values (the slopes of a
    table of values near 1 carry their rounding, about 1e-4 of the gradients'
    scale)."""
    a, b, s_max = F.read_table(os.path.join(GOLDEN, "ol_table_n8.txt" if n == 8 else "ol_table_n4.txt"))
    a, b = (np.asarray(x, np.float32).astype(np.float64) for x in (a, b))
    return O.Config(n_bands=n, exp_mode=2, ol_table=(a, b, s_max), **kw)


@pytest.mark.parametrize("n", [2, 4, 6, 8])
def test_ol_table_forward(n):
    sc = S.random_scene(800 + n, 397, 21, n, inside_fraction=0.1)
    cfg = _cfg(n)
    B, k, f, _, status = gpu_run(sc, cfg)
    assert status == 0
    ref = O.shade_forward(cfg, *[sc[x] for x in FIELDS])
    err = rel_err(B, ref["radiance"])
    assert err.max() <= TOL, f"radiance max err {err.max():.3e}"


@pytest.mark.parametrize("n,n_spheres", [(4, 40), (6, 12)])
def test_ol_table_backward(n, n_spheres):
    sc = S.random_scene(820 + n, 300, n_spheres, n, inside_fraction=0.1)
    cfg = _cfg(n)
    dB = np.random.default_rng(10).normal(size=sc["points"].shape).astype(np.float32)
    B, k, f, g, status = gpu_run(sc, cfg, dB=dB)
    assert status == 0
    ref = O.shade_backward(cfg, *[sc[x] for x in FIELDS], dB)
    for name in ("d_light", "d_albedo", "d_centers", "d_radii", "d_points", "d_normals"):
        err = grad_err(name, g[name], ref)
        assert err.max() <= TOL, f"{name}: max err {err.max():.3e}"


def test_gaussian_table_reproduces_mode_0():
    """A fine table sampling a = b = exp(s^2 / 8 pi) gives the default method's
    radiance to interpolation error."""
    s = np.linspace(0.0, 1.0, 2049)
    a = np.exp(s * s / (8 * np.pi))
    sc = S.random_scene(840, 300, 30, 4)
    cfg = O.Config(n_bands=4, exp_mode=2, ol_table=(a, a, 1.0))
    B2, *_ = gpu_run(sc, cfg)
    B0, *_ = gpu_run(sc, O.Config(n_bands=4))
    assert rel_err(B2, B0).max() <= 2e-5


def test_table_required_and_validated():
    import torch
    from paper_2104_00359_gb300 import Config, Scene, _lib
    dev = torch.device("cuda:0")
    light = torch.zeros((3, 16), device=dev)
    scene = Scene(None, None, light, Config(n_bands=4, exp_mode=2))
    pts = torch.zeros((4, 3), device=dev)
    nrm = torch.tensor([[0.0, 0.0, 1.0]] * 4, device=dev)
    with pytest.raises(_lib.ShsError) as e:
        scene.shade(pts, nrm, pts)
    assert e.value.status == 1
    for bad in ((np.ones(1), np.ones(1), 1.0), (np.ones(3), np.ones(3), 0.0),
                (np.array([1.0, np.nan]), np.ones(2), 1.0)):
        with pytest.raises(_lib.ShsError):
            scene.set_ol_table(*bad)
    scene.set_ol_table(np.ones(3), np.ones(3), 1.0)
    out = scene.shade(pts, nrm, pts)
    torch.cuda.synchronize()
    assert torch.all(out == 0)
    scene.close()
    plain = Scene(None, None, light, Config(n_bands=4))
    with pytest.raises(_lib.ShsError):
        plain.set_ol_table(np.ones(3), np.ones(3), 1.0)
    plain.close()


def test_ol_table_on_the_tensor_core_tail():
    """8 bands, split FP16 tensor-core squarings with the fitted step, against
    the oracle at the tensor-core gate (k from the GPU)."""
    import torch
    from paper_2104_00359_gb300 import Config, Scene
    from paper_2104_00359_gb300._lib import SHS_FP16
    sc = S.random_scene(860, 500, 30, 8, inside_fraction=0.05)
    cfg = _cfg(8)
    dev = torch.device("cuda:0")
    T = {k: torch.from_numpy(sc[k]).to(dev) for k in FIELDS}
    P = sc["points"].shape[0]
    scene = Scene(T["centers"], T["radii"], T["light"], Config(n_bands=8, precision=SHS_FP16, exp_mode=2))
    scene.set_ol_table(*cfg.ol_table)
    sv = scene.new_saved(P, dev)
    B = scene.shade(T["points"], T["normals"], T["albedo"], saved=sv)
    torch.cuda.synchronize()
    assert scene.device_status() == 0
    k = scene.saved_views(sv, P)[1].cpu().numpy().astype(np.int64)
    scene.close()
    ref = O.shade_forward(cfg, *[sc[x] for x in FIELDS], k=k)["radiance"]
    assert rel_err(B.cpu().numpy(), ref).max() <= 2e-3


def test_table_scene_in_the_serving_batch():
    """A job whose scene uses the table, batched with default jobs by the
    continuous-batching server, gives the same results as alone."""
    from paper_2104_00359_gb300 import Config, serve
    jobs = []
    for j, mode in enumerate((2, 0, 2)):
        sc = S.random_scene(880 + j, 700 + 300 * j, 30, 4, inside_fraction=0.05)
        target = np.random.default_rng(j).uniform(0, 1, sc["points"].shape).astype(np.float32)
        cfg = _cfg(4)
        jobs.append((j, sc, target, Config(n_bands=4, exp_mode=mode, ol_table=cfg.ol_table if mode == 2 else None)))
    srv = serve.Server(hbm_budget_bytes=1e9, n_slots=3, max_batch=4)
    for j, sc, target, c in jobs:
        assert srv.add_job(j, sc["points"], sc["normals"], sc["albedo"], sc["centers"], sc["radii"],
                           sc["light"], c, target=target)
    runner = serve.PerCallRunner(srv.jobs)
    alone = {}
    for j, *_ in jobs:
        runner.run(serve.Request(-1, j, "fwdbwd", 0.0)).synchronize()
        job = srv.jobs[j]
        alone[j] = (job.radiance.cpu().numpy().copy(), job.grads["d_light"].cpu().numpy().copy())
    got = {}

    def grab(r, job):
        got[r.job_id] = (job.radiance.cpu().numpy().copy(), job.grads["d_light"].cpu().numpy().copy())

    for j, *_ in jobs:
        srv.submit(j, "fwdbwd", on_done=grab)
    srv.drain()
    srv.close()
    for j, sc, target, c in jobs:
        assert rel_err(got[j][0], alone[j][0]).max() <= TOL
        assert rel_err(got[j][1], alone[j][1]).max() <= TOL
    # and the table jobs follow the oracle's table method
    ref = O.shade_forward(_cfg(4), *[jobs[0][1][x] for x in FIELDS])["radiance"]
    assert rel_err(got[0][0], ref).max() <= TOL


def test_ol_table_with_horizon_cull_backward():
    """The table step and horizon culling together (the fused backward is
    compiled per combination); points whose cull decision is within rounding
    of the tangent plane are left out, as in the culling tests."""
    sc = S.random_scene(890, 300, 33, 4, inside_fraction=0.05)
    nh = sc["normals"].astype(np.float64)
    nh /= np.linalg.norm(nh, axis=1, keepdims=True)
    d = sc["centers"].astype(np.float64)[None] - sc["points"].astype(np.float64)[:, None]
    margin = np.einsum("pjc,pc->pj", d, nh) + sc["radii"].astype(np.float64)[None]
    keep = np.all(np.abs(margin) > 1e-4 * (1.0 + np.abs(d).sum(-1)), axis=1)
    for k in ("points", "normals", "albedo"):
        sc[k] = np.ascontiguousarray(sc[k][keep])
    cfg = _cfg(4, horizon_cull=True)
    dB = np.random.default_rng(11).normal(size=sc["points"].shape).astype(np.float32)
    B, k, f, g, status = gpu_run(sc, cfg, dB=dB)
    assert status == 0
    ref = O.shade_backward(cfg, *[sc[x] for x in FIELDS], dB)
    assert rel_err(B, ref["forward"]["radiance"]).max() <= TOL
    for name in ("d_light", "d_albedo", "d_centers", "d_radii", "d_points", "d_normals"):
        err = grad_err(name, g[name], ref)
        assert err.max() <= TOL, f"{name}: max err {err.max():.3e}"
