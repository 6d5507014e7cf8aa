"""Parity at the benchmark's full size and launch configuration: the 512x512
capsule-body G-buffer (262,144 points), 100 spheres, n = 4, forward + L2 loss
+ backward exactly as bench.py times it.  Per-point outputs are compared on a
random sample the oracle computes one by one; the scene-level sums over all
262,144 points are recomputed by the oracle in float64 across a spawn process
pool (started before any GPU work of this module)."""

import multiprocessing as mp
import os

import numpy as np
import pytest

from oracle import shs_oracle as O
from paper_2104_00359_gb300 import synthetic as S

from gpu_helpers import FIELDS, grad_err, oracle_k_consistent, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-4
N_SAMPLE = 2048


def _oracle_chunk(args):
    idx, dB, k = args
    sc = S.capsule_body_scene(seed=1, n_bands=4)
    cfg = O.Config(n_bands=4)
    g = O.shade_backward(cfg, *[sc[f][idx] if f in ("points", "normals", "albedo") else sc[f] for f in FIELDS],
                         dB, k=k)
    return {n: g[n] for n in ("d_light", "d_centers", "d_radii", "abs_d_light", "abs_d_centers", "abs_d_radii")}


@pytest.fixture(scope="module")
def pool():
    ctx = mp.get_context("spawn")
    p = ctx.Pool(processes=max(1, min(16, os.cpu_count() or 1)))
    yield p
    p.close()
    p.join()


def test_capsule_body_full_size(pool):
    import torch
    from paper_2104_00359_gb300 import Config, Scene
    sc = S.capsule_body_scene(seed=1, n_bands=4)
    tg = S.perturb_scene(sc, seed=2)
    dev = torch.device("cuda:0")
    T = {k: torch.from_numpy(sc[k]).to(dev) for k in FIELDS}
    cfg = Config(n_bands=4)
    tscene = Scene(torch.from_numpy(tg["centers"]).to(dev), torch.from_numpy(tg["radii"]).to(dev),
                   torch.from_numpy(tg["light"]).to(dev), cfg)
    target = tscene.shade(T["points"], T["normals"], torch.from_numpy(tg["albedo"]).to(dev))
    tscene.close()
    scene = Scene(T["centers"], T["radii"], T["light"], cfg)
    P = sc["points"].shape[0]
    saved = scene.new_saved(P, dev)
    B = scene.shade(T["points"], T["normals"], T["albedo"], saved=saved)
    g = scene.backward_l2(T["points"], T["normals"], T["albedo"], B, target, saved=saved,
                          want=("light", "albedo", "centers", "radii"))
    torch.cuda.synchronize()
    assert scene.device_status() == 0
    fv, kv = scene.saved_views(saved, P)
    k = kv.cpu().numpy().astype(np.int64)
    B_np = B.cpu().numpy()
    dB = (B_np.astype(np.float64) - target.cpu().numpy())
    got = {n: g[n].cpu().numpy() for n in ("d_light", "d_albedo", "d_centers", "d_radii")}
    scene.close()

    ocfg = O.Config(n_bands=4)
    rng = np.random.default_rng(0)
    sel = np.sort(rng.choice(P, N_SAMPLE, replace=False))
    args = [sc[f][sel] if f in ("points", "normals", "albedo") else sc[f] for f in FIELDS]
    ref_fw = O.shade_forward(ocfg, *args)
    oracle_k_consistent(ocfg, ref_fw["f"], k[sel])
    ref_fw = O.shade_forward(ocfg, *args, k=k[sel])
    assert rel_err(B_np[sel], ref_fw["radiance"]).max() <= TOL
    np.testing.assert_allclose(fv.cpu().numpy()[sel], ref_fw["f"], rtol=0, atol=2e-5 * np.abs(ref_fw["f"]).max())
    ref_bw = O.shade_backward(ocfg, *args, dB[sel], k=k[sel])
    assert rel_err(got["d_albedo"][sel], ref_bw["d_albedo"]).max() <= TOL

    chunks = np.array_split(np.arange(P), 64)
    parts = pool.map(_oracle_chunk, [(c, dB[c], k[c]) for c in chunks])
    ref = {n: sum(p[n] for p in parts) for n in parts[0]}
    for name in ("d_light", "d_centers", "d_radii"):
        err = grad_err(name, got[name], ref)
        assert err.max() <= TOL, f"{name}: {err.max():.3e}"
