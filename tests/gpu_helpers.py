"""Shared helpers of the GPU parity tests: run the CUDA library through its
Python binding and compare with the FP64 oracle on the same float32 inputs."""

import numpy as np

from oracle import shs_oracle as O

FIELDS = ("points", "normals", "albedo", "centers", "radii", "light")
GRADS = ("d_light", "d_albedo", "d_centers", "d_radii", "d_points", "d_normals")


def rel_err(got, ref, floor_frac=1e-3):
    """|got - ref| / max(|ref|, floor_frac * max|ref|), elementwise: the
    normalised error used for every parity gate (radiance can be ~0 in shadow
    or negative from SH ringing, so a pure relative error is undefined)."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    if ref.size == 0:
        return np.zeros(0)
    floor = floor_frac * max(np.abs(ref).max(), 1e-30)
    return np.abs(got - ref) / np.maximum(np.abs(ref), floor)


def grad_err(name, got, ref):
    """Normalised error of a gradient output.  Outputs that are sums which may
    cancel (d_light, d_centers, d_radii over points; d_points over spheres)
    also include 1e-2 x the sum of absolute terms in their scale:
    float32 summation of P terms in any order is accurate to a few ulps of that
    sum, so 1e-4 of this scale (1e-6 of the absolute sum) is a rounding-level
    gate, not a loosened one."""
    err = rel_err(got, ref[name])
    a = ref.get("abs_" + name)
    if a is not None:
        r = np.asarray(ref[name], np.float64)
        floor = 1e-3 * max(np.abs(r).max(), 1e-30)
        scale = np.maximum(np.maximum(np.abs(r), floor), 1e-2 * a)
        err = np.abs(np.asarray(got, np.float64) - r) / scale
    return err


def to_dev(sc, dev):
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(sc[k])).to(dev) for k in FIELDS}


def gpu_run(sc, cfg, dB=None, want=None, saved=True, l2_target=None):
    """Forward (+ backward) on cuda:0.  Returns numpy radiance, per-point k,
    gradients dict and the scene's device status."""
    import torch
    from paper_2104_00359_gb300 import Config, Scene
    dev = torch.device("cuda:0")
    T = to_dev(sc, dev)
    N = sc["centers"].shape[0]
    scene = Scene(T["centers"] if N else None, T["radii"] if N else None, T["light"],
                  Config(n_bands=cfg.n_bands, epsilon=cfg.epsilon, exp_tau=cfg.exp_tau,
                         exp_kmax=cfg.exp_kmax, fixed_k=cfg.fixed_k,
                         deterministic=getattr(cfg, "deterministic", True),
                         horizon_cull=getattr(cfg, "horizon_cull", False),
                         exp_mode=getattr(cfg, "exp_mode", 0)))
    if getattr(cfg, "exp_mode", 0) == 2:
        scene.set_ol_table(*cfg.ol_table)
    P = sc["points"].shape[0]
    K = cfg.n_bands ** 2
    sv = scene.new_saved(P, dev)
    B = scene.shade(T["points"], T["normals"], T["albedo"], saved=sv)
    out = {}
    if dB is not None or l2_target is not None:
        w = want or scene.ALL
        if l2_target is not None:
            tgt = torch.from_numpy(np.ascontiguousarray(l2_target)).to(dev)
            g = scene.backward_l2(T["points"], T["normals"], T["albedo"], B, tgt,
                                  saved=sv if saved else None, want=w)
        else:
            g = scene.backward(T["points"], T["normals"], T["albedo"],
                               torch.from_numpy(np.ascontiguousarray(dB, np.float32)).to(dev),
                               saved=sv if saved else None, want=w)
        torch.cuda.synchronize()
        out = {k: (v.cpu().numpy() if v is not None else None) for k, v in g.items()}
    torch.cuda.synchronize()
    fv, kv = scene.saved_views(sv, P)
    k = kv.cpu().numpy().astype(np.int64)
    f = fv.cpu().numpy()
    assert k.min(initial=0) >= 0 and k.max(initial=0) <= 16
    status = scene.device_status()
    scene.close()
    return B.cpu().numpy(), k, f, out, status


def oracle_k_consistent(cfg, f_ref, k_gpu):
    """Points whose GPU k differs from the oracle's must sit at a boundary
    |f_hat| = tau 2^k (a float32 rounding tie).  Returns the mismatch count."""
    k_ref = O.exp_scaling_k(cfg, f_ref)
    bad = np.nonzero(k_ref != k_gpu)[0]
    if bad.size:
        nrm = np.sqrt(np.sum(f_ref[bad, 1:] ** 2, axis=1))
        edge = cfg.exp_tau * 2.0 ** np.minimum(k_ref[bad], k_gpu[bad])
        assert np.all(np.abs(nrm - edge) <= 1e-4 * edge), (bad, nrm, edge)
    return bad.size
