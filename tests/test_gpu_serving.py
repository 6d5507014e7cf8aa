"""Continuous-batching server: every request's result is the same when it
runs alone (per-call API) and inside mixed batches; jobs are admitted under
the HBM budget; batches overlap on the device."""

import numpy as np
import pytest

from oracle import shs_oracle as O
from paper_2104_00359_gb300 import synthetic as S

from gpu_helpers import FIELDS, grad_err, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _jobs(seed=0, n_jobs=6):
    rng = np.random.default_rng(seed)
    out = []
    for j in range(n_jobs):
        n = 4 if j % 3 else 6
        P = int(rng.integers(300, 3000))
        N = int(rng.integers(20, 70))
        sc = S.random_scene(1000 + j, P, N, n, inside_fraction=0.05)
        tg = S.perturb_scene(sc, 2000 + j)
        target = O.shade_forward(O.Config(n_bands=n), *[tg[f] for f in FIELDS])["radiance"].astype(np.float32)
        out.append((j, sc, target))
    return out


@pytest.mark.parametrize("chunk_points", [None, 512])
def test_mixed_batches_match_requests_alone(chunk_points):
    """With chunk_points = 512 every job of more than 512 points runs as
    chunks with their own scenes, spread over several batches, and its scene
    gradients and loss are summed from the chunks'."""
    import torch
    from paper_2104_00359_gb300 import Config, serve
    jobs = _jobs()
    srv = serve.Server(hbm_budget_bytes=2e9, n_slots=3, max_batch=4,
                       chunk_points=chunk_points or serve.CHUNK_POINTS)
    for j, sc, target in jobs:
        assert srv.add_job(j, sc["points"], sc["normals"], sc["albedo"], sc["centers"], sc["radii"],
                           sc["light"], Config(n_bands=sc["n_bands"]), target=target)
    if chunk_points:
        assert sum(len(job.ranges) > 1 for job in srv.jobs.values()) >= 4
    # alone: per-call API on each job's resident buffers
    alone = {}
    runner = serve.PerCallRunner(srv.jobs)
    for j, sc, _ in jobs:
        for op in ("fwd", "fwdbwd"):
            ev = runner.run(serve.Request(-1, j, op, 0.0))
            ev.synchronize()
            job = srv.jobs[j]
            res = {"radiance": job.radiance.cpu().numpy().copy()}
            if op == "fwdbwd":
                res.update({k: v.cpu().numpy().copy() for k, v in job.grads.items() if v is not None})
                res["loss"] = float(job.loss)
            alone[(j, op)] = res
    # mixed: 40 requests submitted in bursts while batches are in flight
    results = []

    def grab(r, job):
        res = {"radiance": job.radiance.cpu().numpy().copy()}
        if r.op == "fwdbwd":
            res.update({k: v.cpu().numpy().copy() for k, v in job.grads.items() if v is not None})
            res["loss"] = float(job.loss)
        results.append((r, res))

    rng = np.random.default_rng(1)
    for burst in range(8):
        for _ in range(5):
            j = int(rng.integers(0, len(jobs)))
            srv.submit(j, "fwdbwd" if rng.random() < 0.4 else "fwd", on_done=grab)
        srv.poll()
    srv.drain()
    assert len(results) == 40
    assert srv.batches >= 2 and srv.max_inflight >= 2
    by_job = {j: sc for j, sc, _ in jobs}
    for r, res in results:
        ref = alone[(r.job_id, r.op)]
        assert rel_err(res["radiance"], ref["radiance"]).max() <= TOL
        if r.op == "fwdbwd":
            # the batched adjoint against the FP64 oracle, for the L2 loss of
            # the radiance this request computed, and against the result alone
            sc = by_job[r.job_id]
            dB = res["radiance"].astype(np.float64) - jobs[r.job_id][2]
            o = O.shade_backward(O.Config(n_bands=sc["n_bands"]), *[sc[f] for f in FIELDS], dB)
            for name in ("d_light", "d_albedo", "d_centers", "d_radii"):
                assert grad_err(name, res[name], o).max() <= TOL, (r.req_id, name, "vs oracle")
                base = dict(o)
                base[name] = ref[name]
                assert grad_err(name, res[name], base).max() <= TOL, (r.req_id, name, "vs alone")
            loss_ref = 0.5 * float(np.sum(dB ** 2))
            assert abs(res["loss"] - loss_ref) <= 1e-5 * loss_ref
            assert abs(res["loss"] - ref["loss"]) <= 1e-5 * abs(ref["loss"])
    srv.close()


def test_admission_under_hbm_budget():
    from paper_2104_00359_gb300 import Config, serve
    jobs = _jobs(seed=3, n_jobs=3)
    sizes = [serve.Job.device_bytes(len(sc["points"]), len(sc["centers"]), sc["n_bands"]) for _, sc, _ in jobs]
    budget = max(sizes[0] + sizes[1], sizes[0] + sizes[2]) + 1
    assert budget < sum(sizes)
    srv = serve.Server(hbm_budget_bytes=budget, n_slots=2, max_batch=4)
    admitted = [srv.add_job(j, sc["points"], sc["normals"], sc["albedo"], sc["centers"], sc["radii"], sc["light"],
                            Config(n_bands=sc["n_bands"]), target=t) for j, sc, t in jobs]
    assert admitted == [True, True, False]
    assert srv.used <= budget
    r2 = srv.submit(2, "fwd")             # waits: job 2 not resident yet
    r0 = srv.submit(0, "fwd")
    for _ in range(200):
        srv.poll()
        if r0.done:
            break
    assert r0.done and not r2.done and not srv.admitted(2)
    srv.remove_job(1)                     # frees memory: job 2 is admitted
    assert srv.admitted(2) and srv.used <= budget
    srv.drain()
    assert r2.done > 0
    srv.close()
