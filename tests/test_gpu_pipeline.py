"""HostStepPipeline: pipelined host-to-host forward + L2 adjoint steps give the
same loss and gradients as the same calls made one at a time on one stream.

The pipeline only reorders copies and launches across streams; the kernels,
their inputs and the deterministic reduction are the same, so results must
match bit for bit, for every step, including steps whose buffer set was
reused while other steps were in flight."""

import numpy as np
import pytest

from paper_2104_00359_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
WANT = ("light", "albedo", "centers", "radii", "points")


def _inputs(seed, P):
    rng = np.random.default_rng(seed)
    sc = S.random_scene(seed, P, 23, 4, inside_fraction=0.05)
    tgt = rng.normal(0.5, 0.2, size=(P, 3)).astype(np.float32)
    return sc, tgt


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_pipeline_matches_direct_calls(depth):
    import torch
    from paper_2104_00359_gb300 import Config, Scene
    from paper_2104_00359_gb300.pipeline import HostStepPipeline
    dev = torch.device("cuda:0")
    P = 3001
    base, _ = _inputs(40, P)
    scene = Scene(*(torch.from_numpy(base[k]).to(dev) for k in ("centers", "radii", "light")),
                  Config(n_bands=4, deterministic=True))
    steps = []
    for i in range(5):
        sc, tgt = _inputs(50 + i, P)
        steps.append({k: torch.from_numpy(np.ascontiguousarray(sc[k])).pin_memory()
                      for k in ("points", "normals", "albedo")} | {"target": torch.from_numpy(tgt).pin_memory()})
    pipe = HostStepPipeline(scene, P, want=WANT, depth=depth, device=dev)
    got = []
    for i, st in enumerate(steps):
        pipe.submit(st["points"], st["normals"], st["albedo"], st["target"])
        if i >= depth - 1:
            got.append({k: v.clone() for k, v in pipe.result(i - depth + 1).items()})
    for i in range(len(steps) - depth + 1, len(steps)):
        got.append({k: v.clone() for k, v in pipe.result(i).items()})
    pipe.synchronize()
    assert pipe.bytes_per_step() == (4 * P * 3 * 4, sum(v.numel() * 4 for v in got[0].values()))
    for i, st in enumerate(steps):
        d = {k: v.to(dev) for k, v in st.items()}
        sv = scene.new_saved(P, dev)
        B = scene.shade(d["points"], d["normals"], d["albedo"], saved=sv)
        ref = scene.backward_l2(d["points"], d["normals"], d["albedo"], B, d["target"], saved=sv, want=WANT)
        torch.cuda.synchronize()
        assert set(got[i]) == {"loss"} | {"d_" + w for w in WANT}
        for k, v in got[i].items():
            r = ref[k].cpu()
            assert torch.isfinite(v).all(), (i, k)
            assert torch.equal(v, r), (i, k, (v - r).abs().max().item())
    scene.close()


def test_pipeline_rejects_bad_inputs_and_stale_handles():
    import torch
    from paper_2104_00359_gb300 import Config, Scene
    from paper_2104_00359_gb300.pipeline import HostStepPipeline
    dev = torch.device("cuda:0")
    P = 257
    sc, tgt = _inputs(60, P)
    scene = Scene(*(torch.from_numpy(sc[k]).to(dev) for k in ("centers", "radii", "light")), Config(n_bands=4))
    pipe = HostStepPipeline(scene, P, depth=1, device=dev)
    h = {k: torch.from_numpy(np.ascontiguousarray(sc[k])) for k in ("points", "normals", "albedo")}
    t = torch.from_numpy(tgt)
    with pytest.raises(ValueError):
        pipe.submit(h["points"][:-1], h["normals"], h["albedo"], t)
    with pytest.raises(ValueError):
        pipe.submit(h["points"].double(), h["normals"], h["albedo"], t)
    a = pipe.submit(h["points"], h["normals"], h["albedo"], t)
    pipe.submit(h["points"], h["normals"], h["albedo"], t)
    with pytest.raises(ValueError):
        pipe.result(a)
    pipe.synchronize()
    scene.close()
