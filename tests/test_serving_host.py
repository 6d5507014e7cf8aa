"""Host-side admission logic of the server, with fake jobs (no GPU)."""

import pytest


def test_budget_queue_order(monkeypatch):
    torch = pytest.importorskip("torch")
    from paper_2104_00359_gb300 import serve
    from paper_2104_00359_gb300.shade import Config

    class FakeJob:
        def __init__(self, job_id, points, centers, config, target=None, **kw):
            self.job_id, self.P, self.N, self.config, self.target = job_id, len(points), len(centers), config, target
            self.busy = False

        def bytes(self):
            return serve.Job.device_bytes(self.P, self.N, self.config.n_bands, self.target is not None)

        def close(self):
            pass

    srv = serve.Server.__new__(serve.Server)
    srv.budget, srv.jobs, srv.used = 0.0, {}, 0
    srv.waiting_jobs = serve.deque()
    srv.device = "cpu"
    srv.chunk_points = serve.CHUNK_POINTS
    srv.batch_work = serve.BATCH_WORK
    monkeypatch.setattr(serve, "Job", type("J", (FakeJob,), {"device_bytes": staticmethod(serve.Job.device_bytes)}))
    monkeypatch.setattr(torch.cuda, "current_stream", lambda: type("S", (), {"synchronize": lambda self: None})())
    size = serve.Job.device_bytes(1000, 10, 4, False)
    srv.budget = 2.5 * size
    cfg = Config(n_bands=4)
    pts, ctr = [0] * 1000, [0] * 10
    assert srv.add_job("a", pts, [0], [0], ctr, [0], [0], cfg)
    assert srv.add_job("b", pts, [0], [0], ctr, [0], [0], cfg)
    assert not srv.add_job("c", pts, [0], [0], ctr, [0], [0], cfg)
    assert not srv.add_job("d", pts, [0], [0], ctr, [0], [0], cfg)   # FIFO: waits behind c
    assert list(srv.jobs) == ["a", "b"]
    srv.remove_job("a")
    assert list(srv.jobs) == ["b", "c"] and srv.used <= srv.budget
    srv.remove_job("b")
    assert list(srv.jobs) == ["c", "d"]
    with pytest.raises(ValueError):
        srv.add_job("huge", [0] * 10 ** 7, [0], [0], ctr, [0], [0], cfg)
