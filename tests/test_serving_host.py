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


def test_fill_order_small_tasks_first():
    """With small_work set, a batch considers the pending tasks of estimated
    work <= small_work first (in arrival order), then the rest (in arrival
    order); with small_work = 0 it is arrival order alone."""
    pytest.importorskip("torch")
    from types import SimpleNamespace
    from paper_2104_00359_gb300 import serve

    def job(P, N, n):
        return SimpleNamespace(P=P, N=N, config=SimpleNamespace(n_bands=n), ranges=[(0, P)])

    srv = serve.Server.__new__(serve.Server)
    srv.jobs = {"big": job(1_000_000, 400, 6), "small": job(20_000, 50, 4), "mid": job(200_000, 100, 4)}
    reqs = [serve.Request(i, j, "fwd", 0.0) for i, j in enumerate(["big", "small", "mid", "small", "big"])]
    srv.pending = serve.deque((r, None) for r in reqs)
    srv.small_work = 0.0
    assert list(srv._fill_order()) == [0, 1, 2, 3, 4]
    srv.small_work = serve.task_work(100_000, 100, 4, "fwd")
    assert list(srv._fill_order()) == [1, 3, 0, 2, 4]
    assert serve.task_work(20_000, 50, 4, "fwdbwd") == 3.5 * serve.task_work(20_000, 50, 4, "fwd")
