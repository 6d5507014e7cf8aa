"""Continuous-batching server for many concurrent analysis-by-synthesis jobs.

Each job keeps its state resident on the device: its scene (spheres + SH
lighting, Sec. 3.3), its G-buffer (points, normals, albedo), the target image
of its L2 loss (Sec. 3.5, Eq. 15) and its output buffers.  Jobs are admitted
only while their device bytes fit the HBM budget; the rest wait and are
admitted as memory frees up.  Requests ("fwd": shade; "fwdbwd": shade + L2 loss
+ adjoint) queue per arrival; whenever one of the batch slots is free, the
server packs up to ``max_batch`` ready requests of distinct jobs into one
``shs_shade_batch`` call (one persistent launch per band count and pass) on
that slot's stream.  Batches in different slots overlap on the device, and
requests that arrive while batches run join the next free slot -- continuous
batching, not a queue in front of one call at a time.

A large job can be split into chunks of at most ``chunk_points`` points, each with
its own resident scene (the same spheres and lighting), saved state and
scene-gradient buffers; its request becomes one task per chunk, and a batch
takes at most one task of a request.  So no launch carries more than a chunk
of any request, and a small request waits behind at most a chunk of a large
one instead of its whole service time (the persistent batch kernels hold
every SM until their work list drains).  The chunks' scene gradients and
losses are summed when the request's last chunk completes.

Short tasks may go first: with ``small_work`` > 0, a batch is filled with the
pending tasks of estimated work at most ``small_work`` (in arrival order)
before the others (in arrival order).  Every batch still takes the oldest
eligible task when nothing else fits, and the work cap leaves room for the
long tasks, so they are delayed, not starved.

The per-call baseline (``PerCallRunner``) serves the same stream of requests
one at a time with ``shs_shade`` / ``shs_shade_backward_l2`` on one stream.
"""

from __future__ import annotations

import ctypes
import time
from collections import deque
from dataclasses import dataclass, field

import torch

from . import _lib
from ._lib import ShsRequest, check, ptr
from .shade import Config, Scene


def _load():
    return _lib.load()


MAX_BATCH = 32
# Chunking is off by default: measured on the serving mix it lengthened the
# tails (the host loop handles many more, smaller batches); a cap on a
# batch's work bounds the wait for SMs instead.
CHUNK_POINTS = 1 << 40
# Estimated work a batch may carry (task_work units; about 3 ms on a GB300):
# the persistent batch kernels hold every SM until their work list drains,
# so this bounds how long a newly arrived request waits for SMs.
BATCH_WORK = 3.0e8
# Tasks up to this estimated work (about a 100k-point forward with 250
# spheres at 4 bands) are taken first when a batch is filled (0: arrival
# order only); measured on the serving mix it cuts the p99 of requests under
# 100k points by a quarter at an unchanged overall p99.
SMALL_WORK = 1.0e8


def task_work(points, spheres, n_bands, op):
    """Work estimate of one task: point-sphere pairs weighted by the band
    count's cost per pair (relative to 4 bands), the adjoint counted as
    forward + 2.5 x forward."""
    per_pair = (n_bands * n_bands + 4.0) / 20.0
    return points * max(spheres, 1) * per_pair * (3.5 if op == "fwdbwd" else 1.0)


class Job:
    """A job's resident device state (and, for a job of more than
    ``chunk_points`` points, that of its chunks)."""

    def __init__(self, job_id, points, normals, albedo, centers, radii, light, config: Config, target=None,
                 device="cuda", chunk_points=CHUNK_POINTS):
        self.job_id = job_id
        self.config = config
        dev = torch.device(device)
        f32 = lambda t: torch.as_tensor(t, dtype=torch.float32).to(dev).contiguous()
        self.points, self.normals, self.albedo = f32(points), f32(normals), f32(albedo)
        self.centers, self.radii, self.light = f32(centers), f32(radii), f32(light)
        self.target = f32(target) if target is not None else None
        self.P = int(self.points.shape[0])
        self.N = int(self.centers.shape[0])
        self.scene = Scene(self.centers if self.N else None, self.radii if self.N else None, self.light, config)
        self.saved = self.scene.new_saved(self.P, dev)
        self.radiance = torch.empty((self.P, 3), dtype=torch.float32, device=dev)
        self.grads = self.scene._grad_buffers(self.P, dev, ("light", "albedo", "centers", "radii"))
        self.loss = torch.zeros((), dtype=torch.float32, device=dev)
        self.busy = False
        self.active = None           # the request the job serves now
        # chunks: [p0, p1) point ranges; a chunked job gets per-chunk scenes,
        # saved state and scene-gradient buffers
        nch = max(1, -(-self.P // int(chunk_points)))
        bounds = [round(i * self.P / nch) for i in range(nch + 1)]
        self.ranges = [(bounds[i], bounds[i + 1]) for i in range(nch)]
        self.chunks = []
        if nch > 1:
            K = config.n_bands ** 2
            for p0, p1 in self.ranges:
                sc = Scene(self.centers if self.N else None, self.radii if self.N else None, self.light, config)
                z = lambda *sh: torch.zeros(sh, dtype=torch.float32, device=dev)
                self.chunks.append(dict(scene=sc, saved=sc.new_saved(p1 - p0, dev), d_light=z(3, K),
                                        d_centers=z(max(self.N, 1), 3), d_radii=z(max(self.N, 1)), loss=z()))

    @staticmethod
    def device_bytes(P, N, n_bands, with_target=True, chunk_points=CHUNK_POINTS):
        """Bytes a job holds on the device (inputs, outputs, saved state,
        scene, and for a chunked job the chunks' scenes and saved state)."""
        K = n_bands * n_bands
        per_point = 4 * (9 + 3 + (3 if with_target else 0) + 3 + K + 1)
        scene = 16 * N + 4 * (3 * K + 4) + 4 * 2 * (3 * K + 1 + 4 * N) + 4 * (3 * K + 4 * N)
        nch = max(1, -(-P // int(chunk_points)))
        chunked = 0 if nch == 1 else P * 4 * (K + 1) + nch * (scene + 4 * (3 * K + 4 * N + 1) + 4096)
        return P * per_point + scene + chunked + 4096

    def bytes(self):
        return self.device_bytes(self.P, self.N, self.config.n_bands, self.target is not None,
                                 self.ranges[0][1] if len(self.ranges) > 1 else CHUNK_POINTS)

    def request_struct(self, op, chunk=0):
        """The shs_request of chunk `chunk` (the whole job when unchunked)."""
        r = ShsRequest()
        p0, p1 = self.ranges[chunk]
        c = self.chunks[chunk] if self.chunks else None
        r.scene = (c["scene"] if c else self.scene).handle.value
        r.n_points = p1 - p0
        r.points, r.normals, r.albedo = (t[p0:p1].data_ptr() for t in (self.points, self.normals, self.albedo))
        r.radiance = self.radiance[p0:p1].data_ptr()
        r.saved = (c["saved"] if c else self.saved).data_ptr()
        if op == "fwdbwd":
            r.target = self.target[p0:p1].data_ptr()
            r.loss = (c["loss"] if c else self.loss).data_ptr()
            r.d_albedo = self.grads["d_albedo"][p0:p1].data_ptr()
            for k in ("d_light", "d_centers", "d_radii"):
                v = self.grads[k]
                if v is None:
                    continue
                setattr(r, k, (c[k] if c else v).data_ptr())
        return r

    def finish(self, op):
        """After the last chunk of a request: the chunks' scene sums."""
        if op != "fwdbwd" or not self.chunks:
            return
        self.loss.copy_(torch.stack([c["loss"] for c in self.chunks]).sum(0))
        self.grads["d_light"].copy_(torch.stack([c["d_light"] for c in self.chunks]).sum(0))
        if self.N:
            self.grads["d_centers"].copy_(torch.stack([c["d_centers"][:self.N] for c in self.chunks]).sum(0))
            self.grads["d_radii"].copy_(torch.stack([c["d_radii"][:self.N] for c in self.chunks]).sum(0))
        torch.cuda.current_stream().synchronize()

    def close(self):
        self.scene.close()
        for c in self.chunks:
            c["scene"].close()


@dataclass
class Request:
    req_id: int
    job_id: object
    op: str                      # "fwd" or "fwdbwd"
    arrival: float               # host time (perf_counter) the request became available
    launched: float = 0.0
    done: float = 0.0
    batch: int = -1
    pairs: int = 0
    on_done: object = None
    left: int = 0                # chunk tasks not yet completed
    expand: int = 0              # chunk tasks still to queue once its first chunk is batched

    @property
    def latency(self):
        return self.done - self.arrival


@dataclass
class _Slot:
    stream: torch.cuda.Stream
    ctx: ctypes.c_void_p
    event: torch.cuda.Event = None
    requests: list = field(default_factory=list)


class Server:
    """Continuous-batching request loop (see module docstring)."""

    def __init__(self, hbm_budget_bytes=80e9, n_slots=3, max_batch=MAX_BATCH, device="cuda",
                 chunk_points=CHUNK_POINTS, batch_work=BATCH_WORK, small_work=SMALL_WORK):
        if not 1 <= max_batch <= MAX_BATCH:
            raise ValueError(f"max_batch must be in 1..{MAX_BATCH}")
        if chunk_points < 128:
            raise ValueError("chunk_points must be at least one 128-point tile")
        self.lib = _load()
        self.device = device
        self.chunk_points = int(chunk_points)
        self.batch_work = float(batch_work)
        self.small_work = float(small_work)
        self.budget = float(hbm_budget_bytes)
        self.max_batch = max_batch
        self.jobs = {}
        self.waiting_jobs = deque()       # (job_id, kwargs) not yet admitted
        self.used = 0
        self.pending = deque()            # requests not yet launched
        self.completed = []
        self.batches = 0
        self.max_inflight = 0
        self._req_ids = 0
        self.slots = []
        for _ in range(n_slots):
            h = ctypes.c_void_p()
            check(self.lib.shs_batch_create(ctypes.byref(h)), "shs_batch_create")
            self.slots.append(_Slot(torch.cuda.Stream(device=device), h))

    # -- jobs ------------------------------------------------------------
    def add_job(self, job_id, points, normals, albedo, centers, radii, light, config: Config, target=None):
        """Admit the job if its device bytes fit the budget, else queue it.
        Returns True when admitted now."""
        kw = dict(points=points, normals=normals, albedo=albedo, centers=centers, radii=radii, light=light,
                  config=config, target=target)
        need = Job.device_bytes(len(points), len(centers), config.n_bands, target is not None, self.chunk_points)
        if need > self.budget:
            raise ValueError(f"job {job_id} needs {need} bytes, more than the whole budget")
        if self.used + need <= self.budget and not self.waiting_jobs:
            self._admit(job_id, kw)
            return True
        self.waiting_jobs.append((job_id, kw))
        return False

    def _admit(self, job_id, kw):
        job = Job(job_id, device=self.device, chunk_points=self.chunk_points, **kw)
        # the job's uploads and scene set-up ran on the current stream; the
        # batch slots use their own streams
        torch.cuda.current_stream().synchronize()
        self.jobs[job_id] = job
        self.used += job.bytes()

    def remove_job(self, job_id):
        job = self.jobs.pop(job_id)
        if job.busy:
            raise RuntimeError("job has a request in flight")
        self.used -= job.bytes()
        job.close()
        self._admit_waiting()

    def _admit_waiting(self):
        while self.waiting_jobs:
            job_id, kw = self.waiting_jobs[0]
            need = Job.device_bytes(len(kw["points"]), len(kw["centers"]), kw["config"].n_bands,
                                    kw["target"] is not None, self.chunk_points)
            if self.used + need > self.budget:
                break
            self.waiting_jobs.popleft()
            self._admit(job_id, kw)

    def admitted(self, job_id):
        return job_id in self.jobs

    # -- requests ----------------------------------------------------------
    def submit(self, job_id, op="fwd", arrival=None, on_done=None):
        if op not in ("fwd", "fwdbwd"):
            raise ValueError("op must be 'fwd' or 'fwdbwd'")
        r = Request(self._req_ids, job_id, op, time.perf_counter() if arrival is None else arrival,
                    on_done=on_done)
        self._req_ids += 1
        # one task per chunk of the job (its chunk count is known once admitted)
        self.pending.append((r, None))
        return r

    def _retire(self, slot):
        for r, chunk in slot.requests:
            r.left -= 1
            if r.left:
                continue
            job = self.jobs[r.job_id]
            job.finish(r.op)
            r.done = time.perf_counter()
            job.busy = False
            job.active = None
            if r.on_done is not None:
                r.on_done(r, job)
            self.completed.append(r)
        slot.requests = []
        slot.event = None

    def poll(self):
        """Retire finished batches, then launch ready requests into free
        slots.  Returns the number of requests launched."""
        for slot in self.slots:
            if slot.event is not None and slot.event.query():
                self._retire(slot)
        launched = 0
        for slot in self.slots:
            if slot.event is not None:
                continue
            batch, work = [], 0.0
            taken = set()
            for pos in self._fill_order():
                if len(batch) >= self.max_batch:
                    break
                r, chunk = self.pending[pos]
                job = self.jobs.get(r.job_id)
                # a job serves one request at a time; a batch takes one task of a request
                if job is None or (job.busy and job.active is not r) or any(b[0] is r for b in batch):
                    continue
                w = self._work(r, chunk)
                if batch and work + w > self.batch_work:
                    continue
                work += w
                taken.add(pos)
                if chunk is None:
                    # first task of the request: expand it into its chunks
                    if r.op == "fwdbwd" and job.target is None:
                        raise ValueError(f"job {r.job_id} has no target for a fwdbwd request")
                    r.left = len(job.ranges)
                    r.pairs = job.P * job.N
                    r.expand = len(job.ranges) - 1
                    chunk = 0
                    job.busy = True
                    job.active = r
                batch.append((r, chunk))
            # the rest stay in arrival order; a newly started chunked request
            # leaves its remaining chunks at the back
            keep = deque(t for i, t in enumerate(self.pending) if i not in taken)
            for r, _ in batch:
                if r.expand:
                    keep.extend((r, c) for c in range(1, r.expand + 1))
                    r.expand = 0
            self.pending = keep
            if not batch:
                break
            arr = (ShsRequest * len(batch))()
            now = time.perf_counter()
            for i, (r, chunk) in enumerate(batch):
                job = self.jobs[r.job_id]
                arr[i] = job.request_struct(r.op, chunk)
                if not r.launched:
                    r.launched = now
                r.batch = self.batches
            check(self.lib.shs_shade_batch(slot.ctx, arr, len(batch), ctypes.c_void_p(slot.stream.cuda_stream)),
                  "shs_shade_batch")
            slot.event = torch.cuda.Event()
            slot.event.record(slot.stream)
            slot.requests = batch
            self.batches += 1
            launched += len(batch)
        inflight = sum(1 for s in self.slots if s.event is not None)
        self.max_inflight = max(self.max_inflight, inflight)
        return launched

    def _work(self, r, chunk):
        job = self.jobs.get(r.job_id)
        if job is None:
            return 0.0
        c0 = 0 if chunk is None else chunk
        return task_work(job.ranges[c0][1] - job.ranges[c0][0], job.N, job.config.n_bands, r.op)

    def _fill_order(self):
        """Positions in `pending` in the order a batch considers them."""
        n = len(self.pending)
        if self.small_work <= 0.0:
            return range(n)
        small = [i for i, (r, c) in enumerate(self.pending) if self._work(r, c) <= self.small_work]
        ss = set(small)
        return small + [i for i in range(n) if i not in ss]

    def idle(self):
        return not self.pending and all(s.event is None for s in self.slots)

    def drain(self, timeout_s=600.0):
        t0 = time.perf_counter()
        while not self.idle():
            self.poll()
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError("server did not drain")

    def close(self):
        torch.cuda.synchronize()
        for slot in self.slots:
            self.lib.shs_batch_destroy(slot.ctx)
        for job in self.jobs.values():
            job.close()
        self.jobs.clear()


class PerCallRunner:
    """Baseline: each request as its own shs_shade (+ shs_shade_backward_l2)
    call, one at a time in arrival order, on one stream."""

    def __init__(self, server_jobs):
        self.jobs = server_jobs
        self.stream = torch.cuda.Stream()

    def run(self, req: Request):
        job = self.jobs[req.job_id]
        with torch.cuda.stream(self.stream):
            job.scene.shade(job.points, job.normals, job.albedo, saved=job.saved, out=job.radiance)
            if req.op == "fwdbwd":
                lib = job.scene.lib
                g = job.grads
                check(lib.shs_shade_backward_l2(job.scene.handle, job.P, ptr(job.points), ptr(job.normals),
                                                ptr(job.albedo), ptr(job.saved), ptr(job.radiance),
                                                ptr(job.target), ptr(job.loss), ptr(g["d_light"]),
                                                ptr(g["d_albedo"]), ptr(g["d_centers"]), ptr(g["d_radii"]),
                                                None, None, ctypes.c_void_p(self.stream.cuda_stream)),
                      "shs_shade_backward_l2")
        ev = torch.cuda.Event()
        ev.record(self.stream)
        return ev


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return float("nan")
    return xs[min(len(xs) - 1, int(round(q * (len(xs) - 1))))]
