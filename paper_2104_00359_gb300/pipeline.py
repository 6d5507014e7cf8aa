"""Host-to-host analysis-by-synthesis steps, pipelined over three CUDA streams.

One step takes a batch of shading points (positions, normals, albedo) and a
target image from pinned host memory, shades them against a resident scene,
evaluates the L2 loss 1/2 |B - target|^2 and runs the adjoint (Sec. 3.5) in
the same launch, and brings the requested gradients and the loss back to
pinned host memory.

Uploads, compute and downloads run on separate streams, with ``depth`` sets of
device and host buffers, so step i+1's upload and step i-1's download overlap
step i's kernels.  Each buffer set is reused only after the device has
finished every use of it (events order the streams; nothing synchronises the
host except ``result``).
"""

from __future__ import annotations

import ctypes

import torch

from ._lib import check, ptr


class HostStepPipeline:
    """Pipelined forward + L2 adjoint steps of one ``Scene`` from host buffers.

    ``submit`` enqueues a step and returns a handle; ``result(handle)`` waits
    for that step's download and returns its host outputs (``loss`` and the
    ``d_*`` gradients named in ``want``).  The returned tensors are the
    set's pinned buffers: they stay valid until ``depth`` further submits.
    """

    WANT = ("light", "albedo", "centers", "radii")

    def __init__(self, scene, n_points, want=WANT, depth=2, device=None):
        if depth < 1:
            raise ValueError("depth must be >= 1")
        self.scene = scene
        self.lib = scene.lib
        self.P = int(n_points)
        self.want = tuple(want)
        self.depth = int(depth)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.h2d = torch.cuda.Stream(self.device)
        self.comp = torch.cuda.Stream(self.device)
        self.d2h = torch.cuda.Stream(self.device)
        P, dev = self.P, self.device
        self.sets = []
        for _ in range(self.depth):
            s = {
                "in": {k: torch.empty((P, 3), dtype=torch.float32, device=dev)
                       for k in ("points", "normals", "albedo", "target")},
                "radiance": torch.empty((P, 3), dtype=torch.float32, device=dev),
                "saved": scene.new_saved(P, dev),
                "loss": torch.empty((), dtype=torch.float32, device=dev),
                "grads": scene._grad_buffers(P, dev, self.want),
                "uploaded": torch.cuda.Event(),
                "computed": torch.cuda.Event(),
                "downloaded": torch.cuda.Event(),
                "handle": -1,
            }
            s["host"] = {k: torch.empty(v.shape, dtype=torch.float32).pin_memory()
                         for k, v in s["grads"].items() if v is not None}
            s["host"]["loss"] = torch.empty((), dtype=torch.float32).pin_memory()
            self.sets.append(s)
        # work the caller queued on its stream (scene set-up) comes first
        ready = torch.cuda.Event()
        ready.record(torch.cuda.current_stream(self.device))
        for st in (self.h2d, self.comp, self.d2h):
            st.wait_event(ready)
        self.n_submitted = 0

    def bytes_per_step(self):
        """(host-to-device, device-to-host) bytes one step copies."""
        s = self.sets[0]
        up = sum(t.numel() * 4 for t in s["in"].values())
        down = sum(t.numel() * 4 for t in s["host"].values())
        return up, down

    def submit(self, points, normals, albedo, target):
        """Enqueue one step.  Inputs are [P, 3] float32 CPU tensors; pinned
        ones are copied asynchronously (pageable ones make the copy wait)."""
        h = self.n_submitted
        s = self.sets[h % self.depth]
        src = {"points": points, "normals": normals, "albedo": albedo, "target": target}
        for k, t in src.items():
            if t.dtype != torch.float32 or t.device.type != "cpu" or tuple(t.shape) != (self.P, 3):
                raise ValueError(f"{k} must be a [{self.P}, 3] float32 CPU tensor")
        # the previous step of this set must have finished reading its inputs
        self.h2d.wait_event(s["computed"])
        with torch.cuda.stream(self.h2d):
            for k, t in src.items():
                s["in"][k].copy_(t.contiguous(), non_blocking=True)
        s["uploaded"].record(self.h2d)
        # ... and downloading its outputs before the kernels overwrite them
        self.comp.wait_event(s["uploaded"])
        self.comp.wait_event(s["downloaded"])
        g = s["grads"]
        sp = ctypes.c_void_p(self.comp.cuda_stream)
        i = s["in"]
        check(self.lib.shs_shade(self.scene.handle, self.P, ptr(i["points"]), ptr(i["normals"]),
                                 ptr(i["albedo"]), ptr(s["radiance"]), ptr(s["saved"]), sp), "shs_shade")
        check(self.lib.shs_shade_backward_l2(self.scene.handle, self.P, ptr(i["points"]), ptr(i["normals"]),
                                             ptr(i["albedo"]), ptr(s["saved"]), ptr(s["radiance"]),
                                             ptr(i["target"]), ptr(s["loss"]), ptr(g["d_light"]),
                                             ptr(g["d_albedo"]), ptr(g["d_centers"]), ptr(g["d_radii"]),
                                             ptr(g["d_points"]), ptr(g["d_normals"]), sp),
              "shs_shade_backward_l2")
        s["computed"].record(self.comp)
        self.d2h.wait_event(s["computed"])
        with torch.cuda.stream(self.d2h):
            for k, t in s["host"].items():
                t.copy_(s["loss"] if k == "loss" else g[k], non_blocking=True)
        s["downloaded"].record(self.d2h)
        s["handle"] = h
        self.n_submitted += 1
        return h

    def result(self, handle):
        """Wait for step ``handle`` and return its host outputs."""
        s = self.sets[handle % self.depth]
        if s["handle"] != handle:
            raise ValueError(f"step {handle} is no longer held (buffer set reused by step {s['handle']})")
        s["downloaded"].synchronize()
        return s["host"]

    def synchronize(self):
        """Wait for every submitted step (call before dropping the pipeline:
        its buffers are in use on the side streams until then)."""
        for st in (self.h2d, self.comp, self.d2h):
            st.synchronize()
