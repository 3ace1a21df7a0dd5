"""Serving loop: a resident scene, render requests of any view count and
resolution, continuous batching over several in-flight slots.

The paper trains; serving is the same forward pass (mvgs_render_views) put
behind a request queue.  The loop keeps the Gaussians resident on the device
and runs `slots` workers, each with its own CUDA stream and its own
state/workspace buffers:

  - a worker that becomes free takes every request that has arrived (oldest
    first) up to `max_views` views and `max_pixels` pixels, concatenates their
    cameras into one batch and renders it with one call, so requests of
    different view counts and resolutions share launches;
  - requests that arrive while other batches are on the GPU are taken by the
    next free worker: batches of different workers overlap on the device;
  - admission by memory: every worker may hold at most `memory_budget /
    slots` bytes of state and workspace.  A batch whose record and key counts
    (the library's cheap count passes report them before anything is
    allocated) need more is split in two, the second half going back to the
    front of the queue; a single request that does not fit alone is failed.

Each view is rendered with exactly the arithmetic it would get alone (the
batch only adds other views' keys to the sort), so a request's images do not
depend on what it was batched with.  A request completes when its batch's
stream has finished; its images stay on the device (`Request.images`, packed
per view like the library's images).
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import mvgs

_CAM_FIELDS = ("width", "height", "fx", "fy", "cx", "cy", "viewmat", "campos", "near")


class CameraBatch:
    """Cameras of several requests, concatenated (same fields as the camera
    sets the rasterizer takes: numpy arrays over views)."""

    def __init__(self, parts):
        for f in _CAM_FIELDS:
            setattr(self, f, np.concatenate([getattr(p, f) for p in parts], axis=0))

    @property
    def V(self) -> int:
        return int(self.width.shape[0])


@dataclass
class Request:
    rid: int
    cams: object                      # camera set of the request's views
    t_arrival: float = 0.0            # host clock (time.perf_counter), set on submit
    t_done: float | None = None
    images: torch.Tensor | None = None
    batch: int = -1                   # id of the batch that rendered it
    error: str | None = None
    done: threading.Event = field(default_factory=threading.Event)

    @property
    def views(self) -> int:
        return int(self.cams.width.shape[0])

    @property
    def pixels(self) -> int:
        return int(np.sum(self.cams.width.astype(np.int64) * self.cams.height.astype(np.int64)))

    @property
    def latency(self) -> float | None:
        return None if self.t_done is None else self.t_done - self.t_arrival


class Server:
    def __init__(self, params: dict, sh_degree: int, tile=(16, 16), bg=(0.0, 0.0, 0.0), slots=2, max_views=32,
                 max_pixels=48_000_000, memory_budget=64 << 30, pixels_per_thread=0, device="cuda"):
        self.params = {k: v.contiguous() for k, v in params.items()}
        self.scene_c = mvgs.make_scene(self.params, sh_degree)
        self.tile, self.bg, self.ppt, self.device = tuple(tile), tuple(bg), pixels_per_thread, device
        self.max_views, self.max_pixels = max_views, max_pixels
        self.slot_bytes = memory_budget // slots
        self.queue: collections.deque[Request] = collections.deque()
        self.cv = threading.Condition()
        self.closing = False
        self.batches = 0
        self.batch_log = []  # (batch id, views, pixels, requests, ms on the device)
        self.workers = [threading.Thread(target=self._worker, args=(i,), daemon=True) for i in range(slots)]
        self._dev_index = torch.device(device).index or 0
        for w in self.workers:
            w.start()

    # ---- client side ----
    def submit(self, req: Request) -> Request:
        req.t_arrival = time.perf_counter()
        with self.cv:
            self.queue.append(req)
            self.cv.notify()
        return req

    def close(self):
        with self.cv:
            self.closing = True
            self.cv.notify_all()
        for w in self.workers:
            w.join()

    # ---- workers ----
    def _take_batch(self):
        """Oldest requests first, up to the view and pixel limits (at least one)."""
        batch, views, pixels = [], 0, 0
        while self.queue:
            r = self.queue[0]
            if batch and (views + r.views > self.max_views or pixels + r.pixels > self.max_pixels):
                break
            batch.append(self.queue.popleft())
            views += r.views
            pixels += r.pixels
        return batch

    def _worker(self, index):
        torch.cuda.set_device(self._dev_index)
        stream = torch.cuda.Stream()
        rz = None
        while True:
            with self.cv:
                while not self.queue and not self.closing:
                    self.cv.wait()
                if not self.queue and self.closing:
                    return
                batch = self._take_batch()
                bid = self.batches
                self.batches += 1
            rz = self._render(batch, bid, stream, rz)

    def _render(self, batch, bid, stream, rz):
        cams = CameraBatch([r.cams for r in batch])
        with torch.cuda.stream(stream):
            if rz is None:
                rz = mvgs.Rasterizer(cams, tile=self.tile, bg=self.bg, device=self.device,
                                     pixels_per_thread=self.ppt, max_bytes=self.slot_bytes)
            else:
                rz.set_cameras(cams)
            try:
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                img = rz.forward(self.scene_c, stream=stream)
                ev1.record(stream)
                stream.synchronize()
            except mvgs.MemoryBudgetError as e:
                rz.state = rz.workspace = rz.layout = None
                torch.cuda.empty_cache()
                if len(batch) == 1:
                    r = batch[0]
                    r.error = str(e)
                    r.t_done = time.perf_counter()
                    r.done.set()
                    return rz
                # split: render the first half now, requeue the rest at the front
                half = len(batch) // 2
                with self.cv:
                    for r in reversed(batch[half:]):
                        self.queue.appendleft(r)
                    self.cv.notify()
                return self._render(batch[:half], bid, stream, rz)
        t = time.perf_counter()
        off = 0
        for r in batch:
            n = 3 * r.pixels
            r.images = img[off:off + n]
            off += n
            r.batch = bid
            r.t_done = t
            r.done.set()
        with self.cv:
            self.batch_log.append((bid, cams.V, int(np.sum(cams.width.astype(np.int64) * cams.height)), len(batch),
                                   ev0.elapsed_time(ev1)))
        return rz


def run_trace(server: Server, requests, arrivals_s, realtime=True):
    """Submits requests at their arrival times (seconds from now) and waits for
    all of them; returns the wall time of the whole trace in seconds."""
    t0 = time.perf_counter()
    for r, ta in zip(requests, arrivals_s):
        if realtime:
            dt = t0 + ta - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
        server.submit(r)
    for r in requests:
        r.done.wait()
    return time.perf_counter() - t0


def latency_summary(requests) -> dict:
    lat = np.array([r.latency for r in requests if r.error is None]) * 1e3
    views = sum(r.views for r in requests if r.error is None)
    return {"requests": len(requests), "failed": sum(r.error is not None for r in requests),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "views": int(views)}
