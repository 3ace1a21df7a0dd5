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
    allocated) need more -- or more keys than one call can index (2^32) -- is
    split in two, the second half going back to the front of the queue; a
    single request that does not fit is rendered a part of its views at a
    time, and fails only if one of its views does not fit alone;
  - a failure inside a batch fails that batch's requests (with the message)
    and the worker carries on;
  - optionally (`coalesce_ms` > 0) a free worker lets arrivals gather before
    it takes a batch: it waits until the queue holds `coalesce_views` views
    or its oldest request has waited `coalesce_ms`, so that at moderate load
    batches hold several requests instead of one (fewer, fuller launches, at
    the price of that wait in latency).

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
                 max_pixels=48_000_000, memory_budget=64 << 30, pixels_per_thread=0, device="cuda", coalesce_ms=0.0,
                 coalesce_views=0):
        self.params = {k: v.contiguous() for k, v in params.items()}
        self.scene_c = mvgs.make_scene(self.params, sh_degree)
        self.tile, self.bg, self.ppt, self.device = tuple(tile), tuple(bg), pixels_per_thread, device
        self.max_views, self.max_pixels = max_views, max_pixels
        self.slot_bytes = memory_budget // slots
        self.queue: collections.deque[Request] = collections.deque()
        self.cv = threading.Condition()
        self.closing = False
        self.coalesce_s, self.coalesce_views = coalesce_ms / 1e3, coalesce_views
        self.batches = 0
        # per batch: (batch id, views, pixels, requests, ms on the device, ms from
        # taking the batch to its completion on the host clock)
        self.batch_log = []
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

    def cancel_pending(self, reason="cancelled"):
        """Fails every request still waiting in the queue."""
        with self.cv:
            pending = list(self.queue)
            self.queue.clear()
        t = time.perf_counter()
        for r in pending:
            r.error = reason
            r.t_done = t
            r.done.set()
        return len(pending)

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

    def _worker_stream(self):
        """The worker's own CUDA stream, on the server's device."""
        torch.cuda.set_device(self._dev_index)
        return torch.cuda.Stream()

    def _worker(self, index):
        stream = self._worker_stream()
        rz = None
        while True:
            with self.cv:
                while True:
                    while not self.queue and not self.closing:
                        self.cv.wait()
                    if not self.queue and self.closing:
                        return
                    if self.coalesce_s > 0 and not self.closing:
                        age = time.perf_counter() - self.queue[0].t_arrival
                        if sum(r.views for r in self.queue) < self.coalesce_views and age < self.coalesce_s:
                            self.cv.wait(self.coalesce_s - age)
                            continue
                    break
                batch = self._take_batch()
                bid = self.batches
                self.batches += 1
            t_take = time.perf_counter()
            try:
                rz = self._render(batch, bid, stream, rz, t_take)
            except Exception as e:  # a failed batch fails its requests, not the server
                rz = None
                torch.cuda.empty_cache()
                t = time.perf_counter()
                for r in batch:
                    if not r.done.is_set():
                        r.error = f"{type(e).__name__}: {e}"
                        r.t_done = t
                        r.done.set()

    @staticmethod
    def _too_big(e):
        return isinstance(e, mvgs.MemoryBudgetError) or (isinstance(e, mvgs.MvgsError) and
                                                          e.status == mvgs.EOVERFLOW)

    def _forward(self, cams, stream, rz):
        """One library call for a camera batch; returns (images, ms, rz)."""
        with torch.cuda.stream(stream):
            if rz is None:
                rz = mvgs.Rasterizer(cams, tile=self.tile, bg=self.bg, device=self.device,
                                     pixels_per_thread=self.ppt, max_bytes=self.slot_bytes)
            else:
                rz.set_cameras(cams)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            try:
                img = rz.forward(self.scene_c, stream=stream)
            except Exception:
                rz.state = rz.workspace = rz.layout = None
                torch.cuda.empty_cache()
                raise
            ev1.record(stream)
            stream.synchronize()
        return img, ev0.elapsed_time(ev1), rz

    def _render_request_in_parts(self, r, stream, rz):
        """A request too large for one call: its views a part at a time."""
        parts, ms = [], 0.0
        todo = [list(range(r.views))]
        while todo:
            idx = todo.pop(0)
            sub = CameraBatch([_subset(r.cams, idx)])
            try:
                img, t, rz = self._forward(sub, stream, rz)
            except Exception as e:
                if not self._too_big(e) or len(idx) == 1:
                    raise
                half = len(idx) // 2
                todo[:0] = [idx[:half], idx[half:]]
                continue
            parts.append(img.clone())
            ms += t
        return torch.cat(parts), ms, rz

    def _render(self, batch, bid, stream, rz, t_take):
        cams = CameraBatch([r.cams for r in batch])
        try:
            img, ms, rz = self._forward(cams, stream, rz)
        except Exception as e:
            if not self._too_big(e):
                raise
            rz = None
            if len(batch) == 1:
                img, ms, rz = self._render_request_in_parts(batch[0], stream, rz)
            else:
                # split: render the first half now, requeue the rest at the front;
                # the batch list (the worker's) keeps only the first half, so a
                # failure from here on fails only the requests this worker holds
                half = len(batch) // 2
                with self.cv:
                    for r in reversed(batch[half:]):
                        self.queue.appendleft(r)
                    del batch[half:]
                    self.cv.notify()
                return self._render(batch, bid, stream, rz, t_take)
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
                                   ms, (t - t_take) * 1e3))
        return rz


def _subset(cams, idx):
    """The views `idx` of a camera set (same fields)."""
    out = CameraBatch([cams])
    for f in _CAM_FIELDS:
        setattr(out, f, getattr(out, f)[idx])
    return out


def run_trace(server: Server, requests, arrivals_s, realtime=True, timeout_s=None):
    """Submits requests at their arrival times (seconds from now) and waits for
    all of them, or until `timeout_s` after the start, when requests still
    queued are failed ("timeout") and those on the GPU are waited for; returns
    the wall time of the whole trace in seconds."""
    t0 = time.perf_counter()
    for r, ta in zip(requests, arrivals_s):
        if realtime:
            dt = t0 + ta - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
        server.submit(r)
    for r in requests:
        left = None if timeout_s is None else t0 + timeout_s - time.perf_counter()
        if left is not None and left <= 0:
            server.cancel_pending("timeout")
            left = None
        if not r.done.wait(left):
            server.cancel_pending("timeout")
            r.done.wait()
    return time.perf_counter() - t0


def latency_summary(requests) -> dict:
    ok = [r for r in requests if r.error is None]
    lat = np.array([r.latency for r in ok]) * 1e3
    views = sum(r.views for r in ok)
    return {"requests": len(requests), "completed": len(ok), "failed": len(requests) - len(ok),
            "p50_ms": float(np.percentile(lat, 50)) if len(ok) else None,
            "p99_ms": float(np.percentile(lat, 99)) if len(ok) else None,
            "mean_ms": float(lat.mean()) if len(ok) else None, "views": int(views)}
