"""The serving scheduler's host logic on a machine without a GPU: batching
oldest-first within the limits, splitting a batch over the memory budget
(its tail requeued at the front), rendering a request too large for one call
a part of its views at a time, and failing only the request whose single
view cannot fit.  The device call is replaced by a stand-in that "renders"
every pixel of a view to the view's tag (its fx) and refuses batches over a
view limit the way the rasterizer refuses batches over its memory budget."""
import numpy as np
import pytest
import torch

import synth

NEVER_FITS = 666.0


@pytest.fixture(scope="module")
def serve_mod():
    from paper_2506_12727_gb300 import build
    build.build()
    from paper_2506_12727_gb300 import mvgs, serve
    return mvgs, serve


def _server(serve_mod, monkeypatch, limit, **kw):
    mvgs, serve = serve_mod
    # no device: the scene is never handed to the library here
    monkeypatch.setattr(serve.mvgs, "make_scene", lambda params, sh_degree: None)

    class FakeServer(serve.Server):
        def __init__(self, *a, **k):
            self.calls = []
            super().__init__(*a, **k)

        def _worker_stream(self):
            return None

        def _forward(self, cams, stream, rz):
            self.calls.append([float(f) for f in cams.fx])
            if cams.V > limit or np.any(cams.fx == NEVER_FITS):
                raise mvgs.MemoryBudgetError(cams.V, limit)
            parts = [torch.full((3 * int(w) * int(h),), float(f)) for w, h, f in zip(cams.width, cams.height, cams.fx)]
            return torch.cat(parts), 0.0, rz

    scene = synth.make_scene(8, 0)
    params = {k: torch.tensor(getattr(scene, k), dtype=torch.float32) for k in
              ("means", "log_scales", "quats", "opacity_logits", "sh")}
    return FakeServer(params, 0, device="cpu", **kw)


def _requests(serve, sizes, special=None):
    reqs, tag = [], 1.0
    for i, nv in enumerate(sizes):
        res = [(8 + 2 * ((tag + j) % 3), 4 + ((tag + j) % 2)) for j in range(nv)]
        cams = synth.make_cameras([(int(w), int(h)) for w, h in res], seed=i)
        cams.fx = np.arange(tag, tag + nv, dtype=np.float32)
        if special is not None and i == special:
            cams.fx[-1] = NEVER_FITS
        tag += nv
        reqs.append(serve.Request(rid=i, cams=cams))
    return reqs


def _expected(r):
    return torch.cat([torch.full((3 * int(w) * int(h),), float(f))
                      for w, h, f in zip(r.cams.width, r.cams.height, r.cams.fx)])


def test_batches_are_split_to_fit_and_every_request_gets_its_own_views(serve_mod, monkeypatch):
    mvgs, serve = serve_mod
    srv = _server(serve_mod, monkeypatch, limit=4, slots=1, max_views=8)
    reqs = _requests(serve, [1, 2, 3, 1, 2, 2, 1])
    # hold the worker until everything is queued, so the first batch is the
    # oldest requests up to 8 views
    with srv.cv:
        for r in reqs:
            r.t_arrival = 0.0
            srv.queue.append(r)
        srv.cv.notify()
    for r in reqs:
        assert r.done.wait(10), r.rid
    srv.close()
    for r in reqs:
        assert r.error is None, r.error
        assert torch.equal(r.images, _expected(r)), r.rid
    # every successful call stayed within the limit, and requests were never
    # reordered: the tags of the calls that succeeded, concatenated, are 1..12
    ok = [c for c in srv.calls if len(c) <= 4]
    assert [t for c in ok for t in c] == [float(t) for t in range(1, 13)]
    # the first call took requests 0-3 (7 views, under max_views 8) and was split
    assert srv.calls[0] == [1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 7.0]


def test_a_request_too_large_for_one_call_is_rendered_in_parts(serve_mod, monkeypatch):
    mvgs, serve = serve_mod
    srv = _server(serve_mod, monkeypatch, limit=2, slots=1)
    (r,) = _requests(serve, [7])
    srv.submit(r)
    assert r.done.wait(10)
    srv.close()
    assert r.error is None, r.error
    assert torch.equal(r.images, _expected(r))
    # halving until the parts fit: the calls that succeeded hold at most 2
    # views and cover the request's views once, in order
    ok = [c for c in srv.calls if len(c) <= 2]
    assert [t for c in ok for t in c] == [float(t) for t in range(1, 8)]
    assert srv.calls[0] == [float(t) for t in range(1, 8)]


def test_only_the_request_whose_view_cannot_fit_fails(serve_mod, monkeypatch):
    mvgs, serve = serve_mod
    srv = _server(serve_mod, monkeypatch, limit=8, slots=2)
    reqs = _requests(serve, [2, 3, 1], special=1)
    for r in reqs:
        srv.submit(r)
    for r in reqs:
        assert r.done.wait(10), r.rid
    srv.close()
    assert reqs[1].error is not None and "MemoryBudgetError" in reqs[1].error
    for r in (reqs[0], reqs[2]):
        assert r.error is None, r.error
        assert torch.equal(r.images, _expected(r))


def test_a_failure_after_a_split_fails_only_the_half_that_failed(serve_mod, monkeypatch):
    """A batch over the limit is split and its tail requeued; when the first
    half then fails, the requeued requests are rendered, not failed."""
    mvgs, serve = serve_mod
    srv = _server(serve_mod, monkeypatch, limit=2, slots=1, max_views=8)
    reqs = _requests(serve, [2, 2], special=0)  # request 0 holds a view that never fits
    with srv.cv:
        for r in reqs:
            r.t_arrival = 0.0
            srv.queue.append(r)
        srv.cv.notify()
    for r in reqs:
        assert r.done.wait(10), r.rid
    srv.close()
    assert reqs[0].error is not None and "MemoryBudgetError" in reqs[0].error
    assert reqs[1].error is None, reqs[1].error
    assert torch.equal(reqs[1].images, _expected(reqs[1]))


def test_coalescing_gathers_arrivals_into_one_batch(serve_mod, monkeypatch):
    """With a coalescing window a free worker waits for more views (up to the
    window) before taking a batch: three requests arriving 20 ms apart share
    one batch; a lone request goes once the window has passed."""
    import time
    mvgs, serve = serve_mod
    srv = _server(serve_mod, monkeypatch, limit=64, slots=1, coalesce_ms=2000.0, coalesce_views=6)
    reqs = _requests(serve, [2, 2, 2])
    for r in reqs:
        srv.submit(r)
        time.sleep(0.02)
    for r in reqs:
        assert r.done.wait(10), r.rid
    assert len(srv.batch_log) == 1 and srv.batch_log[0][3] == 3
    for r in reqs:
        assert torch.equal(r.images, _expected(r))
    srv.close()
    srv = _server(serve_mod, monkeypatch, limit=64, slots=1, coalesce_ms=50.0, coalesce_views=100)
    (r,) = _requests(serve, [1])
    t0 = time.perf_counter()
    srv.submit(r)
    assert r.done.wait(10)
    waited = time.perf_counter() - t0
    srv.close()
    assert r.error is None and 0.04 <= waited < 5.0
