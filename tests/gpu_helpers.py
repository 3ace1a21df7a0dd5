"""Shared helpers of the GPU parity tests: run the CUDA path through the C
ABI on seeded inputs and lay its per-record outputs out like the oracle's
dense (view, Gaussian) arrays."""
import numpy as np
import torch

PARAMS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def scene_to_device(scene, requires_grad=False):
    return {k: torch.tensor(getattr(scene, k), dtype=torch.float32, device="cuda").contiguous() for k in PARAMS}


def grads_like(params):
    return {k: torch.empty_like(v) for k, v in params.items()}


def gpu_forward(mvgs, scene, cams, tile=(16, 16), bg=(0.0, 0.0, 0.0), params=None):
    params = params if params is not None else scene_to_device(scene)
    sc = mvgs.make_scene(params, scene.sh_degree)
    rz = mvgs.Rasterizer(cams, tile=tile, bg=bg)
    img = rz.forward(sc)
    torch.cuda.synchronize()
    return rz, sc, params, img


def dense_records(rz, N, V):
    """GPU records scattered to dense [V*N] arrays (oracle layout)."""
    rec = {k: v.cpu().numpy() for k, v in rz.records().items()}
    idx = rec["v"].astype(np.int64) * N + rec["g"].astype(np.int64)
    R = V * N
    out = dict(valid=np.zeros(R, np.int32), xy=np.zeros((R, 2)), conic=np.zeros((R, 3)), opac=np.zeros(R),
               rgb=np.zeros((R, 3)), radius=np.zeros(R, np.int32), depth=np.zeros(R), rect=np.zeros((R, 4), np.int32),
               clamp=np.zeros(R, np.int32), rec_index=np.full(R, -1, np.int64))
    out["valid"][idx] = 1
    out["xy"][idx] = rec["xy"]
    out["conic"][idx] = rec["conic_o"][:, :3]
    out["opac"][idx] = rec["conic_o"][:, 3]
    out["rgb"][idx] = rec["rgb_r"][:, :3]
    out["radius"][idx] = rec["rgb_r"][:, 3].astype(np.int32)
    out["depth"][idx] = rec["depth"]
    out["rect"][idx] = rec["rect"]
    out["clamp"][idx] = rec["clamp"]
    out["rec_index"][idx] = np.arange(len(idx))
    out["raw"] = rec
    return out


def assert_close_frac(got, ref, rtol, atol, what, max_bad=0):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    err = np.abs(got - ref)
    bad = err > atol + rtol * np.abs(ref)
    nb = int(bad.sum())
    if nb > max_bad:
        i = np.unravel_index(np.argmax(err - (atol + rtol * np.abs(ref))), err.shape)
        raise AssertionError(f"{what}: {nb} of {err.size} entries outside tolerance (rtol={rtol}, atol={atol}); "
                             f"worst at {i}: got {got[i]!r} ref {ref[i]!r}")


def assert_close_rows(got, ref, rtol, atol, what, max_bad=0):
    """Like assert_close_frac, with the relative part taken against the norm of
    each Gaussian's gradient vector for the tensor (the row), not the single
    component: a component much smaller than its row's norm comes out of
    cancelling float32 terms of the row's size and is only that accurate."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    g2 = got.reshape(got.shape[0], -1)
    r2 = ref.reshape(ref.shape[0], -1)
    err = np.abs(g2 - r2)
    lim = atol + rtol * np.linalg.norm(r2, axis=1, keepdims=True)
    bad = err > lim
    nb = int(bad.sum())
    if nb > max_bad:
        i = np.unravel_index(np.argmax(err - lim), err.shape)
        raise AssertionError(f"{what}: {nb} of {err.size} entries outside tolerance (rtol={rtol} of the row norm, "
                             f"atol={atol}); worst at {i}: got {g2[i]!r} ref {r2[i]!r}")


# ---------------------------------------------------------------------------
# the oracle on large workloads: its C routines hold no global state and
# ctypes releases the GIL while they run, so independent views (projection,
# 3D gradients) and independent pixels (brute force) run on host threads
# ---------------------------------------------------------------------------
def _threads():
    import os
    return max(1, min(32, os.cpu_count() or 1))


def oracle_project(scene, cams, tile):
    """oracle.project, one view per host thread (same dense [V*N] layout)."""
    import concurrent.futures
    import oracle
    with concurrent.futures.ThreadPoolExecutor(min(_threads(), cams.V)) as ex:
        parts = list(ex.map(lambda v: oracle.project(scene, cams.subset([v]), tile), range(cams.V)))
    out = {k: np.concatenate([p[k] for p in parts]) for k in parts[0] if isinstance(parts[0][k], np.ndarray)}
    out["N"], out["V"], out["tile"] = scene.n, cams.V, tuple(tile)
    return out


def oracle_bruteforce(cams, P, pix, bg=(0.0, 0.0, 0.0)):
    """oracle.render_pixels_bruteforce over chunks of pixels on host threads."""
    import concurrent.futures
    import oracle
    chunks = np.array_split(np.asarray(pix), _threads())
    with concurrent.futures.ThreadPoolExecutor(len(chunks)) as ex:
        parts = list(ex.map(lambda c: oracle.render_pixels_bruteforce(cams, P, c, bg=bg), chunks))
    return tuple(np.concatenate([p[i] for p in parts]) for i in range(4))


def oracle_window_forward_backward(scene, cams, tile, win, dimg_fn, bg=(0.0, 0.0, 0.0)):
    """oracle.forward + oracle.backward restricted to a pixel window per view,
    with the projection and the 3D gradients (summed over views) computed
    one view per thread.  `dimg_fn(ref)` returns dL/dimage (packed) from the
    forward's outputs.  Returns (ref, dimg, grads, g2d)."""
    import concurrent.futures
    import oracle
    P = oracle_project(scene, cams, tile)
    S = oracle.sort_keys(cams, tile, P["valid"], P["rect"], P["depth"].astype(np.float32), win)
    img, T, last, amb, chash, depth = oracle.render(cams, P, S, bg, win, want_hash=True)
    ref = dict(P=P, S=S, img=img, T=T, last=last, amb=amb, chash=chash, depth=depth)
    dimg = dimg_fn(ref)
    g2d, e1 = oracle.render_backward(cams, P, S, dimg.astype(np.float64), bg, win)
    N = scene.n

    def one(v):
        return oracle.project_backward(scene, cams.subset([v]), tile, g2d[v * N:(v + 1) * N])
    with concurrent.futures.ThreadPoolExecutor(min(_threads(), cams.V)) as ex:
        parts = list(ex.map(one, range(cams.V)))
    grads = {k: sum(p[k] for p in parts) for k in parts[0]}
    return ref, dimg, grads, g2d
