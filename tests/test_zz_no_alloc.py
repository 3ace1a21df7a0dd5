"""The loss entry point that allocates nothing (mvgs_dssim_loss_noalloc).

Callers that cannot allocate device memory (a plug-in inside another
framework's memory pool, a process that reserves all memory up front, a loop
that must never enter the allocator) call this variant: the library keeps the
loss's scratch in a static device array instead of a caller workspace.  Its
results must equal mvgs_dssim_loss's bit for bit on the same inputs (both run
the same deterministic kernels), with and without the gradient output, on
consecutive calls (the array keeps the previous call's contents), and calls
too large for the array must be refused without running.  With stage timing
on, its launches count as the D-SSIM stage.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _case(rng, shapes):
    imgs = [rng.uniform(size=(3, h, w)).astype(np.float32) for h, w in shapes]
    tgts = [np.clip(i + rng.normal(0, 0.15, size=i.shape), 0, 1).astype(np.float32) for i in imgs]
    return (torch.tensor(synth.pack_images(imgs), device="cuda"), torch.tensor(synth.pack_images(tgts), device="cuda"),
            np.array(shapes, np.int32))


def test_noalloc_matches_workspace_entry_point_on_consecutive_calls(cuda_lib):
    mvgs = cuda_lib
    rng = np.random.default_rng(61)
    for shapes in ([(832, 1264)], [(37, 52), (16, 16), (100, 7), (480, 640)]):
        img, tgt, hw = _case(rng, shapes)
        V = len(shapes)
        ref_loss = torch.empty(V, device="cuda")
        ref_grad = torch.empty_like(img)
        ws = torch.empty(mvgs.dssim_workspace_size(hw), dtype=torch.uint8, device="cuda")
        mvgs.dssim_loss(img, tgt, hw, 0.2, ref_loss, ref_grad, ws)
        ref_only = torch.empty(V, device="cuda")
        mvgs.dssim_loss(img, tgt, hw, 0.2, ref_only, None, ws)
        for _ in range(2):
            loss = torch.full((V,), float("nan"), device="cuda")
            grad = torch.full_like(img, float("nan"))
            mvgs.dssim_loss_noalloc(img, tgt, hw, 0.2, loss, grad)
            only = torch.full((V,), float("nan"), device="cuda")
            mvgs.dssim_loss_noalloc(img, tgt, hw, 0.2, only, None)  # the loss alone
            torch.cuda.synchronize()
            # the same deterministic kernels (no atomics) on the same inputs:
            # equal bit for bit, whichever scratch they use
            assert torch.equal(loss, ref_loss)
            assert torch.equal(grad, ref_grad)
            assert torch.equal(only, ref_only)


def test_noalloc_refuses_calls_larger_than_its_buffer(cuda_lib):
    mvgs = cuda_lib
    hw = np.array([[1080, 1920], [832, 1264]], np.int32)  # about 3.1 million pixels
    img = torch.zeros(3 * int((hw[:, 0] * hw[:, 1]).sum()), device="cuda")
    loss = torch.zeros(2, device="cuda")
    with pytest.raises(mvgs.MvgsError) as e:
        mvgs.dssim_loss_noalloc(img, img, hw, 0.2, loss, None)
    assert e.value.status == mvgs.ENOSPACE
    assert "static buffer" in mvgs.last_error()


def test_noalloc_is_timed_as_the_dssim_stage(cuda_lib):
    mvgs = cuda_lib
    img, tgt, hw = _case(np.random.default_rng(62), [(64, 96)])
    loss = torch.empty(1, device="cuda")
    mvgs.profile_read()
    mvgs.profile_enable(True)
    try:
        for _ in range(3):
            mvgs.dssim_loss_noalloc(img, tgt, hw, 0.2, loss, None)
        torch.cuda.synchronize()
    finally:
        mvgs.profile_enable(False)
    ms, calls = mvgs.profile_read()["dssim"]
    assert calls == 3 and ms > 0
