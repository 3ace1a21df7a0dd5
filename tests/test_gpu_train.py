"""Densification step and Adam on the GPU.

  - mvgs_densify against oracle/densify.py: the decisions (hence the output
    count, sources and kinds) bit-exact -- both sides decide in float64 from
    the same float32 inputs -- and the new parameters within float32
    rounding (copies bit-exact);
  - mvgs_densify_carry copies kind-0 rows and zeros the rest;
  - mvgs_adam_step against torch.optim.Adam (float64, CPU) over several steps.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import PARAMS
from oracle import densify as odens

pytestmark = pytest.mark.gpu


def _setup(n, seed):
    rng = np.random.default_rng(seed)
    p = dict(means=rng.normal(size=(n, 3)), log_scales=rng.normal(-3, 0.8, size=(n, 3)),
             quats=rng.normal(size=(n, 4)), opacity_logits=rng.normal(0, 2, size=n), sh=rng.normal(size=(n, 16, 3)))
    p = {k: v.astype(np.float32) for k, v in p.items()}
    e1 = rng.exponential(1.0, n).astype(np.float32)
    e2 = rng.exponential(1.0, n).astype(np.float32)
    den = rng.integers(0, 6, n).astype(np.float32)
    z = rng.normal(size=(n, 2, 3)).astype(np.float32)
    return p, e1, e2, den, z


@pytest.mark.parametrize("n", [0, 1, 257, 50_000])
def test_densify_matches_oracle(cuda_lib, n):
    p, e1, e2, den, z = _setup(n, 5 + n)
    pl, le = odens.thresholds(0.1, float(np.exp(-2.5)))
    dev = {k: torch.tensor(v, device="cuda") for k, v in p.items()}
    t = lambda a: torch.tensor(a, device="cuda")
    m_adam = torch.randn(n, 16, 3, device="cuda")
    new, src, kind, (m_new,) = cuda_lib.densify(dev, 3, t(e1), t(e2), t(den), t(z), 0.4, 0.6, pl, le,
                                                carry=[m_adam])
    torch.cuda.synchronize()
    out, osrc, okind, d = odens.densify({k: v.astype(np.float64) for k, v in p.items()}, e1, e2, den, z, 0.4, 0.6,
                                        pl, le)
    if n >= 257:
        assert d["pruned"].any() and d["split"].any() and d["cloned"].any()
    np.testing.assert_array_equal(src.cpu().numpy(), osrc)
    np.testing.assert_array_equal(kind.cpu().numpy(), okind)
    for k in ("quats", "opacity_logits", "sh"):
        np.testing.assert_array_equal(new[k].cpu().numpy().astype(np.float64), out[k])
    np.testing.assert_allclose(new["means"].cpu().numpy(), out["means"], rtol=0, atol=2e-6)
    np.testing.assert_allclose(new["log_scales"].cpu().numpy(), out["log_scales"], rtol=0, atol=1e-6)
    keep = okind == 0
    mc = m_new.cpu().numpy()
    np.testing.assert_array_equal(mc[keep], m_adam.cpu().numpy()[osrc[keep]])
    assert (mc[~keep] == 0).all()


def test_densify_splits_everything_large(cuda_lib):
    p, e1, e2, den, z = _setup(1000, 9)
    dev = {k: torch.tensor(v, device="cuda") for k, v in p.items()}
    t = lambda a: torch.tensor(a, device="cuda")
    # everything large and above the split threshold: 2 outputs each
    dev["log_scales"].fill_(0.0)
    dev["opacity_logits"].fill_(3.0)
    new, src, kind, _ = cuda_lib.densify(dev, 3, t(np.ones(1000, np.float32)), t(e2), t(np.ones(1000, np.float32)),
                                         t(z), 0.5, 0.5, -10.0, -1.0)
    assert new["means"].shape[0] == 2000 and (kind == 2).all()


def test_adam_matches_torch(cuda_lib):
    rng = np.random.default_rng(4)
    x0 = rng.normal(size=10_001)
    grads = [rng.normal(size=x0.shape) * (10.0 ** rng.uniform(-3, 1)) for _ in range(6)]
    ref = torch.tensor(x0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([ref], lr=1e-2, betas=(0.9, 0.999), eps=1e-15)
    p = torch.tensor(x0, dtype=torch.float32, device="cuda")
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    for step, g in enumerate(grads, 1):
        ref.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        cuda_lib.adam_step(p, torch.tensor(g, dtype=torch.float32, device="cuda"), m, v, 1e-2, step, eps=1e-15)
    torch.cuda.synchronize()
    np.testing.assert_allclose(p.cpu().numpy(), ref.detach().numpy(), rtol=0, atol=2e-6)


@pytest.mark.parametrize("partial,cell", [(False, (1, 1)), (True, (1, 1)), (True, "strip")])
def test_training_loop_reduces_the_loss(cuda_lib, partial, cell):
    import synth
    from gpu_helpers import scene_to_device
    from paper_2506_12727_gb300.train import MultiViewTrainer
    gt = synth.make_scene(3000, 1, seed=31)
    cams = synth.make_cameras([(96, 72)] * 12, radius=3.5, seed=32)
    rz = cuda_lib.Rasterizer(cams, tile=(16, 16))
    img = rz.forward(cuda_lib.make_scene(scene_to_device(gt), 1)).clone()
    off = synth.view_offsets(cams)
    targets = [img[off[v]:off[v + 1]].reshape(3, 72, 96).clone() for v in range(cams.V)]
    rng = np.random.default_rng(33)
    init = scene_to_device(gt)
    init["means"] += torch.tensor(rng.normal(0, 0.02, size=(3000, 3)), dtype=torch.float32, device="cuda")
    init["sh"][:, 0] += torch.tensor(rng.normal(0, 0.3, size=(3000, 3)), dtype=torch.float32, device="cuda")
    init["opacity_logits"] -= 1.0
    tr = MultiViewTrainer(init, 1, cams, targets, views_per_iter=4, partial=partial, densify_every=30, cell=cell,
                          lr=dict(means=1e-3, sh=1e-2), clone_threshold=1e-3, split_threshold=1e-3,
                          prune_opacity=0.004, dense_extent=0.06, seed=1)
    losses = [tr.step() for _ in range(60)]
    print(f"partial={partial}: loss {np.mean(losses[:5]):.4f} -> {np.mean(losses[-5:]):.4f}, "
          f"Gaussians 3000 -> {tr.n}")
    assert np.all(np.isfinite(losses))
    assert np.mean(losses[-5:]) < 0.8 * np.mean(losses[:5])
    assert tr.n != 3000  # the densification step ran and changed the set
