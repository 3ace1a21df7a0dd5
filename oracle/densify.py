"""Oracle of the multi-view densification step (Sec. 5.2.2 and the supplement's
"Experiment details") -- TEST INFRASTRUCTURE ONLY.

The paper keeps 3DGS's adaptive density control and changes its error
metric: Gaussians whose mean E_1 is above the split threshold are split,
those whose mean E_2 is above the clone threshold are cloned (E_1 is good at
splitting, E_2 at cloning), and the pruning threshold is multiplied by the
number of views per iteration.  It does not restate the 3DGS rules around
that; the readings taken (one pass, every Gaussian decided on its own):

  mean E_k  = accum_E_k / denom   (0 where denom = 0; float64 division)
  large     = max_i log_scale_i > log_dense_extent   (max scale > extent)
  pruned    = logit < prune_logit                     (opacity < threshold x views)
  split     = not pruned and large and mean E_1 >= split_threshold
  cloned    = not pruned and not large and mean E_2 >= clone_threshold
  outputs:  pruned -> none; split -> two children; cloned -> the Gaussian
            and a copy; otherwise the Gaussian.  Output order: by source
            index, a Gaussian's outputs in the order listed.
  child k of a split Gaussian (k = 0, 1): mean mu + R(q) (s * z_k) with z_k
            the caller's standard normal sample [n, 2, 3]; log-scale
            log_scale - ln(1.6); rotation, opacity and colour copied.
  kind of each output: 0 the Gaussian itself, 1 a clone's copy, 2 a split
            child (optimiser moments restart at zero for kinds 1 and 2).
The thresholds are taken in the parameters' own spaces (log-scale, logit), so
every decision is a float64 division and comparisons of float32 inputs, and
the CUDA side takes the same decisions bit for bit.
"""
from __future__ import annotations

import numpy as np

SPLIT_SCALE_DIV = 1.6


def quat_rotation(q):
    """Rotation matrices [n, 3, 3] of quaternions (w, x, y, z), normalised."""
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], 1)


def decide(log_scales, opacity_logits, accum_e1, accum_e2, denom, split_threshold, clone_threshold,
           prune_logit, log_dense_extent):
    """Per-Gaussian decisions (pruned, split, cloned) and the number of outputs."""
    denom = np.asarray(denom, np.float64)
    safe = np.where(denom > 0, denom, 1.0)
    m1 = np.where(denom > 0, np.asarray(accum_e1, np.float64) / safe, 0.0)
    m2 = np.where(denom > 0, np.asarray(accum_e2, np.float64) / safe, 0.0)
    large = np.asarray(log_scales, np.float64).max(1) > log_dense_extent
    opac = 1.0 / (1.0 + np.exp(-np.asarray(opacity_logits, np.float64)))
    pruned = np.asarray(opacity_logits, np.float64) < prune_logit
    split = ~pruned & large & (m1 >= split_threshold)
    cloned = ~pruned & ~large & (m2 >= clone_threshold)
    count = np.where(pruned, 0, np.where(split | cloned, 2, 1))
    return dict(pruned=pruned, split=split, cloned=cloned, count=count, mean_e1=m1, mean_e2=m2, large=large,
                opacity=opac)


def thresholds(prune_opacity, dense_extent):
    """(prune_logit, log_dense_extent) from an opacity and a world-space extent."""
    return float(np.log(prune_opacity / (1.0 - prune_opacity))), float(np.log(dense_extent))


def densify(params, accum_e1, accum_e2, denom, normals, split_threshold, clone_threshold, prune_logit,
            log_dense_extent):
    """Returns (new params dict, source index per output, kind per output, decisions)."""
    d = decide(params["log_scales"], params["opacity_logits"], accum_e1, accum_e2, denom, split_threshold,
               clone_threshold, prune_logit, log_dense_extent)
    src, kind, child = [], [], []
    for g in range(len(d["count"])):
        if d["pruned"][g]:
            continue
        if d["split"][g]:
            src += [g, g]
            kind += [2, 2]
            child += [0, 1]
        elif d["cloned"][g]:
            src += [g, g]
            kind += [0, 1]
            child += [-1, -1]
        else:
            src.append(g)
            kind.append(0)
            child.append(-1)
    src = np.array(src, np.int64)
    kind = np.array(kind, np.int32)
    child = np.array(child, np.int64)
    out = {k: np.asarray(v, np.float64)[src].copy() for k, v in params.items()}
    sp = kind == 2
    if sp.any():
        g = src[sp]
        R = quat_rotation(np.asarray(params["quats"], np.float64)[g])
        s = np.exp(np.asarray(params["log_scales"], np.float64)[g])
        z = np.asarray(normals, np.float64)[g, child[sp]]
        out["means"][sp] = np.asarray(params["means"], np.float64)[g] + np.einsum("nij,nj->ni", R, s * z)
        out["log_scales"][sp] = np.asarray(params["log_scales"], np.float64)[g] - np.log(SPLIT_SCALE_DIV)
    return out, src, kind, d
