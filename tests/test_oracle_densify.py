"""Pins of the densification oracle (oracle/densify.py)."""
import numpy as np

import oracle
from oracle import densify


def _params(n, rng):
    return dict(means=rng.normal(size=(n, 3)), log_scales=rng.normal(-3, 0.7, size=(n, 3)),
                quats=rng.normal(size=(n, 4)), opacity_logits=rng.normal(size=n),
                sh=rng.normal(size=(n, 16, 3)))


def test_rotation_matches_the_pinned_oracle_rotation():
    rng = np.random.default_rng(1)
    q = rng.normal(size=(50, 4))
    R = densify.quat_rotation(q)
    for i in range(50):
        np.testing.assert_allclose(R[i], oracle.quat_to_rotation(q[i])[0], atol=1e-12)


def test_hand_made_decisions():
    # columns: (max log-scale, logit, E1, E2, denom) -> expected (pruned, split, cloned, count)
    prune_logit, log_ext = densify.thresholds(0.05, 0.1)
    rows = [
        (np.log(0.5), -5.0, 10.0, 10.0, 1.0, (True, False, False, 0)),   # transparent: pruned
        (np.log(0.5), 1.0, 10.0, 0.0, 1.0, (False, True, False, 2)),     # large, E1 high: split
        (np.log(0.01), 1.0, 0.0, 10.0, 1.0, (False, False, True, 2)),    # small, E2 high: cloned
        (np.log(0.5), 1.0, 0.0, 10.0, 1.0, (False, False, False, 1)),    # large but only E2 high: kept
        (np.log(0.01), 1.0, 10.0, 0.0, 1.0, (False, False, False, 1)),   # small but only E1 high: kept
        (np.log(0.5), 1.0, 10.0, 10.0, 0.0, (False, False, False, 1)),   # never seen: kept
        (np.log(0.5), 1.0, 2.0, 0.0, 4.0, (False, True, False, 2)),      # mean E1 = 0.5 at the threshold
        (np.log(0.5), 1.0, 1.9, 0.0, 4.0, (False, False, False, 1)),     # just below
    ]
    ls = np.array([[r[0], r[0] - 1, r[0] - 2] for r in rows])
    d = densify.decide(ls, np.array([r[1] for r in rows]), np.array([r[2] for r in rows]),
                       np.array([r[3] for r in rows]), np.array([r[4] for r in rows]), 0.5, 0.5, prune_logit,
                       log_ext)
    for i, r in enumerate(rows):
        assert (d["pruned"][i], d["split"][i], d["cloned"][i], d["count"][i]) == r[5], i


def test_outputs_follow_the_decisions():
    rng = np.random.default_rng(2)
    n = 300
    p = _params(n, rng)
    e1, e2 = rng.exponential(1.0, n), rng.exponential(1.0, n)
    den = rng.integers(0, 5, n).astype(float)
    z = rng.normal(size=(n, 2, 3))
    pl, le = densify.thresholds(0.2, np.exp(-3.0))
    out, src, kind, d = densify.densify(p, e1, e2, den, z, 0.8, 0.8, pl, le)
    assert len(src) == d["count"].sum()
    assert np.all(np.diff(src) >= 0)  # ordered by source
    assert not np.isin(np.nonzero(d["pruned"])[0], src).any()
    for g in np.nonzero(d["cloned"])[0]:
        i = np.nonzero(src == g)[0]
        assert list(kind[i]) == [0, 1]
        for k in p:
            np.testing.assert_array_equal(out[k][i[0]], p[k][g])
            np.testing.assert_array_equal(out[k][i[1]], p[k][g])
    for g in np.nonzero(d["split"])[0]:
        i = np.nonzero(src == g)[0]
        assert list(kind[i]) == [2, 2]
        R = densify.quat_rotation(p["quats"][g:g + 1])[0]
        s = np.exp(p["log_scales"][g])
        for c, j in enumerate(i):
            # the child's offset, rotated back, is the scaled normal sample
            np.testing.assert_allclose(R.T @ (out["means"][j] - p["means"][g]), s * z[g, c], atol=1e-12)
            np.testing.assert_allclose(np.exp(out["log_scales"][j]), s / 1.6, rtol=1e-12)
            np.testing.assert_array_equal(out["sh"][j], p["sh"][g])


def test_split_children_sample_the_gaussian():
    # many children of one Gaussian: their offsets have covariance R S^2 R^T
    rng = np.random.default_rng(3)
    n = 40000
    p = dict(means=np.tile([0.3, -0.2, 0.1], (n, 1)), log_scales=np.tile(np.log([0.5, 0.2, 0.1]), (n, 1)),
             quats=np.tile([0.9, 0.2, -0.3, 0.1], (n, 1)), opacity_logits=np.ones(n), sh=np.zeros((n, 1, 3)))
    z = rng.normal(size=(n, 2, 3))
    out, src, kind, d = densify.densify(p, np.ones(n), np.zeros(n), np.ones(n), z, 0.5, 0.5,
                                        *densify.thresholds(0.01, 0.3))
    assert d["split"].all()
    off = out["means"] - p["means"][0]
    R = densify.quat_rotation(p["quats"][:1])[0]
    S = np.diag(np.exp(p["log_scales"][0]))
    cov = R @ S @ S @ R.T
    np.testing.assert_allclose(np.cov(off.T), cov, atol=4e-3)
