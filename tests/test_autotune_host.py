"""The autotuner's selection logic on the host, with the timed device run
replaced by a table: the fastest candidate wins, candidates the library
refuses or that need more keys than the budget are skipped, and results are
cached per (Gaussians, resolutions) signature."""
import types

import numpy as np
import pytest
import torch


@pytest.fixture(scope="module")
def at():
    from paper_2506_12727_gb300 import build
    build.build()
    from paper_2506_12727_gb300 import autotune, mvgs
    return autotune, mvgs


def _cams(res):
    return types.SimpleNamespace(width=np.array([w for w, _ in res]), height=np.array([h for _, h in res]))


def test_fastest_candidate_wins_and_refused_or_over_budget_ones_are_skipped(at, monkeypatch):
    autotune, mvgs = at
    table = {((16, 16), 0, 0): (5.0, 100), ((16, 64), 0, 0): (3.0, 90), ((32, 64), 0, 64): (2.0, 500),
             ((32, 32), 0, 0): None}

    def fake(scene_c, cams, tile, ppt, wb, grads, reps):
        r = table[(tile, ppt, wb)]
        if r is None:
            raise mvgs.MvgsError(mvgs.EINVAL, "refused")
        return r

    monkeypatch.setattr(autotune, "_time_config", fake)
    monkeypatch.setattr(autotune, "_cache", {})
    params = {"means": torch.zeros(4, 3)}
    scene = types.SimpleNamespace(n=4)
    tile, ppt, timings, wb = autotune.autotune(scene, _cams([(64, 48)]), params, candidates=tuple(table),
                                               key_budget=200)
    assert (tile, ppt, wb) == ((16, 64), 0, 0)  # (32, 64) is faster but over the key budget
    assert set(timings) == {"16x16/pptauto/batchauto", "16x64/pptauto/batchauto"}
    # cached per signature: a second call does not time again
    monkeypatch.setattr(autotune, "_time_config", lambda *a: (_ for _ in ()).throw(AssertionError("timed again")))
    assert autotune.autotune(scene, _cams([(64, 48)]), params, candidates=tuple(table), key_budget=200)[0] == (16, 64)


def test_no_candidate_runs(at, monkeypatch):
    autotune, mvgs = at

    def refuse(*a):
        raise mvgs.MvgsError(mvgs.ENOSPACE, "too big")

    monkeypatch.setattr(autotune, "_time_config", refuse)
    monkeypatch.setattr(autotune, "_cache", {})
    with pytest.raises(RuntimeError):
        autotune.autotune(types.SimpleNamespace(n=1), _cams([(8, 8)]), {"means": torch.zeros(1, 3)},
                          candidates=(((16, 16), 0, 0),))
