"""Autotuner: times the launch candidates on the workload, returns the
fastest, and serves the cached choice on the next call."""
import json

import pytest

import gs_synthetic as S
from _util import device_gaussians


@pytest.mark.gpu
def test_tune_picks_and_caches(tmp_path):
    from paper_2501_06838_gb300.tune import tune
    gsets, views = S.config3(n_images=4)
    dgs = [device_gaussians(g) for g in gsets]
    cache = str(tmp_path / "tune.json")
    cands = ((16, 32), (8, 32), (32, 64))
    e1 = tune(dgs, views, with_grads=True, candidates=cands, reps=3, cache=cache)
    assert (e1["tile"], e1["batch"]) in cands
    assert e1["ms"] == min(e1["table"].values())
    with open(cache) as f:
        assert len(json.load(f)) == 1
    e2 = tune(dgs, views, with_grads=True, candidates=cands, reps=3, cache=cache)
    assert e2 == e1
