"""Autotuner (gs_tune): times the launch candidates on the workload, returns
the fastest, and serves the cached choice on the next call; the choice renders
the same image."""
import pytest

import gs_synthetic as S
from _util import device_gaussians


@pytest.mark.gpu
def test_tune_picks_and_caches(tmp_path):
    import torch
    import paper_2501_06838_gb300 as gs
    from paper_2501_06838_gb300.tune import tune
    gsets, views = S.config3(n_images=4)
    dgs = [device_gaussians(g) for g in gsets]
    cache = str(tmp_path / "tune.jsonl")
    e1 = tune(dgs, views, with_grads=True, reps=3, cache=cache)
    assert e1["tile"] in (8, 16, 32) and e1["binning"] in ("sort", "grid")
    # 6 launch shapes x 2 binnings and 2 pair-of-tiles layouts with the tile
    # adjoint, the 6 at tile 16 also with the quadrant adjoint, then the
    # fastest of those with the Gaussian-warp adjoint
    assert e1["raster"] in (1, 2) and e1["adjoint"] in (1, 2, 3)
    assert not e1["from_cache"] and e1["ms"] > 0 and e1["n_timed"] == 21
    assert e1["adjoint"] != 3 or e1["tile"] == 16
    import json
    with open(cache) as f:
        lines = f.read().splitlines()
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert (rec["tile"], rec["batch"]) == (e1["tile"], e1["batch"]) and rec["ms"] > 0
    assert rec["signature"].count("|") >= 5
    e2 = tune(dgs, views, with_grads=True, reps=3, cache=cache)
    assert e2["from_cache"] and (e2["tile"], e2["batch"], e2["binning"], e2["raster"],
                                 e2["adjoint"]) == \
        (e1["tile"], e1["batch"], e1["binning"], e1["raster"], e1["adjoint"])
    # the tuned launch renders the same image as the default one
    for v in views:
        v.binning, v.raster = e1["binning_code"], e1["raster"]
    out_t, _ = gs.render_batched(dgs, views, tile=e1["tile"], batch=e1["batch"], check=True)
    for v in views:
        v.binning, v.raster = 0, 0
    out_d, _ = gs.render_batched(dgs, views, check=True)
    for a, b in zip(out_t, out_d):
        assert torch.allclose(a, b, rtol=1e-5, atol=1e-6 * float(b.abs().max()))


@pytest.mark.gpu
def test_tune_rejects_bad_reps(tmp_path):
    from paper_2501_06838_gb300 import _abi
    from paper_2501_06838_gb300.tune import tune
    gsets, views = S.config1()
    with pytest.raises(_abi.GsError):
        tune([device_gaussians(gsets[0])], views, with_grads=False, reps=0,
             cache=str(tmp_path / "t.txt"))
