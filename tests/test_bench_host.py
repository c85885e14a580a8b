"""Host-side logic of the benchmark (no GPU): the workload views and their
command-line overrides, the CPU baseline's band sample (it must render with
the workload's own window and alignment), the algorithmic byte counts behind
the memory-bound passes' rates, the whole-pipeline FLOP count, and the
reference arm (the oracle timed on the host cores): its JSON line, alone and
under a two-rank launch."""
import argparse

import numpy as np
import pytest

import bench
import gs_synthetic as S
import oracle


def _args(**kw):
    d = dict(norm=None, align=None, ratio=None, adjoint=None, binning=None, raster=None)
    d.update(kw)
    return argparse.Namespace(**d)


def test_view_flags_override_and_keep_fields():
    _, views = S.ratio_ablation(8.0, 0.1)
    out = bench.apply_view_flags(views, _args())
    assert out[0] == views[0]
    out = bench.apply_view_flags(views, _args(norm="peak", align="half", binning="sort",
                                              adjoint="gaussian"))
    v = out[0]
    assert (v.norm, v.align, v.window) == (S.NORM_PEAK, S.ALIGN_HALF, S.WINDOW_RATIO)
    assert (v.binning, v.adjoint) == (1, 2)
    assert (v.lr_h, v.out_w, v.scale) == (views[0].lr_h, views[0].out_w, views[0].scale)
    _, v2 = S.config2()
    r = bench.apply_view_flags(v2, _args(ratio=0.25))[0]
    assert r.window == S.WINDOW_RATIO and abs(r.trunc_k - 0.25) < 1e-7


def test_band_sample_keeps_window_and_alignment():
    """The CPU baseline's band of rows is the workload's own render, cut."""
    g, v = S.ratio_ablation(8.0, 0.1)
    vh = bench.apply_view_flags(v, _args(align="half"))
    for views in (v, vh):
        outs, _, px = bench.oracle_step(g, views, False, band=4)
        u = views[0]
        top = oracle.render(g[0], S.View(u.lr_h, u.lr_w, 4, u.out_w, u.scale, u.trunc_k, u.norm,
                                         window=u.window, align=u.align))
        assert px == 4 * u.out_w
        assert np.array_equal(outs[0], top)


def test_binning_description():
    g, v = S.config2()
    assert bench.binning_desc(0, g, v) == "grid-implicit"
    assert bench.binning_desc(1, g, v) == "sorted pairs"
    wide = [S.View(2, 9000, 8, 36000, 4.0)]
    assert bench.binning_desc(0, g, wide) == "sorted pairs"


def test_hbm_stage_bytes():
    stats = {"n_gaussians": 1000, "tile_pairs": 5000}
    raw = {"preprocess": (0.002, 2), "preprocess_bwd": (0.001, 2),
           "emit": (0.001, 2), "radix_hist": (0.002, 4), "radix_scatter": (0.004, 4),
           "ranges": (0.001, 2), "raster_fwd": (1.0, 2)}
    grid = bench.hbm_stage_rates(raw, 2, stats, "f32", True)
    srt = bench.hbm_stage_rates(raw, 2, stats, "bf16", False)
    assert "raster_fwd" not in grid
    # parameters in, the record (and compact window) and the cleared moments out
    assert grid["preprocess"]["bytes_per_launch"] == 1000 * (36 + 64 + 32 + 8)
    assert srt["preprocess"]["bytes_per_launch"] == 1000 * (18 + 64 + 32)
    # parameters and moments in, gradients and the cleared moments out
    assert grid["preprocess_bwd"]["bytes_per_launch"] == 1000 * (36 + 32 + 36 + 32)
    assert srt["radix_scatter"]["bytes_per_launch"] == 16 * 5000
    assert srt["radix_hist"]["launches_per_step"] == 2
    # rate = bytes x launches / time
    e = grid["preprocess"]
    assert e["achieved_gbs"] == pytest.approx(140000 * 2 / 0.002e-3 / 1e9, rel=1e-3)


def test_pipeline_flops_scale_with_lr_area():
    from paper_2501_06838_gb300.gsasr import GSASRConfig
    cfg = GSASRConfig()
    f4, f2 = bench.pipeline_flops(cfg, 180, 180), bench.pipeline_flops(cfg, 360, 360)
    assert f2["encoder"] == pytest.approx(4 * f4["encoder"], rel=1e-9)
    # window counts and tokens scale with the area; nothing else depends on it
    assert f2["decoder"] == pytest.approx(4 * f4["decoder"], rel=1e-9)
    assert f4["decoder"] > 100 * f4["encoder"]
    # padding to whole windows: 90 -> 96 LR px
    f8 = bench.pipeline_flops(cfg, 90, 90)
    assert f8["decoder"] == pytest.approx(bench.pipeline_flops(cfg, 96, 96)["decoder"], rel=1e-12)


def _ref_line(out: str) -> dict:
    import json
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out
    return json.loads(lines[0])


def test_reference_arm_contract():
    """bench.py --impl reference times the FP64 oracle on the host cores and
    prints one JSON line with the contract's keys (no GPU needed)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--ref-step-seconds", "0.3"], cwd=root,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = _ref_line(r.stdout)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e = d["e2e"]
    assert (e["value"], e["unit"], e["h2d_bytes_per_step"], e["d2h_bytes_per_step"]) == \
        (d["value"], d["unit"], 0, 0)
    assert d["config"]["workload"].startswith("c2")


def test_reference_arm_rank0_only():
    """Under torchrun with two ranks only rank 0 works and prints; both exit 0."""
    import os
    import socket
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1", "--master-port",
                        str(port), "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "3", "--ref-step-seconds", "0.3"], cwd=root,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = _ref_line(r.stdout)
    assert d["impl"] == "reference" and d["n_gpus"] == 2
