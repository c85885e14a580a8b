"""Failure handling, all of it on the host or as status words: invalid
arguments are rejected before any launch; invalid parameter values and a pair
count above the workspace's capacity are flagged by the kernels in the
workspace status word and reported by gs_sync_status. Nothing here faults,
traps or waits on the device."""
import pytest

import gs_synthetic as S
from _util import device_gaussians


def test_missing_library_fails_loudly(tmp_path):
    """No CPU fallback: without the CUDA library the binding refuses to load."""
    with pytest.raises(RuntimeError, match="missing"):
        _load_fresh(str(tmp_path / "nope.so"))


def _load_fresh(path):
    from paper_2501_06838_gb300 import _abi
    saved = _abi._lib
    _abi._lib = None
    try:
        return _abi.load(path)
    finally:
        _abi._lib = saved


@pytest.mark.gpu
def test_invalid_arguments_rejected_on_host():
    import paper_2501_06838_gb300 as gs
    g, v = S.config1()[0][0], S.config1()[1][0]
    dg = device_gaussians(g)
    bad_views = [S.View(48, 48, 194, 192, 4.0),       # taller than floor(s * lr) + 1
                 S.View(48, 48, 192, 192, 0.0),       # scale 0
                 S.View(47, 48, 188, 192, 4.0)]       # n != m * lr_h * lr_w
    for bv in bad_views:
        with pytest.raises(gs.GsError) as ei:
            gs.render(dg, bv)
        assert ei.value.status == 1
    with pytest.raises(gs.GsError):
        gs.render(dg, v, tile=12)


@pytest.mark.gpu
@pytest.mark.parametrize("field,value", [("sigma", 0.0), ("sigma", -1.0), ("rho", 1.0),
                                         ("rho", -1.5), ("offset", float("nan")),
                                         ("alpha", float("inf"))])
def test_invalid_parameter_values_flagged(field, value):
    import torch
    import paper_2501_06838_gb300 as gs
    g = S.draw_gaussians(1, 16, 16, 1)
    dg = device_gaussians(g)
    v = S.View(16, 16, 48, 48, 3.0)
    cap = gs.count_pairs([dg], [v])
    t = getattr(dg, field)
    t.view(-1)[7] = value
    # the sizing pass reports it directly ...
    with pytest.raises(gs.GsError) as ei:
        gs.count_pairs([dg], [v])
    assert ei.value.status == 1
    # ... and the asynchronous render through the workspace status word
    ws = gs.Workspace(gs.workspace_bytes([dg], [v], cap))
    out, _ = gs.render(dg, v, ws=ws)
    with pytest.raises(gs.GsError) as ei:
        gs.sync_status(ws)
    assert ei.value.status == 1
    # the bad Gaussian contributes nothing; the others render
    assert torch.isfinite(out).all()
    gs.sync_status(ws)   # the status word was reset by the previous read


@pytest.mark.gpu
def test_capacity_overflow_flagged():
    import torch
    import paper_2501_06838_gb300 as gs
    g, v = S.config1()[0][0], S.config1()[1][0]
    v.binning = 1   # the sorted pair list: its capacity is what can overflow
    dg = device_gaussians(g)
    need = gs.count_pairs([dg], [v])
    ws = gs.Workspace(gs.workspace_bytes([dg], [v], need // 2))
    out, _ = gs.render(dg, v, ws=ws)
    with pytest.raises(gs.GsError) as ei:
        gs.sync_status(ws)
    assert ei.value.status == 2
    assert torch.all(out == 0)   # nothing binned, nothing drawn
    ws_ok = gs.Workspace(gs.workspace_bytes([dg], [v], need))
    out2, _ = gs.render(dg, v, ws=ws_ok, check=True)
    assert out2.abs().max() > 0
    # grid binning: the forward needs no pair list and still renders in full;
    # the per-tile lists it leaves for the adjoint do not fit, which is flagged
    v.binning = 2
    ws_grid = gs.Workspace(gs.workspace_bytes([dg], [v], need // 2))
    out3, _ = gs.render(dg, v, ws=ws_grid)
    with pytest.raises(gs.GsError) as ei:
        gs.sync_status(ws_grid)
    assert ei.value.status == 2
    assert torch.equal(out3, out2)
    ws_grid_ok = gs.Workspace(gs.workspace_bytes([dg], [v], need))
    out4, _ = gs.render(dg, v, ws=ws_grid_ok, check=True)
    assert torch.equal(out4, out2)


@pytest.mark.gpu
def test_workspace_too_small_rejected():
    import paper_2501_06838_gb300 as gs
    g, v = S.config1()[0][0], S.config1()[1][0]
    dg = device_gaussians(g)
    ws = gs.Workspace(1024)
    with pytest.raises(gs.GsError, match="too small"):
        gs.render(dg, v, ws=ws)
