"""Row bands of one image (`gs_view.row0`): the split of one large image over
several devices. Each band is rendered from all the Gaussians with the whole
image's windows and exponents, so the bands' rows are the image's rows (bit for
bit when a band starts on a tile row), and the image's adjoint is the sum of the
bands' adjoints: the adjoint is linear in the upstream gradient, and a band's
upstream gradient is the image's restricted to its rows.

CPU: the band partition, and the decomposition itself on the FP64 oracle with
two gloo ranks summing their bands' gradients. GPU: bands against the whole
image through the library (both binnings, both adjoints, windows and
alignments), bands as the entries of one batched call, and argument checks.
"""
import os
import socket

import numpy as np
import pytest

import gs_synthetic as S
import oracle
from _util import device_gaussians, normwise, view_with
from paper_2501_06838_gb300.shard import band_rows

FIELDS = ("o_x", "o_y", "sigma_x", "sigma_y", "rho", "r", "g", "b", "alpha")


def test_band_rows_partition():
    for out_h in (1, 15, 16, 17, 100, 1024, 1037):
        for parts in (1, 2, 3, 4, 7):
            for tile in (8, 16, 32):
                bands = band_rows(out_h, parts, tile)
                assert len(bands) == parts
                r = 0
                for r0, n in bands:
                    assert r0 == r and n >= 0
                    assert r0 % tile == 0 or n == 0
                    r += n
                assert r == out_h
                sizes = [n for _, n in bands]
                assert max(sizes) - min(sizes) <= tile * (1 + (out_h % tile != 0))
    with pytest.raises(ValueError):
        band_rows(10, 0)


def test_band_view():
    """band_view restricts a view to its rows and keeps every other field; an
    empty band (more ranks than tile rows) is refused, not sent to the library."""
    from paper_2501_06838_gb300.render import View
    from paper_2501_06838_gb300.shard import band_view
    v = View(48, 40, 192, 160, 4.0, trunc_k=0.1, norm=1, window=1, align=1)
    b = band_view(v, 64, 32)
    assert (b.row0, b.out_h) == (64, 32) and (v.row0, v.out_h) == (0, 192)
    assert (b.lr_h, b.lr_w, b.out_w, b.scale, b.trunc_k, b.norm, b.window, b.align) == \
        (48, 40, 160, 4.0, 0.1, 1, 1, 1)
    bands = band_rows(20, 4, 16)        # two tile rows over four ranks: two empty bands
    assert sum(1 for _, n in bands if n == 0) == 2
    for r0, n in bands:
        if n == 0:
            with pytest.raises(ValueError, match="empty band"):
                band_view(v, r0, n)


def _masked(go, r0, n):
    m = np.zeros_like(go)
    m[:, r0:r0 + n] = go[:, r0:r0 + n]
    return m


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _band_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2501_06838_gb300.shard import allreduce_band_grads, band_rows
        g = S.draw_gaussians(41, 12, 14, 1, (0.3, 2.0))
        v = S.View(12, 14, S.out_size(12, 3.5), S.out_size(14, 3.5), 3.5)
        go = S.grad_out(42, v.out_h, v.out_w)
        r0, n = band_rows(v.out_h, world, 16)[rank]
        # this rank's band gradient: the adjoint of the loss on its rows only
        part = torch.from_numpy(oracle.adjoint(g, v, _masked(go, r0, n)))
        allreduce_band_grads(part)
        q.put((rank, part.numpy()))
    finally:
        dist.destroy_process_group()


def test_two_rank_band_gradients_gloo():
    """Two ranks, one band each: the all-reduced band gradients equal the
    whole image's adjoint (FP64 oracle on both sides)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_band_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = S.draw_gaussians(41, 12, 14, 1, (0.3, 2.0))
    v = S.View(12, 14, S.out_size(12, 3.5), S.out_size(14, 3.5), 3.5)
    full = oracle.adjoint(g, v, S.grad_out(42, v.out_h, v.out_w))
    for r in (0, 1):
        assert np.all(normwise(res[r], full, axis=0) < 1e-12)


CASES = {
    "sigma": lambda: (S.draw_gaussians(43, 40, 52, 1, (0.3, 2.0)),
                      S.View(40, 52, S.out_size(40, 3.3), S.out_size(52, 3.3), 3.3)),
    "m4_ratio": lambda: (S.draw_gaussians(44, 20, 24, 4, (0.2, 3.0)),
                         S.View(20, 24, S.out_size(20, 5.5), S.out_size(24, 5.5), 5.5, trunc_k=0.1,
                                window=S.WINDOW_RATIO)),
    "half_pixel": lambda: (S.draw_gaussians(45, 30, 26, 1, (0.3, 2.0)),
                           S.View(30, 26, S.out_size(30, 2.6), S.out_size(26, 2.6), 2.6,
                                  align=S.ALIGN_HALF)),
}


def _render(g, v, go, binning=0, adjoint=0, row0=0, rows=None):
    import torch
    import paper_2501_06838_gb300 as gs
    vv = view_with(v)
    vv.binning, vv.adjoint, vv.row0 = binning, adjoint, row0
    if rows is not None:
        vv.out_h = rows
    dg = device_gaussians(g)
    out, ws = gs.render(dg, vv, check=True)
    gor = np.ascontiguousarray(go[:, row0:row0 + vv.out_h]).astype(np.float32)
    gr = gs.render_bwd(dg, vv, torch.from_numpy(gor).cuda(), ws, check=True)
    return out.cpu().numpy(), gr.cpu().double().numpy()


@pytest.mark.gpu
@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("binning,adjoint", [(1, 1), (2, 1), (2, 2), (1, 3), (2, 3)])
def test_bands_equal_whole_image(case, binning, adjoint):
    g, v = CASES[case]()
    go = S.grad_out(46, v.out_h, v.out_w)
    out, gr = _render(g, v, go, binning, adjoint)
    ref = oracle.render(g, v)
    assert np.all(normwise(out, ref, axis=(1, 2)) < 1e-5)
    parts, acc = [], np.zeros_like(gr)
    for r0, n in band_rows(v.out_h, 3, 16):
        ob, gb = _render(g, v, go, binning, adjoint, r0, n)
        parts.append(ob)
        acc += gb
    assert np.array_equal(np.concatenate(parts, axis=1), out)
    err = normwise(acc, gr, axis=0)
    assert np.all(err < 2e-6), dict(zip(FIELDS, err))


@pytest.mark.gpu
def test_band_off_tile_rows():
    """A band that does not start on a tile row: same rows up to float32
    rounding of the tile-local coordinates."""
    g, v = CASES["sigma"]()
    go = S.grad_out(47, v.out_h, v.out_w)
    out, gr = _render(g, v, go)
    r0, n = 37, 50
    ob, gb = _render(g, v, go, row0=r0, rows=n)
    assert np.all(normwise(ob, out[:, r0:r0 + n], axis=(1, 2)) < 1e-6)
    ref = oracle.adjoint(g, v, _masked(go, r0, n))
    err = normwise(gb, ref, axis=0)
    assert np.all(err < 1e-5), dict(zip(FIELDS, err))


@pytest.mark.gpu
def test_bands_in_one_batched_call():
    import paper_2501_06838_gb300 as gs
    g, v = CASES["sigma"]()
    dg = device_gaussians(g)
    whole, _ = gs.render(dg, view_with(v), check=True)
    views = []
    for r0, n in band_rows(v.out_h, 4, 16):
        vv = view_with(v)
        vv.row0, vv.out_h = r0, n
        views.append(vv)
    outs, _ = gs.render_batched([dg] * len(views), views, check=True)
    assert np.array_equal(np.concatenate([o.cpu().numpy() for o in outs], axis=1),
                          whole.cpu().numpy())


@pytest.mark.gpu
def test_band_arguments_checked():
    import paper_2501_06838_gb300 as gs
    from paper_2501_06838_gb300 import _abi
    g, v = CASES["sigma"]()
    dg = device_gaussians(g)
    vv = view_with(v)
    vv.row0 = -1
    with pytest.raises(_abi.GsError):
        gs.render(dg, vv, check=True)
    vv = view_with(v)
    vv.row0 = 10          # rows 10 .. 10 + out_h - 1 run past floor(s * lr_h) + 1
    with pytest.raises(_abi.GsError):
        gs.render(dg, vv, check=True)
