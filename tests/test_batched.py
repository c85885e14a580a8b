"""Config 3: 16 images of uneven LR sizes (64..480 x 64..360, multiples of 4)
and non-integer scales in [1.5, 12], rendered in one chain of launches over a
global tile index space; the chain is also captured in a CUDA graph and
replayed. Forward against the FP64 oracle per image (1e-5 normwise per
channel); adjoint on a smaller uneven batch."""
import numpy as np
import pytest

import gs_synthetic as S
import oracle
from _util import device_gaussians, normwise

pytestmark = pytest.mark.gpu


def test_config3_batched_forward_and_graph():
    import torch
    import paper_2501_06838_gb300 as gs
    gsets, views = S.config3()
    dgs = [device_gaussians(g) for g in gsets]
    plan = gs.Plan(dgs, views, with_grads=False)
    outs = [o.clone() for o in plan.fwd()]
    plan.status()
    st = plan.stats()
    assert st["n_tiles"] == sum(((v.out_w + 15) // 16) * ((v.out_h + 15) // 16) for v in views)
    for g, v, o in zip(gsets, views, outs):
        ref = oracle.render(g, v)
        assert np.all(normwise(o.cpu().double().numpy(), ref, axis=(1, 2)) < 1e-5)
    # one CUDA graph for the whole batched chain, replayed twice
    for o in plan.outs:
        o.zero_()
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        plan.fwd(stream)          # warm-up on the capture stream
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=stream):
            plan.fwd(stream)
    for _ in range(2):
        for o in plan.outs:
            o.zero_()
        graph.replay()
        torch.cuda.synchronize()
        for a, b in zip(plan.outs, outs):
            assert torch.equal(a, b)        # the forward is bitwise reproducible
    plan.status()


def test_kernel_timing_under_graph_capture():
    """Launches timed under stream capture record the graph's event nodes:
    every replay re-records them, each read gives the last replay's times."""
    import torch
    import paper_2501_06838_gb300 as gs
    gsets, views = S.config3(4)
    dgs = [device_gaussians(g) for g in gsets]
    plan = gs.Plan(dgs, views, with_grads=False)
    plan.fwd()
    torch.cuda.synchronize()
    gs.timing_read()
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    gs.timing_enable(["raster_fwd"])
    with torch.cuda.graph(graph, stream=stream):
        plan.fwd(stream)
    gs.timing_enable([])
    assert gs.timing_read() == {}          # nothing replayed yet
    for _ in range(3):
        graph.replay()
        torch.cuda.synchronize()
        kt = gs.timing_read()
        assert kt["raster_fwd"][1] == 1 and kt["raster_fwd"][0] > 0.0
    gs.timing_release()
    graph.replay()
    torch.cuda.synchronize()
    assert gs.timing_read() == {}
    plan.status()


def test_batched_equals_single_image_calls():
    import torch
    import paper_2501_06838_gb300 as gs
    gsets, views = S.config3(n_images=4)
    dgs = [device_gaussians(g) for g in gsets]
    outs, _ = gs.render_batched(dgs, views, check=True)
    for dg, v, o in zip(dgs, views, outs):
        single, _ = gs.render(dg, v, check=True)
        assert torch.equal(single, o)


def test_batched_adjoint():
    """Uneven batch of 5 smaller images (sizes and scales drawn like config 3,
    LR sides divided by 4), against the oracle adjoint per image."""
    import torch
    import paper_2501_06838_gb300 as gs
    sizes = S.config3_sizes(7, 5)
    gsets, views = [], []
    for i, (h, w, s) in enumerate(sizes):
        h, w = max(h // 4, 8), max(w // 4, 8)
        gsets.append(S.draw_gaussians(300 + i, h, w, 1, (0.3, 2.0)))
        views.append(S.View(h, w, S.out_size(h, s), S.out_size(w, s), s))
    dgs = [device_gaussians(g) for g in gsets]
    outs, ws = gs.render_batched(dgs, views, check=True)
    gos = [S.grad_out(10 + i, v.out_h, v.out_w) for i, v in enumerate(views)]
    grads = gs.render_batched_bwd(dgs, views, [torch.from_numpy(x).cuda() for x in gos], ws,
                                  check=True)
    for g, v, go, gr in zip(gsets, views, gos, grads):
        ref = oracle.adjoint(g, v, go)
        assert np.all(normwise(gr.cpu().double().numpy(), ref, axis=0) < 1e-5)


@pytest.mark.parametrize("adjoint", [1, 3])
def test_forward_and_adjoint_graph_replays(adjoint):
    """Forward and adjoint captured in one CUDA graph and replayed three times
    with a new upstream gradient each time. 5,250 tiles (21,000 quadrants) are
    more than the adjoint's resident CTAs, so every replay runs the adjoint's
    work counter, which the captured chain must reset: each replay's gradients
    match the oracle's, and the images are bitwise the eager forward's."""
    import torch
    import paper_2501_06838_gb300 as gs
    h, w = 280, 300
    g = S.draw_gaussians(41, h, w, 1, (0.3, 2.0))
    v = S.View(h, w, S.out_size(h, 4.0), S.out_size(w, 4.0), 4.0)
    v.adjoint = adjoint
    assert ((v.out_h + 15) // 16) * ((v.out_w + 15) // 16) == 5250
    plan = gs.Plan([device_gaussians(g)], [v], with_grads=True)
    ref_img = plan.fwd()[0].clone()
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        plan.fwd(stream)
        plan.bwd(stream)          # warm-up on the capture stream
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=stream):
            plan.fwd(stream)
            plan.bwd(stream)
    for seed in (51, 52, 51):
        go = S.grad_out(seed, v.out_h, v.out_w)
        plan.grad_outs[0].copy_(torch.from_numpy(go))
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(plan.outs[0], ref_img)
        ref = oracle.adjoint(g, v, go)
        err = normwise(plan.grads[0].cpu().double().numpy(), ref, axis=0)
        assert np.all(err < 1e-5), err
    plan.status()
    assert gs.read_stats(plan.ws)["adjoint"] == adjoint
