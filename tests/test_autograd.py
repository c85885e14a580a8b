"""torch.autograd.Function wrappers (differentiable render, GSASR Sec. 3.2
"Rendering"): gradients flow through GSRender / GSRenderBatched into upstream
parameters and agree with the oracle's adjoint."""
import numpy as np
import pytest

import gs_synthetic as S
import oracle
from _util import device_gaussians, normwise

pytestmark = pytest.mark.gpu


def test_gsrender_matches_oracle_adjoint():
    import torch
    import paper_2501_06838_gb300 as gs
    g, v = S.config1()[0][0], S.config1()[1][0]
    dg = device_gaussians(g)
    params = [t.clone().requires_grad_(True) for t in dg.tensors()]
    img = gs.GSRender.apply(*params, v, g.ref_grid_m)
    go = S.grad_out(3, v.out_h, v.out_w)
    (img * torch.from_numpy(go).cuda()).sum().backward()
    ref = oracle.adjoint(g, v, go)
    got = np.concatenate([params[0].grad.cpu().numpy(), params[1].grad.cpu().numpy(),
                          params[2].grad.cpu().numpy()[:, None], params[3].grad.cpu().numpy(),
                          params[4].grad.cpu().numpy()[:, None]], 1)
    assert np.all(normwise(got, ref, axis=0) < 1e-5)


def test_gsrender_chain_rule_through_activations():
    """A head-style reparametrisation upstream of the renderer: autograd's chain
    rule through torch ops composes with the renderer's adjoint."""
    import torch
    import paper_2501_06838_gb300 as gs
    torch.manual_seed(0)
    n, H, W, s = 16 * 16, 16, 16, 2.5
    raw = torch.randn(n, 9, device="cuda", dtype=torch.float64, requires_grad=True)
    v = S.View(H, W, S.out_size(H, s), S.out_size(W, s), s)

    def params(r):
        return (torch.tanh(r[:, 0:2]) * 0.5, 0.3 + 1.5 * torch.sigmoid(r[:, 2:4]),
                0.9 * torch.tanh(r[:, 4]), torch.sigmoid(r[:, 5:8]), torch.sigmoid(r[:, 8]))

    p = [t.float().contiguous() for t in params(raw)]
    img = gs.GSRender.apply(*p, v, 1)
    w = torch.randn_like(img)
    (img * w).sum().backward()
    g_gpu = raw.grad.clone()
    # same chain with the oracle adjoint in place of the renderer
    with torch.no_grad():
        p32 = [t.float() for t in params(raw)]
    gset = S.GaussianSet(*[t.double().cpu().numpy() for t in p32], lr_h=H, lr_w=W, ref_grid_m=1)
    A = torch.from_numpy(oracle.adjoint(gset, v, w.double().cpu().numpy())).cuda()
    raw.grad = None
    pp = params(raw)
    dots = (pp[0] * A[:, 0:2]).sum() + (pp[1] * A[:, 2:4]).sum() + (pp[2] * A[:, 4]).sum() + \
           (pp[3] * A[:, 5:8]).sum() + (pp[4] * A[:, 8]).sum()
    dots.backward()
    err = (g_gpu - raw.grad).abs().max() / raw.grad.abs().max()
    assert err < 2e-5, float(err)


def test_gsrender_batched_autograd():
    import torch
    import paper_2501_06838_gb300 as gs
    sizes = [(12, 16, 2.5), (20, 8, 3.25), (8, 8, 1.5)]
    gsets = [S.draw_gaussians(50 + i, h, w, 1) for i, (h, w, _) in enumerate(sizes)]
    views = [S.View(h, w, S.out_size(h, s), S.out_size(w, s), s) for h, w, s in sizes]
    cat = [torch.cat([t for t in ts]) for ts in zip(*[device_gaussians(g).tensors() for g in gsets])]
    params = [t.clone().requires_grad_(True) for t in cat]
    outs = gs.GSRenderBatched.apply(views, 1, [g.n for g in gsets], None, *params)
    gos = [S.grad_out(20 + i, v.out_h, v.out_w) for i, v in enumerate(views)]
    loss = sum((o * torch.from_numpy(x).cuda()).sum() for o, x in zip(outs, gos))
    loss.backward()
    o = 0
    for g, v, go in zip(gsets, views, gos):
        ref = oracle.adjoint(g, v, go)
        got = np.concatenate([params[0].grad[o:o + g.n].cpu().numpy(),
                              params[1].grad[o:o + g.n].cpu().numpy(),
                              params[2].grad[o:o + g.n].cpu().numpy()[:, None],
                              params[3].grad[o:o + g.n].cpu().numpy(),
                              params[4].grad[o:o + g.n].cpu().numpy()[:, None]], 1)
        assert np.all(normwise(got, ref, axis=0) < 1e-5)
        o += g.n
