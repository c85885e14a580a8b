"""Config 4: reduced-precision parameter storage (BF16, FP16) with FP32
arithmetic, LR 480x270 with 4 Gaussians per LR pixel (N = 518,400), sigma in
[0.2, 3] LR px, at x8 (3840x2160) and x12 (5760x3240).

Two comparisons (GSASR's render is defined on real-valued parameters):
  (i)  arithmetic: the GPU against the FP64 oracle fed the SAME rounded values,
       1e-5 normwise per channel (forward) and per field (adjoint);
  (ii) storage: the GPU against the oracle on the FP32 originals, i.e. the error
       that rounding the parameters to BF16 / FP16 causes. Reported as max-abs,
       normwise and PSNR; the 3e-3 bound applies to the RMS error relative to
       the image maximum (the max-norm error of BF16 storage alone is ~7e-3).
       The adjoint's storage error is reported the same way per gradient field
       (normwise and RMS relative to the field's largest magnitude), and the
       same 3e-3 RMS bound applies to every field.
"""
import numpy as np
import pytest

import gs_synthetic as S
import oracle
from _util import device_gaussians, normwise, psnr

pytestmark = pytest.mark.gpu
FIELDS = ("o_x", "o_y", "sigma_x", "sigma_y", "rho", "r", "g", "b", "alpha")


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("scale", [8.0, 12.0])
def test_config4(dtype, scale, record_property):
    import torch
    import paper_2501_06838_gb300 as gs
    gset, views = S.config4(scale, dtype)
    g, v = gset[0], views[0]
    dg = device_gaussians(g)
    out, ws = gs.render(dg, v, check=True)
    go = S.grad_out(1, v.out_h, v.out_w)
    gr = gs.render_bwd(dg, v, torch.from_numpy(go).cuda(), ws, check=True)
    out = out.cpu().double().numpy()
    gr = gr.cpu().double().numpy()
    # (i) arithmetic error against the same rounded parameters
    ref = oracle.render(g, v)
    e_img = normwise(out, ref, axis=(1, 2))
    assert np.all(e_img < 1e-5), e_img
    ref_g = oracle.adjoint(g, v, go)
    e_g = normwise(gr, ref_g, axis=0)
    assert np.all(e_g < 1e-5), dict(zip(FIELDS, e_g))
    # (ii) storage error against the FP32 originals
    ref32 = oracle.render(g.originals, v)
    diff = out - ref32
    rms_rel = float(np.sqrt(np.mean(diff ** 2)) / np.abs(ref32).max())
    stats = {"max_abs": float(np.abs(diff).max()),
             "normwise": float(normwise(out, ref32, axis=(1, 2)).max()),
             "rms_rel": rms_rel, "psnr_db": psnr(out, ref32)}
    record_property("storage_error", stats)
    print(f"{dtype} x{scale:g}: storage error {stats}")
    assert rms_rel < 3e-3, stats
    # the adjoint's storage error, per field, against the FP32 originals
    ref_g32 = oracle.adjoint(g.originals, v, go)
    gd = gr - ref_g32
    peak = np.abs(ref_g32).max(axis=0)
    g_stats = {f: {"normwise": float(np.abs(gd[:, k]).max() / peak[k]),
                   "rms_rel": float(np.sqrt(np.mean(gd[:, k] ** 2)) / peak[k])}
               for k, f in enumerate(FIELDS)}
    record_property("adjoint_storage_error", g_stats)
    print(f"{dtype} x{scale:g}: adjoint storage error {g_stats}")
    assert all(e["rms_rel"] < 3e-3 for e in g_stats.values()), g_stats
