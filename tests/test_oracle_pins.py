"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: each check has an independent
source of truth (a closed form, a symmetry of Eq. 4, a brute force with another
code path, an independent differentiator). Citations: GSASR, arXiv 2501.06838.
"""
import json
import math
import os

import numpy as np
import pytest

import gs_synthetic as S
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def one(mx, my, sx, sy, rho, rgb=(0.25, 0.5, 0.75), alpha=0.8):
    """A GaussianSet of explicit absolute-centre Gaussians (lists allowed)."""
    mx, my, sx, sy, rho, alpha = (np.atleast_1d(np.asarray(a, dtype=np.float64))
                                  for a in (mx, my, sx, sy, rho, alpha))
    n = max(len(mx), len(rho))
    b = lambda a: np.broadcast_to(a, (n,)).astype(np.float64)
    rgb = np.broadcast_to(np.asarray(rgb, dtype=np.float64), (n, 3)).copy()
    f32 = lambda a: a.astype(np.float32).astype(np.float64)
    return S.GaussianSet(f32(np.stack([b(mx), b(my)], 1)), f32(np.stack([b(sx), b(sy)], 1)),
                         f32(b(rho)), f32(rgb), f32(b(alpha)), lr_h=1, lr_w=1, ref_grid_m=0)


# --------------------------------------------------------------------------
# Normalisation, centre, covariance: Poisson summation (Eq. 2 and Eq. 4).
# For a smooth Gaussian sampled on the HR lattice (spacing 1/s in LR units),
# sum_x f(x/s) = s^2 * (1 + eps), |eps| <= 4 exp(-2 pi^2 lambda_min s^2), and
# the sampled first and second moments equal mu, Sigma to the same order.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("sx,sy,rho,s", [(1.3, 0.9, 0.6, 3.0), (0.7, 1.1, -0.75, 4.0),
                                         (1.0, 1.0, 0.0, 2.5), (2.0, 0.5, 0.3, 6.0)])
def test_poisson_sum_and_moments(sx, sy, rho, s):
    lam = np.linalg.eigvalsh([[sx * sx, rho * sx * sy], [rho * sx * sy, sy * sy]]).min()
    assert 4 * math.exp(-2 * math.pi ** 2 * lam * s * s) < 1e-12
    L = 12.0 * max(sx, sy)                 # LR half-extent of the canvas
    size = int(2 * L * s) + 1
    mu = (L + 0.137, L - 0.291)
    g = one(mu[0], mu[1], sx, sy, rho)
    alpha, c = g.alpha[0], g.rgb[0]
    v = S.View(size, size, size, size, s, trunc_k=0.0)
    img = oracle.render(g, v)
    total = img.sum(axis=(1, 2))
    np.testing.assert_allclose(total, s * s * alpha * c, rtol=1e-10)
    # moments in LR units
    I = img[2]
    ys, xs = np.mgrid[0:size, 0:size] / np.float64(np.float32(s))
    m0 = I.sum()
    mx_, my_ = (I * xs).sum() / m0, (I * ys).sum() / m0
    g_mu = g.offset[0]
    assert abs(mx_ - g_mu[0]) < 1e-9 and abs(my_ - g_mu[1]) < 1e-9
    vxx = (I * (xs - g_mu[0]) ** 2).sum() / m0
    vyy = (I * (ys - g_mu[1]) ** 2).sum() / m0
    vxy = (I * (xs - g_mu[0]) * (ys - g_mu[1])).sum() / m0
    gs_, gr = g.sigma[0], g.rho[0]
    assert abs(vxx - gs_[0] ** 2) < 1e-8
    assert abs(vyy - gs_[1] ** 2) < 1e-8
    assert abs(vxy - gr * gs_[0] * gs_[1]) < 1e-8          # pins the sign of rho
    # peak normalisation: the sum is 2 pi sx sy sqrt(1 - rho^2) s^2 alpha c
    vp = S.View(size, size, size, size, s, trunc_k=0.0, norm=S.NORM_PEAK)
    tp = oracle.render(g, vp).sum(axis=(1, 2))
    D = (1 - gr) * (1 + gr)
    np.testing.assert_allclose(tp, 2 * math.pi * gs_[0] * gs_[1] * math.sqrt(D) * s * s * alpha * c,
                               rtol=1e-10)
    # the peak value itself in peak mode is alpha * c (at the centre pixel when the
    # centre sits on a pixel)
    g2 = one(20.0, 20.0, sx, sy, rho)
    v2 = S.View(64, 64, 64, 64, 1.0, trunc_k=0.0, norm=S.NORM_PEAK)
    np.testing.assert_allclose(oracle.render(g2, v2)[:, 20, 20], g2.alpha[0] * g2.rgb[0], rtol=1e-15)


# --------------------------------------------------------------------------
# Constant-colour field (Eq. 3): Gaussians with alpha = 1/m on the reference
# grid of m per LR pixel tile the plane; interior pixels equal c up to the
# Poisson aliasing term (<= 4 exp(-2 pi^2 sigma^2 m) relative).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("m", [1, 4, 9, 16])
def test_constant_colour_field(m):
    H = W = 24
    sig = 1.2
    n = m * H * W
    c = np.array([0.25, 0.5, 0.75])
    f32 = lambda a: a.astype(np.float32).astype(np.float64)
    g = S.GaussianSet(np.zeros((n, 2)), np.full((n, 2), sig), np.zeros(n), np.tile(c, (n, 1)),
                      f32(np.full(n, 1.0 / m)), lr_h=H, lr_w=W, ref_grid_m=m)
    s = 2.0
    v = S.View(H, W, int(H * s), int(W * s), s, trunc_k=0.0)
    img = oracle.render(g, v)
    lo, hi = int(9 * s), int(15 * s)                 # >= 7.5 sigma from the border
    interior = img[:, lo:hi, lo:hi]
    alpha32 = np.float32(1.0 / m) * m                # alpha is stored in float32
    # m = 9: the sub-grid steps of 1/3 are rounded to float32, so the lattice is
    # regular only to ~1e-7 LR px and the field is flat only to ~1e-7.
    tol = 2e-8 if m in (1, 4, 16) else 2e-7
    for k in range(3):
        np.testing.assert_allclose(interior[k], c[k] * alpha32, rtol=tol)


def test_reference_positions():
    """p sits on an equal-interval sqrt(m) x sqrt(m) sub-grid of each LR pixel
    (Sec. 3.2); checked through the rendered mean of single Gaussians."""
    H, W = 5, 7
    for m in (1, 4, 9, 16):
        n = int(math.isqrt(m))
        gids = [0, m * W + 1, m * (3 * W + 5) + (m - 1), m * (4 * W + 6) + (m // 2)]
        for gid in gids:
            cell, sub = divmod(gid, m)
            i, j = divmod(cell, W)
            b, a = divmod(sub, n)
            px = j - 0.5 + (a + 0.5) / n
            py = i - 0.5 + (b + 0.5) / n
            mu = oracle.centre(S.GaussianSet(np.zeros((H * W * m, 2)), np.ones((H * W * m, 2)),
                                             np.zeros(H * W * m), np.ones((H * W * m, 3)),
                                             np.ones(H * W * m), H, W, m), S.View(H, W, H, W, 1.0), gid)
            assert abs(mu[0] - px) < 1e-6 and abs(mu[1] - py) < 1e-6


# --------------------------------------------------------------------------
# The truncation window (Algorithm 1 box, 3-sigma footprint): with rho = 0 the
# truncated sum factorises into two 1-D sums over |x - s mu| <= s k sigma.
# --------------------------------------------------------------------------
def test_truncated_box_separable():
    rng = np.random.default_rng(5)
    for _ in range(20):
        s = float(np.float32(rng.uniform(1.5, 7.0)))
        sx, sy = rng.uniform(0.4, 2.5, 2)
        mx, my = rng.uniform(8, 12, 2)
        g = one(mx, my, sx, sy, 0.0)
        gmx, gmy = g.offset[0]
        gsx, gsy = g.sigma[0]
        W = H = int(24 * s)
        v = S.View(24, 24, H, W, s, trunc_k=3.0)

        def window(mu, sig, n):
            lo, hi = s * mu - s * 3.0 * sig, s * mu + s * 3.0 * sig
            assert min(abs(lo - round(lo)), abs(hi - round(hi))) > 1e-4   # no float32 tie
            xs = np.arange(n)
            return xs[(xs >= lo) & (xs <= hi)]

        xs, ys = window(gmx, gsx, W), window(gmy, gsy, H)
        fx = np.exp(-0.5 * (xs / s - gmx) ** 2 / gsx ** 2)
        fy = np.exp(-0.5 * (ys / s - gmy) ** 2 / gsy ** 2)
        Z = 1.0 / (2 * math.pi * gsx * gsy)
        expect = g.alpha[0] * g.rgb[0] * Z * fx.sum() * fy.sum()
        img = oracle.render(g, v)
        np.testing.assert_allclose(img.sum(axis=(1, 2)), expect, rtol=1e-12)
        # nothing is drawn outside the box
        mask = np.zeros((H, W), bool)
        mask[ys[0]:ys[-1] + 1, xs[0]:xs[-1] + 1] = True
        assert np.all(img[:, ~mask] == 0.0)


def test_truncated_mass_erf():
    """Captured mass of the 3-sigma box for a wide Gaussian -> erf(3/sqrt 2)^2."""
    with open(os.path.join(GOLDEN, "closed_forms.json")) as f:
        gold = json.load(f)
    s = 10.0
    g = one(20.03, 19.97, 2.0, 2.5, 0.0)
    v = S.View(40, 40, 400, 400, s, trunc_k=3.0)
    frac = oracle.render(g, v).sum(axis=(1, 2)) / (s * s * g.alpha[0] * g.rgb[0])
    # Euler-Maclaurin edge error of the box sum is O(f_edge / (s sigma)) ~ 1e-3
    np.testing.assert_allclose(frac, gold["erf3_squared"], atol=2e-3)


# --------------------------------------------------------------------------
# Scale convention (Eq. 4) and symmetries of the lattice.
# --------------------------------------------------------------------------
def test_integer_scale_subsampling():
    rng = np.random.default_rng(1)
    n = 60
    g = one(rng.uniform(2, 14, n).round(3), rng.uniform(2, 14, n).round(3),
            rng.uniform(0.3, 1.5, n), rng.uniform(0.3, 1.5, n), rng.uniform(-0.9, 0.9, n),
            rng.uniform(0, 1, (n, 3)), rng.uniform(0, 1, n))
    base = oracle.render(g, S.View(16, 16, 16, 16, 1.0))
    for s in (2, 4):
        up = oracle.render(g, S.View(16, 16, 16 * s, 16 * s, float(s)))
        np.testing.assert_allclose(up[:, ::s, ::s], base, rtol=1e-13, atol=1e-15)
    # s = 1 is Eq. 3: the LR representation itself, checked against a direct sum
    I = np.zeros((3, 16, 16))
    r = oracle.rects(g, S.View(16, 16, 16, 16, 1.0))
    for i in range(n):
        x0, x1, y0, y1 = r[i]
        mx, my = g.offset[i]
        sx, sy = g.sigma[i]
        rh = g.rho[i]
        D = (1 - rh) * (1 + rh)
        for y in range(y0, y1 + 1):
            for x in range(x0, x1 + 1):
                u, w = x - mx, y - my
                q = (u * u / sx ** 2 - 2 * rh * u * w / (sx * sy) + w * w / sy ** 2) / D
                I[:, y, x] += g.alpha[i] * g.rgb[i] * math.exp(-q / 2) / (2 * math.pi * sx * sy * math.sqrt(D))
    np.testing.assert_allclose(base, I, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("trunc", [0.0, 3.0])
def test_translation(trunc):
    """Shifting every centre by t with s*t integer shifts the image by s*t pixels
    (Eq. 4). Dyadic centres and sigmas keep every float32 window edge exact."""
    rng = np.random.default_rng(2)
    n = 40
    d = lambda a: (a * 256).round() / 256
    mx = d(rng.uniform(9, 12, n))
    my = d(rng.uniform(10, 14, n))
    args = (d(rng.uniform(0.3, 1.2, n)), d(rng.uniform(0.3, 1.2, n)), rng.uniform(-0.9, 0.9, n),
            rng.uniform(0, 1, (n, 3)), rng.uniform(0, 1, n))
    s = 2.0
    v = S.View(32, 32, 64, 64, s, trunc_k=trunc)
    a = oracle.render(one(mx, my, *args), v)
    b = oracle.render(one(mx + 3.0, my - 2.0, *args), v)
    # shift by (3, -2) LR px = (6, -4) HR px
    np.testing.assert_allclose(b[:, 4:60, 6:64], a[:, 8:64, 0:58], rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("trunc", [0.0, 3.0])
def test_rotation_90(trunc):
    rng = np.random.default_rng(3)
    n = 50
    s = 2.0
    Wo = 64
    mx = (rng.uniform(4, 28, n) * 256).round() / 256
    my = (rng.uniform(4, 28, n) * 256).round() / 256
    sx = (rng.uniform(0.3, 1.5, n) * 256).round() / 256
    sy = (rng.uniform(0.3, 1.5, n) * 256).round() / 256
    rho = rng.uniform(-0.9, 0.9, n)
    rgb, al = rng.uniform(0, 1, (n, 3)), rng.uniform(0, 1, n)
    v = S.View(32, 32, Wo, Wo, s, trunc_k=trunc)
    a = oracle.render(one(mx, my, sx, sy, rho, rgb, al), v)
    # (x, y) -> (y, W-1-x): mu' = (mu_y, (W-1)/s - mu_x), sigma swapped, rho -> -rho
    b = oracle.render(one(my, (Wo - 1) / s - mx, sy, sx, -rho, rgb, al), v)
    for k in range(3):
        np.testing.assert_allclose(b[k], np.rot90(a[k]), rtol=1e-12, atol=1e-16)


def test_rotation_invariant_sum():
    """An arbitrary rotation of Sigma keeps det Sigma, so the untruncated sum is
    unchanged (Poisson summation)."""
    s = 3.0
    base = None
    for th in np.linspace(0, math.pi, 7):
        R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
        Sg = R @ np.diag([1.4 ** 2, 0.8 ** 2]) @ R.T
        sx, sy = math.sqrt(Sg[0, 0]), math.sqrt(Sg[1, 1])
        rho = Sg[0, 1] / (sx * sy)
        g = one(20.0, 20.0, sx, sy, rho)
        v = S.View(40, 40, 120, 120, s, trunc_k=0.0)
        gs_, gr = g.sigma[0], g.rho[0]
        t = oracle.render(g, v).sum() / (gs_[0] * gs_[1] * math.sqrt((1 - gr) * (1 + gr)))
        v2 = S.View(40, 40, 120, 120, s, trunc_k=0.0, norm=S.NORM_PEAK)
        tp = oracle.render(g, v2).sum() / (gs_[0] * gs_[1] * math.sqrt((1 - gr) * (1 + gr)))
        base = tp if base is None else base
        np.testing.assert_allclose(tp, base, rtol=1e-9)


def test_linearity():
    gs, vs = S.config1()
    g, v = gs[0], vs[0]
    full = oracle.render(g, v)
    half = g.n // 2
    a = S.GaussianSet(g.offset[:half], g.sigma[:half], g.rho[:half], g.rgb[:half], g.alpha[:half],
                      g.lr_h, g.lr_w, 1)
    # the second half keeps its reference positions by using absolute centres
    mu = np.stack([oracle.centre(g, v, i) for i in range(half, g.n)])
    b = S.GaussianSet(mu, g.sigma[half:], g.rho[half:], g.rgb[half:], g.alpha[half:],
                      g.lr_h, g.lr_w, 0)
    np.testing.assert_allclose(oracle.render(a, v) + oracle.render(b, v), full, rtol=1e-12, atol=1e-14)


# --------------------------------------------------------------------------
# Brute force: the rectangle loop equals the all-pairs loop with the window's
# defining float32 inequalities (no integer rectangle, no clamping).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed,s", [(0, 2.7), (1, 1.0), (2, 5.3), (3, 3.0)])
def test_rect_equals_allpairs(seed, s):
    rng = np.random.default_rng(seed)
    n = 200
    H, W = 20, 26
    g = one(rng.uniform(-2, W + 2, n), rng.uniform(-2, H + 2, n), rng.uniform(0.2, 2.5, n),
            rng.uniform(0.2, 2.5, n), rng.uniform(-0.95, 0.95, n), rng.uniform(0, 1, (n, 3)),
            rng.uniform(0, 1, n))
    v = S.View(H, W, S.out_size(H, s), S.out_size(W, s), s)
    a = oracle.render(g, v)
    b = oracle.render(g, v, mode="allpairs")
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-15)


# --------------------------------------------------------------------------
# Adjoint: three independent differentiators.
# --------------------------------------------------------------------------
def test_adjoint_vs_complex_step():
    gs, vs = S.config1()
    g, v = gs[0], vs[0]
    go = S.grad_out(1, v.out_h, v.out_w)
    ids = S.sample_indices(7, g.n, 40)
    for norm in (S.NORM_DENSITY, S.NORM_PEAK):
        vv = S.View(v.lr_h, v.lr_w, v.out_h, v.out_w, v.scale, norm=norm)
        A = oracle.adjoint(g, vv, go)[ids]
        C = oracle.complex_step(g, vv, go, ids)
        np.testing.assert_allclose(A, C, rtol=1e-10, atol=1e-12 * np.abs(C).max())


def test_adjoint_vs_torch_autograd():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    n, H, W, s = 12, 10, 12, 2.5
    g = one(rng.uniform(1, 11, n), rng.uniform(1, 9, n), rng.uniform(0.3, 1.5, n),
            rng.uniform(0.3, 1.5, n), rng.uniform(-0.9, 0.9, n), rng.uniform(0, 1, (n, 3)),
            rng.uniform(0, 1, n))
    v = S.View(H, W, S.out_size(H, s), S.out_size(W, s), s)
    go = rng.standard_normal((3, v.out_h, v.out_w))
    rect = oracle.rects(g, v)
    t = lambda a: torch.tensor(a, dtype=torch.float64, requires_grad=True)
    mx, my = t(g.offset[:, 0]), t(g.offset[:, 1])
    sx, sy = t(g.sigma[:, 0]), t(g.sigma[:, 1])
    rho, rgb, al = t(g.rho), t(g.rgb), t(g.alpha)
    ys, xs = torch.meshgrid(torch.arange(v.out_h, dtype=torch.float64),
                            torch.arange(v.out_w, dtype=torch.float64), indexing="ij")
    X, Y = xs / v.scale, ys / v.scale
    mask = torch.zeros(n, v.out_h, v.out_w, dtype=torch.float64)
    for i in range(n):
        x0, x1, y0, y1 = rect[i]
        mask[i, y0:y1 + 1, x0:x1 + 1] = 1.0
    # a dense restatement of the multivariate normal density, written via its
    # covariance matrix (not via the oracle's expanded quadratic form)
    cov = torch.stack([torch.stack([sx * sx, rho * sx * sy], -1),
                       torch.stack([rho * sx * sy, sy * sy], -1)], -2)
    d = torch.stack([X[None] - mx[:, None, None], Y[None] - my[:, None, None]], -1)
    prec = torch.linalg.inv(cov)
    q = torch.einsum("nhwi,nij,nhwj->nhw", d, prec, d)
    f = torch.exp(-0.5 * q) / (2 * math.pi * torch.sqrt(torch.linalg.det(cov)))[:, None, None]
    I = torch.einsum("nhw,nk->khw", f * mask * al[:, None, None], rgb)
    L = (I * torch.tensor(go)).sum()
    L.backward()
    ref = torch.stack([mx.grad, my.grad, sx.grad, sy.grad, rho.grad, rgb.grad[:, 0],
                       rgb.grad[:, 1], rgb.grad[:, 2], al.grad], 1).numpy()
    A = oracle.adjoint(g, v, go)
    np.testing.assert_allclose(A, ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())
    np.testing.assert_allclose(oracle.render(g, v), I.detach().numpy(), rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("window,norm,head", [(S.WINDOW_SIGMA, S.NORM_DENSITY, False),
                                               (S.WINDOW_RATIO, S.NORM_PEAK, False),
                                               (S.WINDOW_SIGMA, S.NORM_DENSITY, True)])
def test_adjoint_dot_product(window, norm, head):
    """<g, J d> = <J^T g, d> for the whole render: J d is the directional
    derivative of the render itself (all Gaussians moved at once along a random
    direction d, windows frozen) by Richardson-extrapolated central differences;
    J^T g is the hand adjoint. Ties the adjoint to the forward the parity tests
    use, not to a per-Gaussian loss routine."""
    rng = np.random.default_rng(29)
    h, w, m, s = 6, 5, 4, 2.7
    g = S.draw_raw_head(3, h, w, m) if head else S.draw_gaussians(3, h, w, m, (0.4, 1.6))
    v = S.View(h, w, S.out_size(h, s), S.out_size(w, s), s,
               trunc_k=0.3 if window == S.WINDOW_RATIO else 3.0, norm=norm, window=window)
    rect = oracle.rects(g, v)
    go = rng.standard_normal((3, v.out_h, v.out_w))
    d = [rng.standard_normal(a.shape) for a in g.fields()]

    def loss(t):
        moved = S.GaussianSet(*(a + t * da for a, da in zip(g.fields(), d)), lr_h=h, lr_w=w,
                              ref_grid_m=m, head=g.head)
        return float(np.sum(go * oracle.render(moved, v, frozen_rects=rect, threads=1)))

    # steps of 3e-5: the h^4 remainder and the rounding both stay near 1e-11
    e = 3e-5
    c1 = (loss(e) - loss(-e)) / (2 * e)
    c2 = (loss(2 * e) - loss(-2 * e)) / (4 * e)
    jd = (4 * c1 - c2) / 3
    A = oracle.adjoint(g, v, go, threads=1, frozen_rects=rect)
    flat = np.concatenate([d[0], d[1], d[2][:, None], d[3], d[4][:, None]], 1)
    jtg = float(np.sum(A * flat))
    assert abs(jd - jtg) <= 1e-9 * abs(jtg)


def test_adjoint_vs_central_difference_config2():
    """Config 2's check: central differences (h = 1e-4) on 64 Gaussians (seed 2)."""
    gs, vs = S.config2()
    g, v = gs[0], vs[0]
    go = S.grad_out(1, v.out_h, v.out_w)
    ids = S.sample_indices(2, g.n, 64)
    A = oracle.adjoint(g, v, go)[ids]
    F = oracle.central_difference(g, v, go, ids, h=1e-4)
    scale = np.abs(A).max(axis=0)
    assert np.all(np.abs(A - F).max(axis=0) <= 1e-6 * scale)


def test_golden_regression():
    """A small render stored by tests/golden/make_golden.py (oracle only)."""
    with open(os.path.join(GOLDEN, "oracle_small.json")) as f:
        gold = json.load(f)
    g = one(*[np.array(gold["params"][k]) for k in ("mx", "my", "sx", "sy", "rho")],
            np.array(gold["params"]["rgb"]), np.array(gold["params"]["alpha"]))
    v = S.View(**gold["view"])
    img = oracle.render(g, v)
    np.testing.assert_allclose(img[:, gold["probe_y"], gold["probe_x"]], np.array(gold["values"]),
                               rtol=1e-12)


# --------------------------------------------------------------------------
# Algorithm 1's ratio window: |x - s mu_x| < s r W, |y - s mu_y| < s r H (an
# open box whose half-widths are a fraction r of the HR image). With rho = 0
# the windowed sum factorises into two 1-D sums over that open interval.
# --------------------------------------------------------------------------
def test_ratio_window_separable():
    rng = np.random.default_rng(15)
    for _ in range(20):
        s = float(np.float32(rng.uniform(1.5, 7.0)))
        r = float(np.float32(rng.uniform(0.03, 0.12)))
        Wl, Hl = 30, 22
        sx, sy = rng.uniform(0.4, 2.5, 2)
        mx, my = rng.uniform(8, 20, 1)[0], rng.uniform(6, 14, 1)[0]
        g = one(mx, my, sx, sy, 0.0)
        gmx, gmy = g.offset[0]
        gsx, gsy = g.sigma[0]
        Wo, Ho = S.out_size(Wl, s), S.out_size(Hl, s)
        v = S.View(Hl, Wl, Ho, Wo, s, trunc_k=r, window=S.WINDOW_RATIO)

        def window(mu, L, n):
            lo, hi = s * mu - s * r * L, s * mu + s * r * L
            assert min(abs(lo - round(lo)), abs(hi - round(hi))) > 1e-4   # no float32 tie
            xs = np.arange(n)
            return xs[(xs > lo) & (xs < hi)]

        xs, ys = window(gmx, Wl, Wo), window(gmy, Hl, Ho)
        fx = np.exp(-0.5 * (xs / s - gmx) ** 2 / gsx ** 2)
        fy = np.exp(-0.5 * (ys / s - gmy) ** 2 / gsy ** 2)
        Z = 1.0 / (2 * math.pi * gsx * gsy)
        expect = g.alpha[0] * g.rgb[0] * Z * fx.sum() * fy.sum()
        img = oracle.render(g, v)
        np.testing.assert_allclose(img.sum(axis=(1, 2)), expect, rtol=1e-12)
        mask = np.zeros((Ho, Wo), bool)
        mask[ys[0]:ys[-1] + 1, xs[0]:xs[-1] + 1] = True
        assert np.all(img[:, ~mask] == 0.0)
        r4 = oracle.rects(g, v)[0]
        assert (r4[0], r4[1], r4[2], r4[3]) == (xs[0], xs[-1], ys[0], ys[-1])


@pytest.mark.parametrize("window,k,align", [(1, 0.05, 0), (1, 0.1, 1), (0, 3.0, 1), (1, 0.02, 1)])
def test_flags_rect_equals_allpairs(window, k, align):
    """Rectangle loop == all-pairs loop with the window's own float32 inequalities,
    for the ratio window and for the half-pixel alignment."""
    rng = np.random.default_rng(31 + int(k * 100) + align)
    n = 150
    H, W = 20, 26
    g = one(rng.uniform(-2, W + 2, n), rng.uniform(-2, H + 2, n), rng.uniform(0.2, 2.5, n),
            rng.uniform(0.2, 2.5, n), rng.uniform(-0.95, 0.95, n), rng.uniform(0, 1, (n, 3)),
            rng.uniform(0, 1, n))
    s = 2.7
    v = S.View(H, W, S.out_size(H, s), S.out_size(W, s), s, trunc_k=k, window=window, align=align)
    a = oracle.render(g, v)
    b = oracle.render(g, v, mode="allpairs")
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-15)


# --------------------------------------------------------------------------
# Half-pixel alignment: HR pixel x samples (x + 1/2)/s - 1/2.
# --------------------------------------------------------------------------
def _dyadic_set(seed, n, lo, hi, W):
    rng = np.random.default_rng(seed)
    d = lambda a: (a * 256).round() / 256
    return (d(rng.uniform(lo, hi, n)), d(rng.uniform(lo, hi, n)), d(rng.uniform(0.3, 1.5, n)),
            d(rng.uniform(0.3, 1.5, n)), rng.uniform(-0.9, 0.9, n), rng.uniform(0, 1, (n, 3)),
            rng.uniform(0, 1, n))


@pytest.mark.parametrize("trunc", [0.0, 3.0])
def test_half_pixel_mirror(trunc):
    """With W_out = s W, mirroring every Gaussian about the LR image centre
    (mu_x -> W - 1 - mu_x, rho -> -rho) mirrors the aligned HR image exactly;
    the literal Eq. 4 sampling does not have this symmetry for s != 1."""
    W = H = 24
    s = 3.0
    mx, my, sx, sy, rho, rgb, al = _dyadic_set(8, 40, 3, 21, W)
    for align, exact in ((S.ALIGN_HALF, True), (S.ALIGN_EQ4, False)):
        v = S.View(H, W, int(s * H), int(s * W), s, trunc_k=trunc, align=align)
        a = oracle.render(one(mx, my, sx, sy, rho, rgb, al), v)
        b = oracle.render(one((W - 1) - mx, my, sx, sy, -rho, rgb, al), v)
        if exact:
            np.testing.assert_allclose(b, a[:, :, ::-1], rtol=1e-12, atol=1e-16)
        else:
            assert np.max(np.abs(b - a[:, :, ::-1])) > 1e-3 * np.max(np.abs(a))


def test_half_pixel_odd_scale_subsampling():
    """For odd integer s the aligned HR pixel s x + (s - 1)/2 samples LR point x,
    so it equals pixel x of the s = 1 render (Eq. 3), windows included."""
    W = H = 16
    mx, my, sx, sy, rho, rgb, al = _dyadic_set(9, 60, 2, 14, W)
    g = one(mx, my, sx, sy, rho, rgb, al)
    base = oracle.render(g, S.View(H, W, H, W, 1.0))
    for s in (3, 5):
        h = (s - 1) // 2
        up = oracle.render(g, S.View(H, W, H * s, W * s, float(s), align=S.ALIGN_HALF))
        np.testing.assert_allclose(up[:, h::s, h::s], base, rtol=1e-13, atol=1e-15)
    one_ = oracle.render(g, S.View(H, W, H, W, 1.0, align=S.ALIGN_HALF))
    np.testing.assert_array_equal(one_, base)


@pytest.mark.parametrize("window,k,align", [(1, 0.08, 0), (0, 3.0, 1), (1, 0.05, 1)])
def test_adjoint_vs_complex_step_flags(window, k, align):
    """The hand adjoint under the ratio window and the half-pixel sampling, against
    complex-step derivatives of the forward with the same frozen windows."""
    g = S.draw_gaussians(6, 14, 18, 1, (0.3, 2.0))
    s = 2.7
    v = S.View(14, 18, S.out_size(14, s), S.out_size(18, s), s, trunc_k=k, window=window,
               align=align)
    go = S.grad_out(2, v.out_h, v.out_w)
    ids = S.sample_indices(3, g.n, 30)
    adj = oracle.adjoint(g, v, go)[ids]
    cs = oracle.complex_step(g, v, go, ids)
    np.testing.assert_allclose(adj, cs, rtol=1e-10, atol=1e-12 * np.abs(cs).max())


# --------------------------------------------------------------------------
# Fused Gaussian head (Sec. 3.2, Gaussian Primary Head): sigmoid for sigma, c,
# alpha; tanh for rho; the offset as predicted (mu = p + o).
# --------------------------------------------------------------------------
HEAD = S.Head(sigma_lo=0.2, sigma_span=2.8, rho_scale=0.9, offset_scale=1.0, offset_tanh=0)


def test_head_float32_sequences_accuracy():
    """The window's float32 exp / sigmoid / tanh against numpy's float64 ones."""
    x = np.linspace(-20, 20, 40001, dtype=np.float32)
    e = oracle.head_f32(x, "exp").astype(np.float64)
    ref = np.exp(x.astype(np.float64))
    assert np.max(np.abs(e - ref) / ref) < 4 * 2.0 ** -23
    s = oracle.head_f32(x, "sigmoid").astype(np.float64)
    assert np.max(np.abs(s - 1 / (1 + np.exp(-x.astype(np.float64))))) < 3e-7
    t = oracle.head_f32(x, "tanh").astype(np.float64)
    assert np.max(np.abs(t - np.tanh(x.astype(np.float64)))) < 3e-7
    assert np.all(np.diff(s) >= 0) and np.all(np.diff(t) >= 0)   # monotone


@pytest.mark.parametrize("head", [HEAD, S.Head(),
                                  S.Head(0.1, 1.5, 0.95, 0.5, offset_tanh=1)])
def test_head_render_equals_physical_render(head):
    """Untruncated (no window decision): the raw render equals the render of the
    physical parameters computed with numpy's own activations."""
    g = S.draw_raw_head(12, 10, 12, 1, head)
    sig = lambda z: 1.0 / (1.0 + np.exp(-z))
    f = lambda a: float(np.float32(a))   # the head's constants are float32 in the ABI
    o = f(head.offset_scale) * (np.tanh(g.offset) if head.offset_tanh else g.offset)
    phys = S.GaussianSet(o, f(head.sigma_lo) + f(head.sigma_span) * sig(g.sigma),
                         f(head.rho_scale) * np.tanh(g.rho), sig(g.rgb), sig(g.alpha),
                         g.lr_h, g.lr_w, 1)
    v = S.View(10, 12, 27, 33, 2.75, trunc_k=0.0)
    np.testing.assert_allclose(oracle.render(g, v), oracle.render(phys, v), rtol=1e-12, atol=1e-15)


def test_head_windows_follow_float32_sequence():
    """Truncated: the head's windows are those of sigma and o taken from the
    float32 sequences (and the render matches the physical render on them)."""
    head = S.Head(0.2, 2.8, 0.9, 1.0, offset_tanh=1)
    g = S.draw_raw_head(13, 10, 12, 4, head)
    s32 = np.float32(head.sigma_lo) + np.float32(head.sigma_span) * oracle.head_f32(g.sigma, "sigmoid").reshape(g.sigma.shape)
    o32 = np.float32(head.offset_scale) * oracle.head_f32(g.offset, "tanh").reshape(g.offset.shape)
    win = S.GaussianSet(o32.astype(np.float64), s32.astype(np.float32).astype(np.float64),
                        np.zeros(g.n), np.ones((g.n, 3)), np.ones(g.n), g.lr_h, g.lr_w, 4)
    v = S.View(10, 12, 30, 36, 3.0)
    assert np.array_equal(oracle.rects(g, v), oracle.rects(win, v))


@pytest.mark.parametrize("head", [HEAD, S.Head(0.1, 1.5, 0.95, 0.5, offset_tanh=1)])
def test_head_adjoint_vs_complex_step_and_fd(head):
    """Gradients with respect to the raw head outputs: hand chain rule against
    complex-step and central differences through the activations."""
    g = S.draw_raw_head(14, 14, 16, 1, head)
    v = S.View(14, 16, S.out_size(14, 2.7), S.out_size(16, 2.7), 2.7)
    go = S.grad_out(3, v.out_h, v.out_w)
    ids = S.sample_indices(4, g.n, 25)
    adj = oracle.adjoint(g, v, go)[ids]
    cs = oracle.complex_step(g, v, go, ids)
    np.testing.assert_allclose(adj, cs, rtol=1e-10, atol=1e-12 * np.abs(cs).max())
    fd = oracle.central_difference(g, v, go, ids[:8], h=1e-5)
    np.testing.assert_allclose(adj[:8], fd, rtol=1e-6, atol=1e-7 * np.abs(fd).max())


def test_thread_count_invariance():
    """The oracle's host threads split the work without changing a bit of the
    result (no race and a fixed summation order), forward and adjoint."""
    gs, vs = S.config1()
    g, v = gs[0], vs[0]
    go = S.grad_out(1, v.out_h, v.out_w)
    ref, ref_a = oracle.render(g, v, threads=1), oracle.adjoint(g, v, go, threads=1)
    for t in (2, 5, 8):
        assert np.array_equal(oracle.render(g, v, threads=t), ref)
        assert np.array_equal(oracle.adjoint(g, v, go, threads=t), ref_a)


@pytest.mark.parametrize("rho", [-0.9, -0.5, 0.3, 0.85])
def test_truncated_mass_correlated(rho):
    """The 3-sigma box of a correlated Gaussian captures the bivariate normal
    probability P(|X| <= 3, |Y| <= 3) at correlation rho (scipy's CDF, an
    independent routine): the box is the marginal extent, not the conditional
    one. That mass lies between 1 - 2 erfc(3/sqrt 2) and 1 - erfc(3/sqrt 2)
    (union bound; the r = 0.1 vs r = 1 argument of the paper's r ablation)."""
    stats = pytest.importorskip("scipy.stats")
    s = 10.0
    g = one(20.03, 19.97, 2.0, 1.6, rho)
    v = S.View(40, 40, 400, 400, s, trunc_k=3.0)
    full = oracle.render(g, S.View(40, 40, 400, 400, s, trunc_k=0.0)).sum(axis=(1, 2))
    frac = oracle.render(g, v).sum(axis=(1, 2)) / full
    r = float(g.rho[0])
    mvn = stats.multivariate_normal(mean=[0.0, 0.0], cov=[[1.0, r], [r, 1.0]])
    expect = float(mvn.cdf([3.0, 3.0], lower_limit=[-3.0, -3.0]))
    tail = math.erfc(3 / math.sqrt(2))
    assert 1 - 2 * tail - 1e-9 <= expect <= 1 - tail + 1e-9
    # the lattice sum's box-edge error is O(f_edge / (s sigma)); here (s sigma >= 16)
    # it stays below 1e-5, far below what a wrong box would change (a box of the
    # conditional extents captures 0.75-0.84 at these rho)
    np.testing.assert_allclose(frac, expect, atol=1e-4)
