"""Randomised pins of the oracle (hypothesis; CPU): for drawn small problems,
any window (3-sigma box or ratio box), alignment, normalisation, reference
grid and scale (including s < 1), the rectangle loop equals the all-pairs
brute force that tests the window inequalities pixel by pixel; the hand
adjoint equals the complex-step derivative of the same forward; the render
is linear in colour and opacity and additive over disjoint sets of Gaussians;
the adjoint is linear in the upstream gradient (the property the row-band
split of one image relies on); and with the fused head (drawn head constants,
raw outputs in) the rectangle loop still equals the brute force and the raw
adjoint the complex step through the activations."""
import numpy as np
import pytest

import gs_synthetic as S
import oracle

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
given, settings = hyp.given, hyp.settings


@st.composite
def problems(draw, absolute=False):
    m = 0 if absolute else draw(st.sampled_from([1, 4, 9]))
    lr_h, lr_w = draw(st.integers(2, 6)), draw(st.integers(2, 6))
    scale = float(np.float32(draw(st.floats(0.6, 5.0))))
    window = draw(st.sampled_from([S.WINDOW_SIGMA, S.WINDOW_RATIO]))
    k = draw(st.sampled_from([3.0, 1.5])) if window == S.WINDOW_SIGMA else \
        draw(st.sampled_from([0.1, 0.25, 0.6]))
    align = draw(st.sampled_from([S.ALIGN_EQ4, S.ALIGN_HALF]))
    norm = draw(st.sampled_from([S.NORM_DENSITY, S.NORM_PEAK]))
    seed = draw(st.integers(0, 2 ** 31 - 1))
    rng = np.random.default_rng(seed)
    n = m * lr_h * lr_w if m else draw(st.integers(1, 12))
    f32 = lambda a: np.asarray(a, np.float64).astype(np.float32).astype(np.float64)
    off = f32(rng.uniform(-0.7, 0.7, (n, 2)) if m else
              rng.uniform(-1.0, 1.0, (n, 2)) * [lr_w, lr_h] + [lr_w / 2, lr_h / 2])
    sig = f32(np.exp(rng.uniform(np.log(0.15), np.log(2.5), (n, 2))))
    rho = f32(rng.uniform(-0.95, 0.95, n))
    rgb = f32(rng.uniform(0, 1, (n, 3)))
    alpha = f32(rng.uniform(0, 1, n))
    g = S.GaussianSet(off, sig, rho, rgb, alpha, lr_h, lr_w, ref_grid_m=m)
    out_h = max(1, S.out_size(lr_h, scale))
    out_w = max(1, S.out_size(lr_w, scale))
    v = S.View(lr_h, lr_w, out_h, out_w, scale, trunc_k=k, norm=norm, window=window, align=align)
    return g, v, rng


def _rel(a, b):
    den = max(float(np.abs(b).max()), 1e-300)
    return float(np.abs(a - b).max()) / den


@settings(max_examples=40, deadline=None)
@given(problems())
def test_rect_loop_equals_brute_force(p):
    g, v, _ = p
    a = oracle.render(g, v, mode="rect", threads=1)
    b = oracle.render(g, v, mode="allpairs", threads=1)
    assert _rel(a, b) < 1e-13


@settings(max_examples=25, deadline=None)
@given(problems())
def test_adjoint_equals_complex_step(p):
    g, v, rng = p
    go = rng.normal(size=(3, v.out_h, v.out_w))
    ids = np.arange(min(g.n, 6))
    adj = oracle.adjoint(g, v, go, threads=1)[ids]
    cs = oracle.complex_step(g, v, go, ids)
    # per field, relative to the field's scale over the checked Gaussians
    for f in range(9):
        den = max(np.abs(cs[:, f]).max(), 1e-12)
        assert np.abs(adj[:, f] - cs[:, f]).max() / den < 1e-9, f


@settings(max_examples=25, deadline=None)
@given(problems(absolute=True))
def test_linear_in_colour_and_additive(p):
    g, v, rng = p
    base = oracle.render(g, v, threads=1)
    # colour and opacity enter linearly
    g2 = S.GaussianSet(g.offset, g.sigma, g.rho, g.rgb * 0.5, g.alpha, g.lr_h, g.lr_w, 0)
    assert _rel(oracle.render(g2, v, threads=1), 0.5 * base) < 1e-14
    g3 = S.GaussianSet(g.offset, g.sigma, g.rho, g.rgb, g.alpha * 0.25, g.lr_h, g.lr_w, 0)
    assert _rel(oracle.render(g3, v, threads=1), 0.25 * base) < 1e-14
    # additive over a split of the set (absolute centres: any split is a valid set)
    if g.n >= 2:
        k = int(rng.integers(1, g.n))
        a = oracle.render(g.subset(np.arange(k)), v, threads=1)
        b = oracle.render(g.subset(np.arange(k, g.n)), v, threads=1)
        assert _rel(a + b, base) < 1e-13


@settings(max_examples=20, deadline=None)
@given(problems())
def test_adjoint_linear_in_upstream_gradient(p):
    g, v, rng = p
    g1 = rng.normal(size=(3, v.out_h, v.out_w))
    g2 = rng.normal(size=(3, v.out_h, v.out_w))
    a = oracle.adjoint(g, v, g1 + 2.0 * g2, threads=1)
    b = oracle.adjoint(g, v, g1, threads=1) + 2.0 * oracle.adjoint(g, v, g2, threads=1)
    assert _rel(a, b) < 1e-12


@st.composite
def head_problems(draw):
    m = draw(st.sampled_from([1, 4]))
    lr_h, lr_w = draw(st.integers(2, 5)), draw(st.integers(2, 5))
    scale = float(np.float32(draw(st.floats(0.8, 4.0))))
    head = S.Head(sigma_lo=float(np.float32(draw(st.floats(0.0, 0.5)))),
                  sigma_span=float(np.float32(draw(st.floats(0.3, 3.0)))),
                  rho_scale=float(np.float32(draw(st.floats(0.0, 0.95)))),
                  offset_scale=float(np.float32(draw(st.floats(0.1, 1.0)))),
                  offset_tanh=draw(st.sampled_from([0, 1])))
    g = S.draw_raw_head(draw(st.integers(0, 2 ** 31 - 1)), lr_h, lr_w, m, head,
                        spread=draw(st.sampled_from([0.5, 1.5, 3.0])))
    window = draw(st.sampled_from([S.WINDOW_SIGMA, S.WINDOW_RATIO]))
    k = 3.0 if window == S.WINDOW_SIGMA else draw(st.sampled_from([0.15, 0.4]))
    v = S.View(lr_h, lr_w, max(1, S.out_size(lr_h, scale)), max(1, S.out_size(lr_w, scale)),
               scale, trunc_k=k, window=window,
               align=draw(st.sampled_from([S.ALIGN_EQ4, S.ALIGN_HALF])),
               norm=draw(st.sampled_from([S.NORM_DENSITY, S.NORM_PEAK])))
    return g, v, np.random.default_rng(draw(st.integers(0, 1000)))


@settings(max_examples=25, deadline=None)
@given(head_problems())
def test_head_rect_loop_and_adjoint(p):
    """With the fused head (raw outputs in, drawn head constants): the rectangle
    loop equals the brute force, and the adjoint with respect to the raw values
    equals the complex-step derivative through the activations."""
    g, v, rng = p
    a = oracle.render(g, v, mode="rect", threads=1)
    b = oracle.render(g, v, mode="allpairs", threads=1)
    assert _rel(a, b) < 1e-13
    go = rng.normal(size=(3, v.out_h, v.out_w))
    ids = np.arange(min(g.n, 5))
    adj = oracle.adjoint(g, v, go, threads=1)[ids]
    cs = oracle.complex_step(g, v, go, ids)
    for f in range(9):
        den = max(np.abs(cs[:, f]).max(), 1e-12)
        assert np.abs(adj[:, f] - cs[:, f]).max() / den < 1e-9, f
