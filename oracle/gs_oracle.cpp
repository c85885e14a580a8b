// FP64 CPU oracle for the scale-aware 2D Gaussian rasterizer of GSASR
// (arXiv 2501.06838). TEST INFRASTRUCTURE ONLY: the tests, the smoke check and
// the benchmark's CPU-baseline leg use it to check and time the CUDA library.
// It shares no code, header or table with the CUDA path, and no product code
// calls it.
//
// What it computes (Sec. 3.1):
//   G_i(x, y)      = alpha_i * c_i * f_i(x, y)                          (Eq. 1)
//   f_i(x, y)      = Z_i * exp(-q_i / 2),
//   q_i            = (u^2/sx^2 - 2 rho u v/(sx sy) + v^2/sy^2) / (1 - rho^2),
//   Z_i            = 1 / (2 pi sx sy sqrt(1 - rho^2))                    (Eq. 2)
//                    (norm = peak: Z_i = 1, c is then the peak colour)
//   I_SR(x, y; s)  = sum_i G_i(x / s, y / s),  u = x/s - mu_x, v = y/s - mu_y
//                                                                        (Eq. 4)
// with the sum restricted, as in Algorithm 1, to the pixels inside a box window
// around each Gaussian. The window is the integer pixel rectangle R_i of either
//   the sigma box  |x - s mu_x| <= s k sx,  |y - s mu_y| <= s k sy  (k = 3), or
//   the ratio box  |x - s mu_x| <  s r W,   |y - s mu_y| <  s r H
// (Algorithm 1's rasterization ratio r, with W, H the LR width and height and
// the HR coordinate compared with the HR centre), whose edges are computed by a
// fixed sequence of float32 operations (documented at `rect_axis_f32`), so that
// the GPU and this oracle take the same integer decision. Everything else is
// FP64.
//
// Pixel alignment: Eq. 4 as printed samples LR point x / s at HR pixel x
// (align = 0). The half-pixel reading samples (x + 1/2) / s - 1/2 (align = 1),
// so that pixel centres, not corners, line up across scales; the HR centre of
// a Gaussian is then s mu + (s - 1)/2.
//
// Centres: with a reference grid of m Gaussians per LR pixel, mu = p + o
// (Sec. 3.2, Gaussian Primary Head), p on an equal-interval sqrt(m) x sqrt(m)
// sub-grid of each LR pixel (Sec. 3.2, Gaussian Embedding). With m = 0 the
// offset array holds mu itself.
//
// Fused Gaussian head (Sec. 3.2, Gaussian Primary Head), optional: the five
// arrays then hold raw head outputs, mapped to the physical parameters by
//   sigma = lo + span * sigmoid(raw), rho = rho_scale * tanh(raw),
//   c = sigmoid(raw), alpha = sigmoid(raw),
//   o = offset_scale * raw  (or offset_scale * tanh(raw)),
// in FP64 for the density and its derivatives. The window, an integer
// decision, takes sigma and o from one fixed sequence of float32 operations
// (exp by Cody-Waite reduction and a Taylor polynomial, see exp_f32), which
// the GPU follows operation for operation.
//
// Adjoint: hand-derived derivatives of the loss L = sum g * I with the windows
// R_i held fixed (the derivative of a moving window edge is not part of it).
// A templated complex-step path differentiates the same forward independently.
//
// Parity: the forward is pinned by closed forms (Poisson-summation sums and
// moments, constant-colour fields, separable truncated sums) and brute force;
// the adjoint by complex step, central differences and torch.autograd.

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <memory>
#include <thread>
#include <vector>

namespace {

struct OView {
  int32_t lr_h, lr_w, out_h, out_w;
  float scale;
  float trunc_k;
  int32_t norm;       // 0 density (Eq. 2 as printed), 1 peak
  int32_t ref_grid_m; // 0 absolute centres, else Gaussians per LR pixel
  int32_t window;     // 0 sigma box (trunc_k = k), 1 ratio box (trunc_k = r)
  int32_t align;      // 0 x / s (Eq. 4 as printed), 1 (x + 1/2) / s - 1/2
};

struct Rect { int32_t x0, x1, y0, y1; };  // inclusive; empty when x0 > x1

struct OHead {
  float sigma_lo, sigma_span, rho_scale, offset_scale;
  int32_t offset_tanh;   // 0: o = offset_scale * raw, 1: o = offset_scale * tanh(raw)
  int32_t pad[3];
};

// e^x in float32 by Cody-Waite range reduction (x = n ln2 + r, ln2 split into
// a 9-bit head and a tail so that n * head is exact) and the degree-7 Taylor
// polynomial of e^r on |r| <= ln2 / 2, each operation one float32 rounding
// (the build disables contraction). Relative error a few ulp.
float exp_f32(float x) {
  const float kL2E = 1.44269502162933349609375f;
  const float kLn2Hi = 0.693359375f;
  const float kLn2Lo = -2.12194441701285541057586669921875e-4f;
  if (x < -87.0f) x = -87.0f;
  if (x > 88.0f) x = 88.0f;
  volatile float t = x * kL2E;
  const float n = std::rint((float)t);
  volatile float a = n * kLn2Hi;
  volatile float b = n * kLn2Lo;
  volatile float r0 = x - a;
  volatile float r = r0 - b;
  const float c[8] = {1.0f, 1.0f, 0.5f, 0.16666667163372039794921875f, 4.1666667908430099487304688e-2f,
                      8.3333337679505348205566406e-3f, 1.3888889225199818611145020e-3f,
                      1.9841270113829523324966431e-4f};
  volatile float p = c[7];
  for (int k = 6; k >= 0; --k) {
    volatile float pr = p * (float)r;
    p = pr + c[k];
  }
  return std::ldexp((float)p, (int)n);
}

float sigmoid_f32(float x) {
  volatile float e = exp_f32(-x);
  volatile float d = 1.0f + e;
  return 1.0f / (float)d;
}

float tanh_f32(float x) {
  const float ax = std::fabs(x);
  volatile float e = exp_f32(-2.0f * ax);
  volatile float num = 1.0f - e;
  volatile float den = 1.0f + e;
  const float t = (float)num / (float)den;
  return x < 0.0f ? -t : t;
}

int isqrt_exact(int m) {
  for (int r = 1; r * r <= m; ++r) if (r * r == m) return r;
  return -1;
}

// Reference position p of Gaussian `gid` on the sub-grid (float32 values):
// gid = ((i * W + j) * m + b * n + a), p = (j + d_a, i + d_b),
// d_a = (2a + 1 - n) / (2n) rounded to float32, then j + d_a rounded to float32.
void ref_pos(int64_t gid, int m, int lr_w, float* px, float* py) {
  int n = isqrt_exact(m);
  int64_t cell = gid / m;
  int sub = (int)(gid % m);
  int64_t i = cell / lr_w, j = cell % lr_w;
  int a = sub % n, b = sub / n;
  volatile float da = (float)((2.0 * a + 1.0 - n) / (2.0 * n));
  volatile float db = (float)((2.0 * b + 1.0 - n) / (2.0 * n));
  volatile float fj = (float)j, fi = (float)i;
  volatile float sx = fj + da;
  volatile float sy = fi + db;
  *px = sx; *py = sy;
}

// The HR centre of one axis in float32: c = s * mu, plus (s - 1)/2 with the
// half-pixel alignment (0.5 s - 0.5 is exact in float32 for s < 2^23).
float hr_centre_f32(float mu, float s, int align) {
  volatile float c = s * mu;
  if (align) {
    volatile float h = 0.5f * s - 0.5f;
    volatile float ch = c + h;
    return ch;
  }
  return c;
}

// One axis of R_i in float32, no contraction (build with -ffp-contract=off),
// c the HR centre from hr_centre_f32:
//   sigma box: r = (s * k) * sigma;  lo = ceil(c - r);      hi = floor(c + r)
//   ratio box: r = (s * ratio) * L;  lo = floor(c - r) + 1; hi = ceil(c + r) - 1
// (L the LR extent of the axis; the ratio box is open, so its integer edges
// are the first integers strictly inside), then lo clamped below at 0, hi
// clamped above at n_out - 1.
void rect_axis_f32(float c, float sigma, float s, float k, int window, int lr_extent, int n_out,
                   int32_t* lo_out, int32_t* hi_out) {
  volatile float sk = s * k;
  volatile float r = window == 0 ? sk * sigma : sk * (float)lr_extent;
  volatile float a = c - r;
  volatile float b = c + r;
  float lo, hi;
  if (window == 0) {
    lo = std::ceil((float)a);
    hi = std::floor((float)b);
  } else {
    lo = std::floor((float)a) + 1.0f;
    hi = std::ceil((float)b) - 1.0f;
  }
  if (!(lo >= 0.0f)) lo = 0.0f;              // also maps NaN to 0
  if (!(hi <= (float)(n_out - 1))) hi = (float)(n_out - 1);
  if (lo > (float)(n_out - 1) || hi < 0.0f || lo > hi) { *lo_out = 1; *hi_out = 0; return; }
  *lo_out = (int32_t)lo; *hi_out = (int32_t)hi;
}

struct Params {
  const double *off, *sig, *rho, *rgb, *alpha;
  int64_t n;
  const double *woff = nullptr, *wsig = nullptr;   // window-defining o, sigma (default: off, sig)
  double woff_at(int64_t k) const { return woff ? woff[k] : off[k]; }
  double wsig_at(int64_t k) const { return wsig ? wsig[k] : sig[k]; }
};

double sigmoid64(double x) { return 1.0 / (1.0 + std::exp(-x)); }

// The physical parameters (FP64) and the window-defining float32 ones of a set
// whose arrays hold raw head outputs.
struct HeadMapped {
  std::vector<double> off, sig, rho, rgb, alpha, woff, wsig;
  HeadMapped(const double* o, const double* sg, const double* rh, const double* c, const double* a,
             int64_t n, const OHead& H)
      : off(2 * n), sig(2 * n), rho(n), rgb(3 * n), alpha(n), woff(2 * n), wsig(2 * n) {
    for (int64_t i = 0; i < n; ++i) {
      for (int k = 0; k < 2; ++k) {
        const double ro = o[2 * i + k], rs = sg[2 * i + k];
        off[2 * i + k] = H.offset_tanh ? (double)H.offset_scale * std::tanh(ro) : (double)H.offset_scale * ro;
        const float o32 = (float)ro;
        volatile float wo = H.offset_tanh ? H.offset_scale * tanh_f32(o32) : H.offset_scale * o32;
        woff[2 * i + k] = (double)(float)wo;
        sig[2 * i + k] = (double)H.sigma_lo + (double)H.sigma_span * sigmoid64(rs);
        volatile float sp = H.sigma_span * sigmoid_f32((float)rs);
        volatile float ws = H.sigma_lo + (float)sp;
        wsig[2 * i + k] = (double)(float)ws;
      }
      rho[i] = (double)H.rho_scale * std::tanh(rh[i]);
      for (int k = 0; k < 3; ++k) rgb[3 * i + k] = sigmoid64(c[3 * i + k]);
      alpha[i] = sigmoid64(a[i]);
    }
  }
  Params params(int64_t n) const {
    Params P{off.data(), sig.data(), rho.data(), rgb.data(), alpha.data(), n};
    P.woff = woff.data();
    P.wsig = wsig.data();
    return P;
  }
};

// d(physical)/d(raw) of the head, per Gaussian and parameter in the gradient
// order (o_x, o_y, sigma_x, sigma_y, rho, r, g, b, alpha).
void head_jacobian(const double* o, const double* sg, const double* rh, const double* c,
                   const double* a, int64_t i, const OHead& H, double* J) {
  for (int k = 0; k < 2; ++k) {
    const double t = std::tanh(o[2 * i + k]);
    J[k] = H.offset_tanh ? (double)H.offset_scale * (1.0 - t * t) : (double)H.offset_scale;
    const double sv = sigmoid64(sg[2 * i + k]);
    J[2 + k] = (double)H.sigma_span * sv * (1.0 - sv);
  }
  const double tr = std::tanh(rh[i]);
  J[4] = (double)H.rho_scale * (1.0 - tr * tr);
  for (int k = 0; k < 3; ++k) {
    const double sc = sigmoid64(c[3 * i + k]);
    J[5 + k] = sc * (1.0 - sc);
  }
  const double sa = sigmoid64(a[i]);
  J[8] = sa * (1.0 - sa);
}

void centre_f32(const Params& P, const OView& V, int64_t i, float* mx, float* my) {
  float ox = (float)P.woff_at(2 * i), oy = (float)P.woff_at(2 * i + 1);
  if (V.ref_grid_m > 0) {
    float px, py;
    ref_pos(i, V.ref_grid_m, V.lr_w, &px, &py);
    volatile float sx = px + ox, sy = py + oy;
    *mx = sx; *my = sy;
  } else {
    *mx = ox; *my = oy;
  }
}

void centre_f64(const Params& P, const OView& V, int64_t i, double* mx, double* my) {
  double px = 0.0, py = 0.0;
  if (V.ref_grid_m > 0) {
    float fx, fy;
    ref_pos(i, V.ref_grid_m, V.lr_w, &fx, &fy);
    px = fx; py = fy;
  }
  *mx = px + P.off[2 * i];
  *my = py + P.off[2 * i + 1];
}

Rect rect_of(const Params& P, const OView& V, int64_t i) {
  Rect R;
  if (!(V.trunc_k > 0.0f)) { R.x0 = 0; R.x1 = V.out_w - 1; R.y0 = 0; R.y1 = V.out_h - 1; return R; }
  float mx, my;
  centre_f32(P, V, i, &mx, &my);
  const float cx = hr_centre_f32(mx, V.scale, V.align), cy = hr_centre_f32(my, V.scale, V.align);
  rect_axis_f32(cx, (float)P.wsig_at(2 * i), V.scale, V.trunc_k, V.window, V.lr_w, V.out_w, &R.x0,
                &R.x1);
  rect_axis_f32(cy, (float)P.wsig_at(2 * i + 1), V.scale, V.trunc_k, V.window, V.lr_h, V.out_h, &R.y0,
                &R.y1);
  return R;
}

// Membership used by the all-pairs mode: the defining inequalities in float32
// with no integer rectangle and no clamping,
//   sigma box: c - s k sigma <= x <= c + s k sigma,
//   ratio box: c - s r L < x < c + s r L.
bool inside_f32(const Params& P, const OView& V, int64_t i, int x, int y) {
  if (!(V.trunc_k > 0.0f)) return true;
  float mx, my;
  centre_f32(P, V, i, &mx, &my);
  float s = V.scale, k = V.trunc_k;
  volatile float cx = hr_centre_f32(mx, s, V.align), cy = hr_centre_f32(my, s, V.align);
  volatile float sk = s * k;
  volatile float rx = V.window == 0 ? sk * (float)P.wsig_at(2 * i) : sk * (float)V.lr_w;
  volatile float ry = V.window == 0 ? sk * (float)P.wsig_at(2 * i + 1) : sk * (float)V.lr_h;
  volatile float ax = cx - rx, bx = cx + rx, ay = cy - ry, by = cy + ry;
  float fx = (float)x, fy = (float)y;
  if (V.window == 0) return fx >= ax && fx <= bx && fy >= ay && fy <= by;
  return fx > ax && fx < bx && fy > ay && fy < by;
}

// The LR coordinate that HR pixel x samples (Eq. 4; half-pixel reading when
// align = 1).
double sample_lr(int x, double s, int align) {
  return align ? ((double)x + 0.5) / s - 0.5 : (double)x / s;
}

// The Gaussian's physical parameters as a scalar type T (double or complex).
template <class T> struct GaussT {
  T mx, my, sx, sy, rho, c[3], alpha;
};

template <class T> GaussT<T> gauss_of(const Params& P, const OView& V, int64_t i) {
  GaussT<T> g;
  double mx, my;
  centre_f64(P, V, i, &mx, &my);
  g.mx = mx; g.my = my;
  g.sx = P.sig[2 * i]; g.sy = P.sig[2 * i + 1];
  g.rho = P.rho[i];
  for (int k = 0; k < 3; ++k) g.c[k] = P.rgb[3 * i + k];
  g.alpha = P.alpha[i];
  return g;
}

// f(x/s, y/s) of Eq. 2 for one Gaussian.
template <class T> T density(const GaussT<T>& g, double s, int norm, int align, int x, int y) {
  const double kPi = 3.14159265358979323846;
  T u = sample_lr(x, s, align) - g.mx;
  T v = sample_lr(y, s, align) - g.my;
  T D = (1.0 - g.rho) * (1.0 + g.rho);
  T q = (u * u / (g.sx * g.sx) - 2.0 * g.rho * u * v / (g.sx * g.sy) + v * v / (g.sy * g.sy)) / D;
  T Z = norm == 0 ? T(1.0) / (2.0 * kPi * g.sx * g.sy * std::sqrt(D)) : T(1.0);
  return Z * std::exp(-0.5 * q);
}

int resolve_threads(int threads) {
  if (threads > 0) return threads;
  unsigned h = std::thread::hardware_concurrency();
  return h ? (int)h : 1;
}

template <class F> void parallel_for(int64_t n, int threads, F&& fn) {
  threads = (int)std::min<int64_t>(std::max(1, threads), std::max<int64_t>(1, n));
  if (threads <= 1) { fn(0, n, 0); return; }
  std::vector<std::thread> pool;
  int64_t chunk = (n + threads - 1) / threads;
  for (int t = 0; t < threads; ++t) {
    int64_t b = t * chunk, e = std::min(n, b + chunk);
    if (b >= e) break;
    pool.emplace_back([&, b, e, t] { fn(b, e, t); });
  }
  for (auto& th : pool) th.join();
}

bool valid_view(const OView* V) {
  if (!V) return false;
  if (V->out_h <= 0 || V->out_w <= 0 || V->lr_h <= 0 || V->lr_w <= 0) return false;
  if (!(V->scale > 0.0f) || !std::isfinite(V->scale)) return false;
  if (V->ref_grid_m < 0 || (V->ref_grid_m > 0 && isqrt_exact(V->ref_grid_m) < 0)) return false;
  if (V->window != 0 && V->window != 1) return false;
  if (V->align != 0 && V->align != 1) return false;
  return true;
}

// Params over either physical arrays or raw head outputs (then mapped).
struct ParamSet {
  std::unique_ptr<HeadMapped> hm;
  Params P;
  ParamSet(const double* off, const double* sig, const double* rho, const double* rgb,
           const double* alpha, int64_t n, const OHead* head)
      : P{off, sig, rho, rgb, alpha, n} {
    if (head) {
      hm.reset(new HeadMapped(off, sig, rho, rgb, alpha, n, *head));
      P = hm->params(n);
    }
  }
};

bool valid_head(const OHead* H) {
  return !H || (H->sigma_span > 0.0f && H->sigma_lo >= 0.0f && std::fabs(H->rho_scale) <= 1.0f &&
                (H->offset_tanh == 0 || H->offset_tanh == 1));
}

}  // namespace

extern "C" {

// Integer rectangles R_i, [n][4] = (x0, x1, y0, y1), inclusive (empty: x0 > x1).
int gso_rects(const double* off, const double* sig, const double* rho, const double* rgb,
              const double* alpha, int64_t n, const OView* V, const OHead* head, int32_t* rects) {
  if (!valid_view(V) || !valid_head(head)) return 1;
  ParamSet PS(off, sig, rho, rgb, alpha, n, head);
  const Params& P = PS.P;
  for (int64_t i = 0; i < n; ++i) {
    Rect R = rect_of(P, *V, i);
    rects[4 * i] = R.x0; rects[4 * i + 1] = R.x1; rects[4 * i + 2] = R.y0; rects[4 * i + 3] = R.y1;
  }
  return 0;
}

// Forward render into out[3][out_h][out_w] (overwritten).
// mode 0: loop each Gaussian over its rectangle (Algorithm 1's loop order),
//         rows of the output split into bands across threads;
// mode 1: all pairs: every pixel against every Gaussian, float32 membership test.
// rects_in (optional, [n][4]) overrides R_i (frozen windows for derivative tests).
int gso_render(const double* off, const double* sig, const double* rho, const double* rgb,
               const double* alpha, int64_t n, const OView* V, const OHead* head, int mode,
               int threads, const int32_t* rects_in, double* out) {
  if (!valid_view(V) || !valid_head(head)) return 1;
  ParamSet PS(off, sig, rho, rgb, alpha, n, head);
  const Params& P = PS.P;
  const OView v = *V;
  const int64_t H = v.out_h, W = v.out_w;
  std::memset(out, 0, sizeof(double) * 3 * H * W);
  threads = resolve_threads(threads);
  const double s = (double)v.scale;
  if (mode == 1) {
    parallel_for(H, threads, [&](int64_t y0, int64_t y1, int) {
      for (int64_t y = y0; y < y1; ++y)
        for (int64_t x = 0; x < W; ++x)
          for (int64_t i = 0; i < n; ++i) {
            if (!inside_f32(P, v, i, (int)x, (int)y)) continue;
            GaussT<double> g = gauss_of<double>(P, v, i);
            double f = density(g, s, v.norm, v.align, (int)x, (int)y);
            for (int k = 0; k < 3; ++k) out[(k * H + y) * W + x] += g.alpha * g.c[k] * f;
          }
    });
    return 0;
  }
  std::vector<Rect> R(n);
  parallel_for(n, threads, [&](int64_t b, int64_t e, int) {
    for (int64_t i = b; i < e; ++i) {
      if (rects_in) R[i] = Rect{rects_in[4 * i], rects_in[4 * i + 1], rects_in[4 * i + 2], rects_in[4 * i + 3]};
      else R[i] = rect_of(P, v, i);
    }
  });
  parallel_for(H, threads, [&](int64_t yb, int64_t ye, int) {
    for (int64_t i = 0; i < n; ++i) {
      const Rect& r = R[i];
      int64_t ylo = std::max<int64_t>(r.y0, yb), yhi = std::min<int64_t>(r.y1, ye - 1);
      if (r.x0 > r.x1 || ylo > yhi) continue;
      GaussT<double> g = gauss_of<double>(P, v, i);
      for (int64_t y = ylo; y <= yhi; ++y)
        for (int64_t x = r.x0; x <= r.x1; ++x) {
          double f = density(g, s, v.norm, v.align, (int)x, (int)y);
          for (int k = 0; k < 3; ++k) out[(k * H + y) * W + x] += g.alpha * g.c[k] * f;
        }
    }
  });
  return 0;
}

// Hand adjoint of L = sum_{k,y,x} grad_out[k,y,x] * I[k,y,x] with frozen R_i.
// grads[n][9] = dL/d(o_x, o_y, sigma_x, sigma_y, rho, r, g, b, alpha).
//   per pixel: G = sum_k g_k c_k, f = Z exp(-q/2)
//   dc_k += g_k alpha f;  dalpha += G f;
//   dtheta += G alpha f (dlogZ/dtheta - dq/dtheta / 2)
//   dq/dmu_x = -(2u/sx^2 - 2 rho v/(sx sy)) / D
//   dq/dmu_y = -(2v/sy^2 - 2 rho u/(sx sy)) / D
//   dq/dsx   = -(2u^2/sx^3 - 2 rho u v/(sx^2 sy)) / D
//   dq/dsy   = -(2v^2/sy^3 - 2 rho u v/(sx sy^2)) / D
//   dq/drho  = (-2uv/(sx sy) + 2 rho q) / D
//   density: dlogZ/dsx = -1/sx, dlogZ/dsy = -1/sy, dlogZ/drho = rho/D; peak: 0.
//   mu = p + o, so dL/do = dL/dmu.
int gso_adjoint(const double* off, const double* sig, const double* rho, const double* rgb,
                const double* alpha, int64_t n, const OView* V, const OHead* head,
                const double* grad_out, int threads, const int32_t* rects_in, double* grads) {
  if (!valid_view(V) || !valid_head(head)) return 1;
  ParamSet PS(off, sig, rho, rgb, alpha, n, head);
  const Params& P = PS.P;
  const OView v = *V;
  const int64_t H = v.out_h, W = v.out_w;
  const double s = (double)v.scale;
  const double kPi = 3.14159265358979323846;
  threads = resolve_threads(threads);
  parallel_for(n, threads, [&](int64_t b, int64_t e, int) {
    for (int64_t i = b; i < e; ++i) {
      Rect r = rects_in ? Rect{rects_in[4 * i], rects_in[4 * i + 1], rects_in[4 * i + 2], rects_in[4 * i + 3]}
                        : rect_of(P, v, i);
      double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
      GaussT<double> g = gauss_of<double>(P, v, i);
      const double sx = g.sx, sy = g.sy, rh = g.rho;
      const double D = (1.0 - rh) * (1.0 + rh);
      const double Z = v.norm == 0 ? 1.0 / (2.0 * kPi * sx * sy * std::sqrt(D)) : 1.0;
      const double dlz_sx = v.norm == 0 ? -1.0 / sx : 0.0;
      const double dlz_sy = v.norm == 0 ? -1.0 / sy : 0.0;
      const double dlz_rh = v.norm == 0 ? rh / D : 0.0;
      if (r.x0 <= r.x1 && r.y0 <= r.y1) {
        for (int64_t y = r.y0; y <= r.y1; ++y)
          for (int64_t x = r.x0; x <= r.x1; ++x) {
            const double u = sample_lr((int)x, s, v.align) - g.mx;
            const double w = sample_lr((int)y, s, v.align) - g.my;
            const double q = (u * u / (sx * sx) - 2.0 * rh * u * w / (sx * sy) + w * w / (sy * sy)) / D;
            const double f = Z * std::exp(-0.5 * q);
            double gk[3], G = 0.0;
            for (int k = 0; k < 3; ++k) { gk[k] = grad_out[(k * H + y) * W + x]; G += gk[k] * g.c[k]; }
            const double dq_mx = -(2.0 * u / (sx * sx) - 2.0 * rh * w / (sx * sy)) / D;
            const double dq_my = -(2.0 * w / (sy * sy) - 2.0 * rh * u / (sx * sy)) / D;
            const double dq_sx = -(2.0 * u * u / (sx * sx * sx) - 2.0 * rh * u * w / (sx * sx * sy)) / D;
            const double dq_sy = -(2.0 * w * w / (sy * sy * sy) - 2.0 * rh * u * w / (sx * sy * sy)) / D;
            const double dq_rh = (-2.0 * u * w / (sx * sy) + 2.0 * rh * q) / D;
            const double Gaf = G * g.alpha * f;
            acc[0] += Gaf * (-0.5 * dq_mx);
            acc[1] += Gaf * (-0.5 * dq_my);
            acc[2] += Gaf * (dlz_sx - 0.5 * dq_sx);
            acc[3] += Gaf * (dlz_sy - 0.5 * dq_sy);
            acc[4] += Gaf * (dlz_rh - 0.5 * dq_rh);
            for (int k = 0; k < 3; ++k) acc[5 + k] += gk[k] * g.alpha * f;
            acc[8] += G * f;
          }
      }
      if (head) {   // chain rule through the head's activations
        double J[9];
        head_jacobian(off, sig, rho, rgb, alpha, i, *head, J);
        for (int k = 0; k < 9; ++k) acc[k] *= J[k];
      }
      for (int k = 0; k < 9; ++k) grads[9 * i + k] = acc[k];
    }
  });
  return 0;
}

// Complex-step derivatives of the same loss for the Gaussians listed in gids:
// dL/dtheta = Im(L(theta + i h)) / h, evaluated with the forward's own formula
// (templated on std::complex<double>) and the frozen windows. grads[k][9].
int gso_complex_step(const double* off, const double* sig, const double* rho, const double* rgb,
                     const double* alpha, int64_t n, const OView* V, const OHead* head,
                     const double* grad_out, const int64_t* gids, int64_t k, double h,
                     double* grads) {
  if (!valid_view(V) || !valid_head(head)) return 1;
  ParamSet PS(off, sig, rho, rgb, alpha, n, head);
  const Params& P = PS.P;
  const OView v = *V;
  const int64_t H = v.out_h, W = v.out_w;
  const double s = (double)v.scale;
  typedef std::complex<double> C;
  auto csig = [](C z) { return 1.0 / (1.0 + std::exp(-z)); };
  for (int64_t t = 0; t < k; ++t) {
    const int64_t i = gids[t];
    if (i < 0 || i >= n) return 2;
    Rect r = rect_of(P, v, i);
    GaussT<double> g0 = gauss_of<double>(P, v, i);
    for (int p = 0; p < 9; ++p) {
      GaussT<C> g;
      g.mx = g0.mx; g.my = g0.my; g.sx = g0.sx; g.sy = g0.sy; g.rho = g0.rho;
      for (int c = 0; c < 3; ++c) g.c[c] = g0.c[c];
      g.alpha = g0.alpha;
      const C ih(0.0, h);
      if (head) {   // perturb the raw head output and map it through the activations
        const OHead& Hd = *head;
        double px = 0.0, py = 0.0;
        if (v.ref_grid_m > 0) {
          float fx, fy;
          ref_pos(i, v.ref_grid_m, v.lr_w, &fx, &fy);
          px = fx; py = fy;
        }
        auto offm = [&](C z) { return Hd.offset_tanh ? (double)Hd.offset_scale * std::tanh(z)
                                                     : (double)Hd.offset_scale * z; };
        switch (p) {
          case 0: g.mx = px + offm(C(off[2 * i], 0.0) + ih); break;
          case 1: g.my = py + offm(C(off[2 * i + 1], 0.0) + ih); break;
          case 2: g.sx = (double)Hd.sigma_lo + (double)Hd.sigma_span * csig(C(sig[2 * i], 0.0) + ih); break;
          case 3: g.sy = (double)Hd.sigma_lo + (double)Hd.sigma_span * csig(C(sig[2 * i + 1], 0.0) + ih); break;
          case 4: g.rho = (double)Hd.rho_scale * std::tanh(C(rho[i], 0.0) + ih); break;
          case 5: case 6: case 7: g.c[p - 5] = csig(C(rgb[3 * i + p - 5], 0.0) + ih); break;
          default: g.alpha = csig(C(alpha[i], 0.0) + ih); break;
        }
      } else switch (p) {
        case 0: g.mx += ih; break;
        case 1: g.my += ih; break;
        case 2: g.sx += ih; break;
        case 3: g.sy += ih; break;
        case 4: g.rho += ih; break;
        case 5: g.c[0] += ih; break;
        case 6: g.c[1] += ih; break;
        case 7: g.c[2] += ih; break;
        default: g.alpha += ih; break;
      }
      C L(0.0, 0.0);
      if (r.x0 <= r.x1 && r.y0 <= r.y1)
        for (int64_t y = r.y0; y <= r.y1; ++y)
          for (int64_t x = r.x0; x <= r.x1; ++x) {
            C f = density(g, s, v.norm, v.align, (int)x, (int)y);
            for (int c = 0; c < 3; ++c) L += grad_out[(c * H + y) * W + x] * (g.alpha * g.c[c] * f);
          }
      grads[9 * t + p] = L.imag() / h;
    }
  }
  return 0;
}

// One Gaussian's share of the loss, L_i = sum_{(x,y) in R_i} g(x,y) . G_i(x/s, y/s),
// with its 9 parameters replaced by theta = (mu_x, mu_y, sigma_x, sigma_y, rho,
// r, g, b, alpha) and R_i computed from the UNPERTURBED inputs (frozen window).
// With a head, theta holds the raw head outputs (o_x, o_y, then the raw values
// of sigma_x, sigma_y, rho, r, g, b, alpha), mapped through the activations.
// Central differences of this function check the adjoint.
double gso_gaussian_loss(const double* off, const double* sig, const double* rho, const double* rgb,
                         const double* alpha, int64_t n, const OView* V, const OHead* head,
                         const double* grad_out, int64_t gid, const double* theta) {
  if (!valid_view(V) || !valid_head(head) || gid < 0 || gid >= n) return NAN;
  ParamSet PS(off, sig, rho, rgb, alpha, n, head);
  const Params& P = PS.P;
  const OView v = *V;
  const int64_t H = v.out_h, W = v.out_w;
  Rect r = rect_of(P, v, gid);
  GaussT<double> g;
  if (head) {
    const OHead& Hd = *head;
    double px = 0.0, py = 0.0;
    if (v.ref_grid_m > 0) {
      float fx, fy;
      ref_pos(gid, v.ref_grid_m, v.lr_w, &fx, &fy);
      px = fx; py = fy;
    }
    auto offm = [&](double z) { return Hd.offset_tanh ? (double)Hd.offset_scale * std::tanh(z)
                                                      : (double)Hd.offset_scale * z; };
    g.mx = px + offm(theta[0]);
    g.my = py + offm(theta[1]);
    g.sx = (double)Hd.sigma_lo + (double)Hd.sigma_span * sigmoid64(theta[2]);
    g.sy = (double)Hd.sigma_lo + (double)Hd.sigma_span * sigmoid64(theta[3]);
    g.rho = (double)Hd.rho_scale * std::tanh(theta[4]);
    for (int c = 0; c < 3; ++c) g.c[c] = sigmoid64(theta[5 + c]);
    g.alpha = sigmoid64(theta[8]);
  } else {
    g.mx = theta[0]; g.my = theta[1]; g.sx = theta[2]; g.sy = theta[3]; g.rho = theta[4];
    for (int c = 0; c < 3; ++c) g.c[c] = theta[5 + c];
    g.alpha = theta[8];
  }
  double L = 0.0;
  if (r.x0 <= r.x1 && r.y0 <= r.y1)
    for (int64_t y = r.y0; y <= r.y1; ++y)
      for (int64_t x = r.x0; x <= r.x1; ++x) {
        double f = density(g, (double)v.scale, v.norm, v.align, (int)x, (int)y);
        for (int c = 0; c < 3; ++c) L += grad_out[(c * H + y) * W + x] * (g.alpha * g.c[c] * f);
      }
  return L;
}

// The FP64 centre mu = p + o of Gaussian gid (p from the reference grid; with a
// head, o from the raw offset).
int gso_centre(const double* off, int64_t n, const OView* V, const OHead* head, int64_t gid,
               double* mu) {
  if (!valid_view(V) || !valid_head(head) || gid < 0 || gid >= n) return 1;
  double o[2] = {off[2 * gid], off[2 * gid + 1]};
  if (head)
    for (int k = 0; k < 2; ++k)
      o[k] = head->offset_tanh ? (double)head->offset_scale * std::tanh(o[k]) : (double)head->offset_scale * o[k];
  double px = 0.0, py = 0.0;
  if (V->ref_grid_m > 0) {
    float fx, fy;
    ref_pos(gid, V->ref_grid_m, V->lr_w, &fx, &fy);
    px = fx; py = fy;
  }
  mu[0] = px + o[0];
  mu[1] = py + o[1];
  return 0;
}

// The window-defining float32 head activations of raw values x[n] (test hook
// for the fixed float32 sequence): kind 0 sigmoid_f32, 1 tanh_f32, 2 exp_f32.
int gso_head_f32(const float* x, int64_t n, int kind, float* y) {
  for (int64_t i = 0; i < n; ++i)
    y[i] = kind == 0 ? sigmoid_f32(x[i]) : kind == 1 ? tanh_f32(x[i]) : exp_f32(x[i]);
  return 0;
}

int gso_hardware_threads(void) { return resolve_threads(0); }

}  // extern "C"
