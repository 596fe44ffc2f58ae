// Sec. VI: iteration-scheduled macro charge densities and their bin
// integrals, GPU-side.  For iteration t of a schedule of T iterations, each
// macro m carries a charge density rho_t over its footprint (local offsets
// dx, dy from its centre, zero outside the w x h rectangle):
//   charge redistribution:  rho = 2 eta^2 / (pi erf^2(eta / sqrt 2))
//                                 exp(-2 eta^2 (dx^2 / w^2 + dy^2 / h^2)),
//     eta(t) = eta_B(a)^(1 - s(a)) eta_A(a)^s(a), a = t / T, scheme A
//     eta_A = sqrt(-2 log r(a)) with log r log-linear from r0 to r1, scheme B
//     eta_B = sqrt(2 ln 2) / beta(a) with beta linear from beta_min to
//     beta_max, s the smoothstep between alpha0 and alpha1;
//   charge restoration, exponential-like:  rho = exp(-(tan^2(pi dx / w) +
//     tan^2(pi dy / h)) / (2 sigma^2)), sigma(t) = -sigma_factor T ln(1 - t / T);
//   linear-like:  rho = max(0, 1 - k rr);  sigmoid-like:  rho = 2 / (1 + exp(k rr)),
//     rr = sqrt(2 (dx^2 / w^2 + dy^2 / h^2)), k(t) = k_factor / tan(pi t / (2 T)).
// The density of bin b gains the integral of rho_t over the bin (area units).
// Gaussian: the separable closed form with erf; exponential-like: separable,
// a composite Gauss-Legendre rule per axis; linear- and sigmoid-like: the
// tensor rule on the bin-macro intersection.  FP64, except the radial models'
// point values and their sums within a panel (FP32, about 1e-7 relative; the
// FP64 rate of GB300 would otherwise set the kernel's time).
//
// A warp per tile of 8 x 4 bins, a lane per bin: the lanes test 32 macros at
// a time against the tile, and each lane adds the integrals of the macros
// overlapping its bin in ascending order.
#include <cmath>

#include "pl_internal.h"

namespace pl {

constexpr int kRhoMaxNodes = 32;

struct RhoArgs {
  int model, panels, nodes;
  double A, c;       // Gaussian: normalization and sqrt(2) eta
  double sscale;     // exponential-like: 1 / (2 sigma^2); < 0: sigma infinite
  int szero;         // exponential-like: sigma = 0 (no charge)
  double k;          // linear- and sigmoid-like; < 0: k infinite (no charge)
  double gx[kRhoMaxNodes], gw[kRhoMaxNodes];  // Gauss-Legendre rule on [-1, 1]
};

// Composite rule of f over [a, b] (one thread).
template <typename F>
__device__ double gl_1d(const RhoArgs &R, double a, double b, F f) {
  const double hp = (b - a) / R.panels;
  double s = 0.0;
  for (int p = 0; p < R.panels; ++p) {
    const double c = a + (p + 0.5) * hp;
    for (int i = 0; i < R.nodes; ++i) s += 0.5 * hp * R.gw[i] * f(c + 0.5 * hp * R.gx[i]);
  }
  return s;
}

// Integral of rho over [ax, bx] x [ay, by] (offsets, already inside the
// macro), one thread.
__device__ double rho_integral(const RhoArgs &R, double w, double h, double ax, double bx,
                               double ay, double by) {
  if (R.model == PL_RHO_GAUSS) {
    const double ix = w * sqrt(M_PI) / (2.0 * R.c) * (erf(R.c * bx / w) - erf(R.c * ax / w));
    const double iy = h * sqrt(M_PI) / (2.0 * R.c) * (erf(R.c * by / h) - erf(R.c * ay / h));
    return R.A * ix * iy;
  }
  if (R.model == PL_RHO_EXP) {
    if (R.szero) return 0.0;
    if (R.sscale < 0.0) return (bx - ax) * (by - ay);
    auto fx = [&](double d) {
      const double tv = tan(M_PI * d / w);
      return exp(-tv * tv * R.sscale);
    };
    auto fy = [&](double d) {
      const double tv = tan(M_PI * d / h);
      return exp(-tv * tv * R.sscale);
    };
    return gl_1d(R, ax, bx, fx) * gl_1d(R, ay, by, fy);
  }
  if (R.k < 0.0) return 0.0;
  // a panel's nodes x nodes points summed in FP32 (weights and values to
  // about 1e-7 relative), the panels in FP64
  const double hx = (bx - ax) / R.panels, hy = (by - ay) / R.panels;
  const float kf = (float)R.k;
  double s = 0.0;
  for (int px = 0; px < R.panels; ++px)
    for (int py = 0; py < R.panels; ++py) {
      const float cu = (float)((ax + (px + 0.5) * hx) / w), cv = (float)((ay + (py + 0.5) * hy) / h);
      const float du = (float)(0.5 * hx / w), dv = (float)(0.5 * hy / h);
      float ps = 0.f;
      for (int i = 0; i < R.nodes; ++i) {
        const float u = cu + du * (float)R.gx[i];
        float row = 0.f;
        for (int j = 0; j < R.nodes; ++j) {
          const float v = cv + dv * (float)R.gx[j];
          const float rr = sqrtf(2.0f * (u * u + v * v));
          const float val = R.model == PL_RHO_LINEAR ? fmaxf(0.0f, 1.0f - kf * rr)
                                                     : 2.0f / (1.0f + __expf(kf * rr));
          row = fmaf((float)R.gw[j], val, row);
        }
        ps = fmaf((float)R.gw[i], row, ps);
      }
      s += 0.25 * hx * hy * (double)ps;
    }
  return s;
}

// A warp per tile of 8 x 4 bins, a lane per bin.  The lanes test 32 macros
// at a time against the tile; for each macro that overlaps it, every lane
// whose bin the macro overlaps adds that macro's integral over its bin, so
// each bin adds its macros in ascending order.
constexpr int kTileX = 8, kTileY = 4;
__global__ void __launch_bounds__(256) k_macro_density(RhoArgs R, int32_t nm, const float *mx,
                                                       const float *my, const float *mw,
                                                       const float *mh, double xl, double yl,
                                                       double wb, double hb, int nbx, int nby,
                                                       double *out) {
  const int lane = threadIdx.x & 31;
  const int ntx = (nbx + kTileX - 1) / kTileX, nty = (nby + kTileY - 1) / kTileY;
  const long long ntile = (long long)ntx * nty;
  for (long long tl = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; tl < ntile;
       tl += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int tx = (int)(tl % ntx), ty = (int)(tl / ntx);
    const int bx = tx * kTileX + (lane % kTileX), by = ty * kTileY + (lane / kTileX);
    const bool mine = bx < nbx && by < nby;
    const double x0 = xl + bx * wb, x1 = xl + (bx + 1) * wb;
    const double y0 = yl + by * hb, y1 = yl + (by + 1) * hb;
    // the tile's extent
    const double tx0 = xl + tx * kTileX * wb, tx1 = xl + min((tx + 1) * kTileX, nbx) * wb;
    const double ty0 = yl + ty * kTileY * hb, ty1 = yl + min((ty + 1) * kTileY, nby) * hb;
    double acc = 0.0;
    for (int m0 = 0; m0 < nm; m0 += 32) {
      const int m = m0 + lane;
      double cx = 0.0, cy = 0.0, w = 0.0, h = 0.0;
      bool ov = false;
      if (m < nm) {
        cx = mx[m];
        cy = my[m];
        w = mw[m];
        h = mh[m];
        ov = w > 0.0 && h > 0.0 && fmax(tx0, cx - 0.5 * w) < fmin(tx1, cx + 0.5 * w) &&
             fmax(ty0, cy - 0.5 * h) < fmin(ty1, cy + 0.5 * h);
      }
      unsigned bal = __ballot_sync(0xffffffffu, ov);
      while (bal) {
        const int src = __ffs(bal) - 1;
        bal &= bal - 1;
        const double scx = __shfl_sync(0xffffffffu, cx, src), scy = __shfl_sync(0xffffffffu, cy, src);
        const double sw = __shfl_sync(0xffffffffu, w, src), sh = __shfl_sync(0xffffffffu, h, src);
        const double ax = fmax(x0 - scx, -0.5 * sw), bx2 = fmin(x1 - scx, 0.5 * sw);
        const double ay = fmax(y0 - scy, -0.5 * sh), by2 = fmin(y1 - scy, 0.5 * sh);
        if (mine && ax < bx2 && ay < by2) acc += rho_integral(R, sw, sh, ax, bx2, ay, by2);
      }
    }
    if (mine) out[(long long)by * nbx + bx] = acc;
  }
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton's method on P_n from
// the guesses cos(pi (i - 1/4) / (n + 1/2)); P_n' from the recurrence).
static void legendre_rule(int n, double *x, double *w) {
  for (int i = 1; i <= n; ++i) {
    double z = std::cos(M_PI * (i - 0.25) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i - 1] = -z;
    w[i - 1] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

}  // namespace pl

extern "C" {

void pl_rho_params_default(pl_rho_params *p) {
  if (!p) return;
  p->model = PL_RHO_GAUSS;
  p->T = 300;
  p->r0 = 0.05;
  p->r1 = 0.9;
  p->beta_min = 0.25;
  p->beta_max = 1.5;
  p->alpha0 = 0.3;
  p->alpha1 = 0.7;
  p->sigma_factor = 0.002;
  p->k_factor = 0.5;
  p->panels = 4;
  p->nodes = 8;
}

pl_status pl_macro_density(const pl_rho_params *rp, int32_t t, int32_t num_macros,
                           const float *mx, const float *my, const float *mw, const float *mh,
                           double xl, double yl, double xh, double yh, int32_t nbx, int32_t nby,
                           double *rho, pl_stream stream) {
  using namespace pl;
  clear_error();
  if (!rp || !rho || num_macros < 0 || (num_macros && (!mx || !my || !mw || !mh))) {
    set_error("NULL or negative argument");
    return PL_ERR_INVALID_ARG;
  }
  if (nbx < 1 || nby < 1 || !(xh > xl) || !(yh > yl) || !std::isfinite(xl) || !std::isfinite(xh) ||
      !std::isfinite(yl) || !std::isfinite(yh)) {
    set_error("bad bin grid or region");
    return PL_ERR_INVALID_ARG;
  }
  if (rp->model < PL_RHO_GAUSS || rp->model > PL_RHO_SIGMOID || rp->T < 1 || t < 0 || t > rp->T ||
      rp->panels < 1 || rp->panels > 64 || rp->nodes < 1 || rp->nodes > kRhoMaxNodes) {
    set_error("bad schedule parameters (model, T >= 1, 0 <= t <= T, panels 1..64, nodes 1..32)");
    return PL_ERR_INVALID_ARG;
  }
  RhoArgs R{};
  R.model = rp->model;
  R.panels = rp->panels;
  R.nodes = rp->nodes;
  legendre_rule(rp->nodes, R.gx, R.gw);
  const double a = (double)t / (double)rp->T;
  if (rp->model == PL_RHO_GAUSS) {
    if (!(rp->r0 > 0.0 && rp->r0 < 1.0 && rp->r1 > 0.0 && rp->r1 < 1.0 && rp->beta_min > 0.0 &&
          rp->beta_max > 0.0 && rp->alpha1 > rp->alpha0)) {
      set_error("Gaussian schedule needs 0 < r0, r1 < 1, beta > 0, alpha1 > alpha0");
      return PL_ERR_INVALID_ARG;
    }
    const double ea = std::sqrt(-2.0 * ((1.0 - a) * std::log(rp->r0) + a * std::log(rp->r1)));
    const double eb = std::sqrt(2.0 * std::log(2.0)) / (rp->beta_min + (rp->beta_max - rp->beta_min) * a);
    double s = 0.0;
    if (a >= rp->alpha1) s = 1.0;
    else if (a > rp->alpha0) {
      const double z = (a - rp->alpha0) / (rp->alpha1 - rp->alpha0);
      s = 3.0 * z * z - 2.0 * z * z * z;
    }
    const double eta = std::pow(eb, 1.0 - s) * std::pow(ea, s);
    const double e = std::erf(eta / std::sqrt(2.0));
    R.A = 2.0 * eta * eta / (M_PI * e * e);
    R.c = std::sqrt(2.0) * eta;
  } else if (rp->model == PL_RHO_EXP) {
    if (!(rp->sigma_factor > 0.0)) {
      set_error("sigma_factor must be > 0");
      return PL_ERR_INVALID_ARG;
    }
    R.szero = t == 0;
    R.sscale = -1.0;
    if (t > 0 && t < rp->T) {
      const double sg = -rp->sigma_factor * rp->T * std::log(1.0 - a);
      R.sscale = 1.0 / (2.0 * sg * sg);
    }
  } else {
    if (!(rp->k_factor > 0.0)) {
      set_error("k_factor must be > 0");
      return PL_ERR_INVALID_ARG;
    }
    R.k = t == 0 ? -1.0 : (t >= rp->T ? 0.0 : rp->k_factor / std::tan(0.5 * M_PI * a));
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const long long ntile = (long long)((nbx + kTileX - 1) / kTileX) * ((nby + kTileY - 1) / kTileY);
  k_macro_density<<<grid_for(ntile * 32, 256, 152 * 16), 256, 0, s>>>(
      R, num_macros, mx, my, mw, mh, xl, yl, (xh - xl) / nbx, (yh - yl) / nby, nbx, nby, rho);
  note_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PL_OK : cuda_fail(e, "pl_macro_density");
}

}  // extern "C"
