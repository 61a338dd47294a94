// Cost model of the level schedule (see bmg_schedule.h).  Per level and per
// V-cycle it counts, for every kernel of Algorithm 1, the bytes it moves and
// the flops it executes, the analogue of the Section 3 terms
// T_smooth, T_residual, T_restrict and T_interp with the halo-exchange
// latency replaced by the launch (or barrier) latency of one GPU.
#include "bmg_schedule.h"

#include <algorithm>
#include <cmath>

namespace bmg {

CostParams& cost_params() {
  // Defaults: GB300 class figures; bmg_calibrate() replaces them with
  // measured values.
  static CostParams p{2.5, 0.35, 6000.0, 1100.0, 60000.0, 120.0, 7.0, 450.0};
  return p;
}

namespace {

struct LevelCost {
  int launches;          // kernel launches (grid mode) == phases (block mode)
  double bytes;          // bytes moved per V-cycle
  double flops;          // flops per V-cycle
};

// Work of one level l >= 1 per V-cycle: nu1 + nu2 sweeps of n_c colours,
// residual, restriction to l-1, interpolation from l-1 (Algorithm 1).
LevelCost level_cost(const Hierarchy* h, int l) {
  const bool fp32 = h->opt.precision == BMG_FP32_REFINE;
  const double w = fp32 ? 4.0 : 8.0;
  const Geom& g = h->geo64[l];
  const double n = double(g.nx) * g.ny;
  const bool nine = l != h->L - 1;
  const int nc = nine ? 4 : 2;
  const int ns = nine ? 9 : 5;
  const int ncoef = nine ? 5 : 3;        // iC (or C), W, S [, SW, NW]
  const int sweeps = h->opt.nu1 + h->opt.nu2;
  LevelCost c{};
  c.launches = sweeps * nc + 3;
  // a colour launch streams every coefficient plane, b and x, writes 1/nc of x
  c.bytes = sweeps * nc * ((ncoef + 2) * w * n + w * n / nc);
  c.flops = sweeps * 2.0 * ns * n;
  // residual
  c.bytes += (ncoef + 3) * w * n;
  c.flops += 2.0 * ns * n;
  // restriction: r, 2 weights per fine point, b_c
  c.bytes += w * n + 2 * w * n + w * n / 4;
  c.flops += 2.0 * 2.25 * n;
  // interpolation: x in and out, weights, x_c
  c.bytes += 2 * w * n + 2 * w * n + w * n / 4;
  c.flops += 2.0 * 2.25 * n;
  return c;
}

}  // namespace

double predict_vcycle_us(const Hierarchy* h, int thr) {
  const CostParams& p = cost_params();
  const bool fp32 = h->opt.precision == BMG_FP32_REFINE;
  const double fg = fp32 ? p.gpu_gflops32 : p.gpu_gflops64;
  const double fc = fp32 ? p.cta_gflops32 : p.cta_gflops64;
  double t = 0.0;
  for (int l = 1; l < h->L; ++l) {
    const LevelCost c = level_cost(h, l);
    if (l >= thr) {
      // full-grid launches: latency + streaming at the GPU rates
      const double work = std::max(c.bytes / (p.gpu_gbs * 1e3), c.flops / (fg * 1e3));
      t += c.launches * p.launch_us + work;
    } else {
      // inside one block: barrier latency + work at one SM's rates
      const double work = std::max(c.bytes / (p.cta_gbs * 1e3), c.flops / (fc * 1e3));
      t += c.launches * p.sync_us + work;
    }
  }
  // the persistent kernel itself and the coarsest solve (n0^2 flops, as the
  // T_cgsolve term of Section 3)
  const double n0 = double(h->n0);
  t += p.launch_us + 2 * std::log2(std::max(2.0, n0)) * p.sync_us + 2.0 * n0 * n0 / (fc * 1e3);
  return t;
}

int choose_threshold(Hierarchy* h) {
  int best = 1;
  double bt = 1e300;
  for (int thr = 1; thr <= h->L; ++thr) {
    const double t = predict_vcycle_us(h, thr);
    if (thr - 1 < 16) h->predicted_us[thr - 1] = t;
    if (t < bt) {
      bt = t;
      best = thr;
    }
  }
  return best;
}

}  // namespace bmg
