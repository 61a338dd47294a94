// Cost model of the level schedule (see bmg_schedule.h).  Per level and per
// V-cycle it counts, for every kernel of Algorithm 1, the bytes it moves and
// the flops it executes, the analogue of the Section 3 terms
// T_smooth, T_residual, T_restrict and T_interp with the halo-exchange
// latency replaced by the launch (or barrier) latency of one GPU.
#include "bmg_schedule.h"

#include <algorithm>
#include <cmath>

#include "bmg_coarse.cuh"

namespace bmg {

CostParams& cost_params() {
  // Defaults: GB300 class figures; bmg_calibrate() replaces them with
  // measured values.
  static CostParams p{2.5, 0.35, 6000.0, 1100.0, 60000.0, 120.0, 7.0, 450.0, 1.0};
  return p;
}

namespace {

struct LevelCost {
  int launches;          // kernel launches (grid mode) == phases (persistent mode)
  double bytes;          // bytes moved per V-cycle by the full-grid kernels
  double bytes_resident; // the same inside the persistent kernel, where a colour
                         // phase touches only its own points' data
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
  // inside the persistent kernel a sweep reads each point's data once
  // (neighbour values come from cache) and writes x once
  c.bytes_resident = sweeps * ((ncoef + 2) * w * n + w * n);
  c.flops = sweeps * 2.0 * ns * n;
  // residual, restriction (r, 2 weights per fine point, b_c), interpolation
  // (x in and out, weights, x_c)
  const double rest = (ncoef + 3) * w * n + (w * n + 2 * w * n + w * n / 4) +
                      (2 * w * n + 2 * w * n + w * n / 4);
  c.bytes += rest;
  c.bytes_resident += rest;
  c.flops += 2.0 * ns * n + 2.0 * 2.25 * n + 2.0 * 2.25 * n;
  return c;
}

// Latency units of one level per V-cycle inside the persistent kernel run
// by `threads` threads: every phase costs one calibrated phase per point a
// thread updates in it (a thread's points are done one after another, each
// waiting on its loads).
double phase_units(const Hierarchy* h, int l, int threads) {
  const Geom& g = h->geo64[l];
  const double n = double(g.nx) * g.ny;
  const int nc = l != h->L - 1 ? 4 : 2;
  const int sweeps = h->opt.nu1 + h->opt.nu2;
  auto units = [&](double pts) { return std::max(1.0, std::ceil(pts / threads)); };
  return sweeps * nc * units(n / nc) + units(n) + units(n / 4) + units(n);
}

}  // namespace

double predict_vcycle_us(const Hierarchy* h, int thr, int ctas) {
  const CostParams& p = cost_params();
  const bool fp32 = h->opt.precision == BMG_FP32_REFINE;
  const double fg = fp32 ? p.gpu_gflops32 : p.gpu_gflops64;
  const double fc = fp32 ? p.cta_gflops32 : p.cta_gflops64;
  const double sync = ctas > 1 ? p.cluster_sync_us : p.sync_us;
  double t = 0.0;
  for (int l = 1; l < h->L; ++l) {
    const LevelCost c = level_cost(h, l);
    if (l >= thr) {
      // full-grid launches: latency + streaming at the GPU rates
      const double work = std::max(c.bytes / (p.gpu_gbs * 1e3), c.flops / (fg * 1e3));
      t += c.launches * p.launch_us + work;
    } else {
      // inside the persistent kernel: barrier latency + work at the rates of
      // `ctas` SMs
      const double work =
          std::max(c.bytes_resident / (ctas * p.cta_gbs * 1e3), c.flops / (ctas * fc * 1e3));
      const int threads = ctas > 1 ? ctas * kCoarseClusterThreads : 1024;
      t += phase_units(h, l, threads) * sync + work;
    }
  }
  // the persistent kernel itself and the coarsest solve (n0^2 flops, as the
  // T_cgsolve term of Section 3)
  const double n0 = double(h->n0);
  t += p.launch_us + 2 * std::log2(std::max(2.0, n0)) * p.sync_us + 2.0 * n0 * n0 / (fc * 1e3);
  return t;
}

void choose_schedule(Hierarchy* h) {
  const bool point = h->opt.smoother == BMG_SMOOTH_POINT;
  int cands[2] = {1, 1};
  int nc = 1;
  if (h->opt.coarse_ctas > 0) {
    cands[0] = h->opt.coarse_ctas;
  } else if (point) {
    const int cmax = max_cluster_ctas(h->opt.precision == BMG_FP32_REFINE);
    if (cmax > 1) cands[nc++] = cmax;
  }
  const int t0 = h->opt.coarse_threshold > 0 ? h->opt.coarse_threshold : 1;
  const int t1 = h->opt.coarse_threshold > 0 ? h->opt.coarse_threshold : h->L;
  double bt = 1e300;
  for (int k = 0; k < nc; ++k) {
    for (int thr = t0; thr <= t1; ++thr) {
      const double t = predict_vcycle_us(h, thr, cands[k]);
      if (t < bt) {
        bt = t;
        h->threshold = thr;
        h->coarse_ctas = cands[k];
      }
    }
  }
  for (int thr = 1; thr <= h->L && thr <= 16; ++thr)
    h->predicted_us[thr - 1] = predict_vcycle_us(h, thr, h->coarse_ctas);
}

}  // namespace bmg

// ---------------------------------------------------------------------------
// Calibration: measure the parameters of the cost model on this device (the
// analogue of measuring alpha, beta, gamma with machine benchmarks in
// Section 3).  Results stay in cost_params() for the process.
// ---------------------------------------------------------------------------

namespace bmg {

namespace {

__global__ void k_empty() {}

// Colour phases of the persistent kernels themselves, timed on a synthetic
// 15 x 15 nine-point level (values all zero: the timing of a phase does not
// depend on them): one thread block, or every block of a cluster.  At one
// point per thread the arithmetic is negligible, so this is the latency of a
// phase (loads, stores, barrier); the cost model adds the arithmetic.
template <class Team>
__global__ void __launch_bounds__(1024) k_phases_real(LevelV<double> L, int phases) {
  for (int p = 0; p < phases; ++p) blk_colour<double, true, Team>(L, four_mask(p & 3));
}

cudaError_t launch_phases_cluster(int ctas, cudaStream_t s, const LevelV<double>& L, int phases) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(ctas));
  cfg.blockDim = dim3(kCoarseClusterThreads);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = unsigned(ctas);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_phases_real<ClusterTeam>, L, phases);
}

// A 15 x 15 nine-point level carved from scratch memory (planes 256-byte
// aligned, interior rows 128-byte aligned as in a hierarchy).
LevelV<double> probe_level(double* scratch) {
  const Geom g = make_geom<double>(15, 15);
  LevelV<double> L{};
  L.nx = g.nx;
  L.ny = g.ny;
  L.pitch = g.pitch;
  size_t off = 0;
  auto plane = [&]() {
    off = (off + 31) & ~size_t(31);                    // 256 bytes
    double* p = scratch + off + base_shift<double>();
    off += g.elems;
    return p;
  };
  L.C = plane();
  L.iC = plane();
  L.W = plane();
  L.S = plane();
  L.SW = plane();
  L.NW = plane();
  L.x = plane();
  L.b = plane();
  return L;
}

template <typename T>
__global__ void k_fma_rate(T* out, int iters, T a, T c) {
  T x0 = T(threadIdx.x) * T(1e-3), x1 = x0 + T(1), x2 = x0 + T(2), x3 = x0 + T(3);
  T x4 = x0 + T(4), x5 = x0 + T(5), x6 = x0 + T(6), x7 = x0 + T(7);
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, c); x1 = fma(x1, a, c); x2 = fma(x2, a, c); x3 = fma(x3, a, c);
    x4 = fma(x4, a, c); x5 = fma(x5, a, c); x6 = fma(x6, a, c); x7 = fma(x7, a, c);
  }
  const T s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
  if (s == T(-12345)) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_stream(const double2* __restrict__ in, double2* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    out[i] = in[i];
}

float time_ms(cudaStream_t s, cudaEvent_t a, cudaEvent_t b) {
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  return ms;
}

}  // namespace

int calibrate(cudaStream_t s, double* out) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return BMG_ECUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  CostParams p = cost_params();
  double* buf = nullptr;
  const size_t stream_elems = size_t(1) << 26;      // 2 x 512 MiB in double
  if (cudaMalloc(&buf, sizeof(double) * (2 * stream_elems + 1024)) != cudaSuccess) {
    cudaGetLastError();
    return BMG_ENOMEM;
  }
  cudaMemsetAsync(buf, 0, sizeof(double) * (2 * stream_elems + 1024), s);
  // launch latency: back-to-back empty launches on the stream
  for (int i = 0; i < 20; ++i) k_empty<<<1, 32, 0, s>>>();
  cudaEventRecord(e0, s);
  const int nl = 400;
  for (int i = 0; i < nl; ++i) k_empty<<<1, 32, 0, s>>>();
  cudaEventRecord(e1, s);
  p.launch_us = 1e3 * time_ms(s, e0, e1) / nl;
  // one colour phase of the persistent kernel on a small nine-point level:
  // in one block, and over the largest cluster the coarse kernel can use
  const LevelV<double> probe = probe_level(buf);
  const int ph = 2000;
  k_phases_real<BlockTeam><<<1, coarse_block_threads(), 0, s>>>(probe, 8);
  cudaEventRecord(e0, s);
  k_phases_real<BlockTeam><<<1, coarse_block_threads(), 0, s>>>(probe, ph);
  cudaEventRecord(e1, s);
  p.sync_us = 1e3 * time_ms(s, e0, e1) / ph;
  const int cmax = max_cluster_ctas(false);
  if (cmax > 1) {
    cudaFuncSetAttribute(k_phases_real<ClusterTeam>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    launch_phases_cluster(cmax, s, probe, 8);
    cudaEventRecord(e0, s);
    launch_phases_cluster(cmax, s, probe, ph);
    cudaEventRecord(e1, s);
    p.cluster_sync_us = 1e3 * time_ms(s, e0, e1) / ph;
  }
  // FMA rates, whole GPU and one block
  const int iters = 1 << 14, tb = 256;
  auto rate = [&](auto tag, int blocks) {
    using T = decltype(tag);
    k_fma_rate<T><<<blocks, tb, 0, s>>>(reinterpret_cast<T*>(buf), 64, T(1.0000001), T(1e-7));
    cudaEventRecord(e0, s);
    k_fma_rate<T><<<blocks, tb, 0, s>>>(reinterpret_cast<T*>(buf), iters, T(1.0000001), T(1e-7));
    cudaEventRecord(e1, s);
    const double ms = time_ms(s, e0, e1);
    return 2.0 * 8.0 * iters * double(blocks) * tb / (ms * 1e6);   // GFLOP/s
  };
  p.gpu_gflops64 = rate(double(0), 4 * sms);
  p.cta_gflops64 = rate(double(0), 1);
  p.gpu_gflops32 = rate(float(0), 8 * sms);
  p.cta_gflops32 = rate(float(0), 1);
  // streaming bandwidth: copy 512 MiB (read + write bytes)
  const size_t n2 = stream_elems / 2;
  const double2* src = reinterpret_cast<const double2*>(buf);
  double2* dst = reinterpret_cast<double2*>(buf + stream_elems);
  k_stream<<<4 * sms, 512, 0, s>>>(src, dst, n2);
  cudaEventRecord(e0, s);
  k_stream<<<4 * sms, 512, 0, s>>>(src, dst, n2);
  cudaEventRecord(e1, s);
  p.gpu_gbs = 2.0 * sizeof(double) * stream_elems / (time_ms(s, e0, e1) * 1e6);
  // one block on an L2-resident 4 MiB buffer
  const size_t small2 = (size_t(1) << 19) / 2;
  k_stream<<<1, coarse_block_threads(), 0, s>>>(src, dst, small2);
  cudaEventRecord(e0, s);
  for (int r = 0; r < 4; ++r) k_stream<<<1, coarse_block_threads(), 0, s>>>(src, dst, small2);
  cudaEventRecord(e1, s);
  p.cta_gbs = 4 * 2.0 * sizeof(double) * (size_t(1) << 19) / (time_ms(s, e0, e1) * 1e6);
  const bool ok = cudaGetLastError() == cudaSuccess;
  cudaFree(buf);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) return BMG_ECUDA;
  cost_params() = p;
  if (out) {
    out[0] = p.launch_us;
    out[1] = p.sync_us;
    out[2] = p.gpu_gbs;
    out[3] = p.gpu_gflops64;
    out[4] = p.gpu_gflops32;
    out[5] = p.cta_gbs;
    out[6] = p.cta_gflops64;
    out[7] = p.cta_gflops32;
    out[8] = p.cluster_sync_us;
    out[9] = double(cmax);
  }
  return BMG_OK;
}

}  // namespace bmg

extern "C" int bmg_calibrate(bmg_stream_t stream, double* params_out) {
  return bmg::calibrate(reinterpret_cast<cudaStream_t>(stream), params_out);
}

extern "C" int bmg_predict_cycle_us(const bmg_hierarchy* hp, int threshold, double* us) {
  const bmg::Hierarchy* h = reinterpret_cast<const bmg::Hierarchy*>(hp);
  if (!h || !us || threshold < 1 || threshold > h->L) return BMG_EINVAL;
  *us = bmg::predict_vcycle_us(h, threshold, h->coarse_ctas);
  return BMG_OK;
}

extern "C" int bmg_max_coarse_ctas(int precision, int* out) {
  if (!out || (precision != BMG_FP64 && precision != BMG_FP32_REFINE)) return BMG_EINVAL;
  *out = bmg::max_cluster_ctas(precision == BMG_FP32_REFINE);
  return BMG_OK;
}
