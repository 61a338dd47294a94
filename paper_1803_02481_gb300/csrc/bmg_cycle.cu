// V-cycle kernels (Algorithm 1): multicolour Gauss-Seidel, residual,
// restriction R = P^T, interpolate-and-correct, the coarsest direct solve,
// the persistent kernel that runs every level below the schedule threshold
// inside one thread block (the single-GPU reading of the coarse-grid
// redistribution of Section 2.2 / Algorithm 2), residual norms with the
// device-side stop test, and the FP64 kernels of iterative refinement.
#include "bmg_coarse.cuh"

#include <cmath>
#include <cstdlib>

namespace bmg {

namespace {

constexpr int kTB = 128;
inline int cdiv(long a, long b) { return int((a + b - 1) / b); }


template <typename T, bool NINE>
__global__ void k_residual(LevelV<T> L, const T* __restrict__ x, const T* __restrict__ b,
                           T* __restrict__ r) {
  griddep_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int j = blockIdx.y + 1;
  if (i > L.nx) return;
  const int o = j * L.pitch + i;
  r[o] = resid_value<T, NINE>(L, x, b[o], o);
}

template <typename T>
__global__ void k_restrict(LevelV<T> F, const T* __restrict__ r, LevelV<T> Cc, int zero_x) {
  griddep_wait();
  const int I = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int J = blockIdx.y + 1;
  if (I > Cc.nx) return;
  const int c = J * Cc.pitch + I;
  const int f = 2 * J * F.pitch + 2 * I;
  Cc.b[c] = restrict_value<T>(F.P, Cc.pitch, r, F.pitch, c, f);
  if (zero_x) Cc.x[c] = T(0);
}

// Residual and restriction in one pass (Algorithm 1: b_{l-1} = P^T (b - A x)).
// A block owns kRRX x kRRY coarse points; it first computes the residual on
// the (2 kRRX + 1) x (2 kRRY + 1) fine points they gather from (one shared
// row and column with each neighbouring block) into shared memory, then
// restricts from there, so r never goes to global memory.  Both steps use
// resid_value and restrict_value, so b_{l-1} is bit-identical to the two
// separate kernels'.
constexpr int kRRX = 32, kRRY = 8, kRRT = 256;

template <typename T, bool NINE>
__global__ void __launch_bounds__(kRRT) k_resid_restrict(LevelV<T> F, LevelV<T> Cc) {
  griddep_wait();
  constexpr int RW = 2 * kRRX + 1, RH = 2 * kRRY + 1;
  __shared__ T rs[RH * RW];
  const int I0 = blockIdx.x * kRRX + 1, J0 = blockIdx.y * kRRY + 1;
  // fine point of rs[0]: (2 I0 - 1, 2 J0 - 1)
  const int fi0 = 2 * I0 - 1, fj0 = 2 * J0 - 1;
  for (int e = threadIdx.x; e < RW * RH; e += kRRT) {
    const int rr = e / RW, cc = e - rr * RW;
    const int i = fi0 + cc, j = fj0 + rr;
    T v = T(0);
    if (i <= F.nx && j <= F.ny) {
      const int o = j * F.pitch + i;
      v = resid_value<T, NINE>(F, F.x, F.b[o], o);
    }
    rs[e] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kRRX * kRRY; e += kRRT) {
    const int dj = e / kRRX, di = e - dj * kRRX;
    const int I = I0 + di, J = J0 + dj;
    if (I > Cc.nx || J > Cc.ny) continue;
    const int c = J * Cc.pitch + I;
    // coarse (I, J) is fine (2I, 2J): rs cell (2 dj + 1, 2 di + 1)
    Cc.b[c] = restrict_value<T>(F.P, Cc.pitch, rs, RW, c, (2 * dj + 1) * RW + 2 * di + 1);
    Cc.x[c] = T(0);
  }
}

// Two adjacent values of T as one aligned vector access.
template <typename T>
struct Pair;
template <>
struct Pair<double> {
  using type = double2;
};
template <>
struct Pair<float> {
  using type = float2;
};

// One thread per coarse cell (I, J), 0 <= I <= ncx, 0 <= J <= ncy: the four
// fine points (2I+1..2I+2, 2J+1..2J+2) -- a cell centre, a y-edge, an x-edge
// and a coarse point -- so every thread does the same work (no divergence on
// the point type) and the weight planes are read contiguously.  The points
// (2I+1, j) and (2I+2, j) of a row are one vector load and store: element 1
// of every row starts a 128-byte line and the pitch is a multiple of it, so
// the pair starts on a multiple of 2 * sizeof(T) bytes.  A pair that would
// reach the ghost column nx + 1 is done point by point.
template <typename T>
__global__ void k_interp(LevelV<T> F, const T* __restrict__ xc, int add_rc, T* __restrict__ out) {
  griddep_wait();
  using V = typename Pair<T>::type;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y;
  const int ncx = (F.nx - 1) >> 1;
  if (I > ncx) return;
  const int i = 2 * I + 1;
#pragma unroll
  for (int dj = 1; dj <= 2; ++dj) {
    const int j = 2 * J + dj;
    if (j > F.ny) continue;
    const int o = j * F.pitch + i;
    if (i + 1 <= F.nx) {
      T c0 = interp_value<T>(F.P, F.cpitch, xc, i, j);
      T c1 = interp_value<T>(F.P, F.cpitch, xc, i + 1, j);
      // Section 3 interpolation equations: + r/C at points that are not
      // coarse points (r is the residual computed after pre-smoothing); i
      // is odd, so (i, j) never is one and (i + 1, j) is one for even j.
      if (add_rc) {
        const V rv = *reinterpret_cast<const V*>(F.r + o);
        const V cv = *reinterpret_cast<const V*>(F.iC + o);
        c0 = fma(rv.x, cv.x, c0);
        if (j & 1) c1 = fma(rv.y, cv.y, c1);
      }
      V xv = *reinterpret_cast<const V*>(F.x + o);
      xv.x += c0;
      xv.y += c1;
      *reinterpret_cast<V*>(out + o) = xv;
    } else if (i <= F.nx) {
      T corr = interp_value<T>(F.P, F.cpitch, xc, i, j);
      if (add_rc) corr = fma(F.r[o], F.iC[o], corr);
      out[o] = F.x[o] + corr;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_coarse_cycle(CoarseArgs<T> a) {
  griddep_wait();
  coarse_cycle_body<T>(a);
}

// The same with line smoothing; fewer threads leave each more registers for
// a block's substitution.
template <typename T>
__global__ void __launch_bounds__(512, 1) k_coarse_cycle_line(CoarseArgs<T> a) {
  griddep_wait();
  coarse_cycle_body<T, true>(a);
}

// The point-smoother sub-cycle over every block of one thread-block cluster
// (launched with a cluster dimension equal to the grid): each phase is spread
// over the cluster's blocks, one per SM, and phases are separated by the
// hardware cluster barrier.
template <typename T>
__global__ void __launch_bounds__(kCoarseClusterThreads, 1) k_coarse_cycle_cluster(CoarseArgs<T> a) {
  griddep_wait();
  coarse_cycle_body<T, false, ClusterTeam>(a);
}

template <typename T>
static cudaError_t launch_cluster_kernel(int ctas, cudaStream_t s, const CoarseArgs<T>& a) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(ctas));
  cfg.blockDim = dim3(kCoarseClusterThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = unsigned(ctas);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, k_coarse_cycle_cluster<T>, a);
}

// Largest cluster size (a power of two up to 16) whose blocks of the cluster
// kernel the device can co-schedule, 1 when clusters are unavailable.
// Sizes above 8 need the non-portable cluster attribute.
template <typename T>
static int max_cluster_ctas_t() {
  int dev = 0, cc = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  cudaDeviceGetAttribute(&cc, cudaDevAttrClusterLaunch, dev);
  if (!cc) return 1;
  cudaFuncSetAttribute(k_coarse_cycle_cluster<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  for (int c = 16; c >= 2; c /= 2) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(c));
    cfg.blockDim = dim3(kCoarseClusterThreads);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = unsigned(c);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_coarse_cycle_cluster<T>, &cfg) == cudaSuccess && n > 0)
      return c;
    cudaGetLastError();
  }
  return 1;
}


// ---------------------------------------------------------------------------
// Norms and the stop test.  Fixed grid, fixed per-thread order and a fixed
// reduction tree, so the result is deterministic.
// ---------------------------------------------------------------------------

constexpr int kNormThreads = 256;

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[kNormThreads / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = v;
  __syncthreads();
  v = lane < kNormThreads / 32 ? red[lane] : 0.0;
  if (w == 0) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  }
  return v;
}

// what == 0: sum of b^2; what == 1: sum of (b - A x)^2 on the finest FP64
// level.  One partial per block.
template <bool NINE>
__global__ void __launch_bounds__(kNormThreads) k_fine_norm(LevelV<double> L, const double* x,
                                                            const double* b, int what,
                                                            double* partials) {
  griddep_wait();
  double acc = 0.0;
  for (int j = blockIdx.x + 1; j <= L.ny; j += gridDim.x) {
    for (int i = threadIdx.x + 1; i <= L.nx; i += blockDim.x) {
      const int o = j * L.pitch + i;
      const double v = what ? resid_value<double, NINE>(L, x, b[o], o) : b[o];
      acc = fma(v, v, acc);
    }
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// Sums the partials; what == 0 stores ||b||^2, else stores ||r||^2 (keeping
// the previous one in scale2), the relative residual and the loop flag.
__global__ void __launch_bounds__(kNormThreads) k_norm_final(const double* partials, int n,
                                                             Scalars* sc, int what, double* hist,
                                                             cudaGraphConditionalHandle cond,
                                                             int use_cond) {
  griddep_wait();
  double acc = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) acc += partials[k];
  acc = block_sum(acc);
  if (threadIdx.x != 0) return;
  if (what == 0) {
    sc->bnorm2 = acc;
    sc->rnorm2 = acc;
    sc->rnorm = sqrt(acc);
    sc->inv = acc > 0.0 ? 1.0 / sc->rnorm : 0.0;
    return;
  }
  sc->scale2 = sc->rnorm2;
  sc->scale = sqrt(sc->scale2);
  sc->rnorm2 = acc;
  sc->rnorm = sqrt(acc);
  sc->inv = acc > 0.0 ? 1.0 / sc->rnorm : 0.0;
  const double rel = sqrt(acc / sc->bnorm2);
  sc->rel = rel;
  if (sc->cycles < BMG_MAX_HISTORY) hist[sc->cycles] = rel;
  const bool finite = isfinite(rel);
  if (!finite) sc->err |= DEV_NAN;
  const int go = (finite && rel > sc->tol && sc->cycles < sc->max_cycles && sc->err == 0) ? 1 : 0;
  sc->go = go;
  sc->cycles += go;
  // inside the solve graph this drives the WHILE node
  if (use_cond) cudaGraphSetConditional(cond, go ? 1u : 0u);
}

// FP32_REFINE: r = b - A x in FP64 on the finest level (partials of ||r||^2)
// and the FP32 right-hand side r / ||r_prev|| of the next FP32 V-cycle; the
// FP32 fine iterate is reset to zero.  The scaling to the FP32 right-hand
// side is done in FP32 (float(r) * float(1/||r_prev||), one more FP32
// rounding than an FP64 product, and one FP64 instruction less per point)
// while 1/||r_prev|| lies in (1e-28, 1e28), where every entry that matters
// for the FP32 correction is a normal FP32 number; outside, in FP64.  The
// choice is uniform over the launch, so each loop is branch-free.
template <bool NINE, bool SCALE32>
__device__ __forceinline__ double refine_rows(const LevelV<double>& L, const LevelV<float>& F,
                                              double inv) {
  const float inv32 = float(inv);
  const double* __restrict__ x = L.x;
  const double* __restrict__ b = L.b;
  float* __restrict__ fb = F.b;
  float* __restrict__ fx = F.x;
  double acc = 0.0;
  for (int j = blockIdx.x + 1; j <= L.ny; j += gridDim.x) {
    for (int i = threadIdx.x + 1; i <= L.nx; i += blockDim.x) {
      const int o = j * L.pitch + i;
      const double r = resid_value<double, NINE>(L, x, b[o], o);
      acc = fma(r, r, acc);
      const int of = j * F.pitch + i;
      fb[of] = SCALE32 ? float(r) * inv32 : float(r * inv);
      fx[of] = 0.0f;
    }
  }
  return acc;
}

template <bool NINE>
__global__ void __launch_bounds__(kNormThreads) k_refine_residual(LevelV<double> L, LevelV<float> F,
                                                                  const Scalars* sc,
                                                                  double* partials) {
  griddep_wait();
  const double inv = sc->inv;
  double acc = (inv > 1e-28 && inv < 1e28) ? refine_rows<NINE, true>(L, F, inv)
                                           : refine_rows<NINE, false>(L, F, inv);
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// x += ||r_prev|| * e  (e the FP32 correction).
// One thread per pair of points (i, i+1), i odd: interior rows start on
// 128-byte boundaries, so the pair is one 16-byte FP64 and one 8-byte FP32
// access; a last unpaired point (i = nx, nx odd) is done alone.
__global__ void k_refine_update(LevelV<double> L, LevelV<float> F, const Scalars* sc) {
  griddep_wait();
  const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + 1;
  const int j = blockIdx.y + 1;
  if (i > L.nx) return;
  const double s = sc->scale;
  double* x = L.x + j * L.pitch + i;
  const float* e = F.x + j * F.pitch + i;
  if (i < L.nx) {
    double2 xv = *reinterpret_cast<const double2*>(x);
    const float2 ev = *reinterpret_cast<const float2*>(e);
    xv.x = fma(s, double(ev.x), xv.x);
    xv.y = fma(s, double(ev.y), xv.y);
    *reinterpret_cast<double2*>(x) = xv;
  } else {
    x[0] = fma(s, double(e[0]), x[0]);
  }
}

}  // namespace

bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("BMG_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}

int max_cluster_ctas(bool fp32) {
  static int cached[2] = {0, 0};
  int& c = cached[fp32 ? 1 : 0];
  if (c == 0) c = fp32 ? max_cluster_ctas_t<float>() : max_cluster_ctas_t<double>();
  return c;
}

// ---------------------------------------------------------------------------
// Launch wrappers
// ---------------------------------------------------------------------------

template <typename T>
void launch_residual(const LevelV<T>& L, bool nine, const T* x, const T* b, T* r,
                     cudaStream_t s) {
  const dim3 grid(cdiv(L.nx, kTB), L.ny);
  if (!nine) prof_begin(BMG_PROF_FINE_RESID, s);
  if (nine)
    launch_pdl(k_residual<T, true>, grid, dim3(kTB), 0, s, L, x, b, r);
  else
    launch_pdl(k_residual<T, false>, grid, dim3(kTB), 0, s, L, x, b, r);
  if (!nine) prof_end(BMG_PROF_FINE_RESID, s);
  count_launch();
}

template <typename T>
void launch_restrict(const LevelV<T>& fine, const T* r, LevelV<T> coarse, bool zero_x,
                     cudaStream_t s) {
  const dim3 grid(cdiv(coarse.nx, kTB), coarse.ny);
  launch_pdl(k_restrict<T>, grid, dim3(kTB), 0, s, fine, r, coarse, zero_x ? 1 : 0);
  count_launch();
}

// Which levels take the fused residual + restriction: BMG_RR_FUSED=0 never,
// 1 always, unset the measured choice: FP32 levels, which are bound by
// memory traffic (the 8191^2 FP32-refined solve 99.5 -> 97.3 ms).  FP64
// levels keep the separate kernels: the FP64 pipe bounds the residual either
// way, and the fused kernel's per-thread loop over several residuals hid
// latency worse (4095^2 solve 3924 -> 3961 ms with fused 9-point levels; on
// the launch-latency-bound small levels too: fused below 512 points wide,
// the 255^2 Poisson cycle took 137.9 instead of 130.3 us).
bool rr_fused(bool nine, bool fp64) {
  (void)nine;
  static const int v = [] {
    const char* e = std::getenv("BMG_RR_FUSED");
    return e && e[0] ? std::atoi(e) : -1;
  }();
  if (v >= 0) return v != 0;
  return !fp64;
}

template <typename T>
void launch_resid_restrict(const LevelV<T>& fine, bool nine, LevelV<T> coarse, cudaStream_t s) {
  const dim3 grid(cdiv(coarse.nx, kRRX), cdiv(coarse.ny, kRRY));
  if (!nine) prof_begin(BMG_PROF_FINE_RESID, s);
  if (nine)
    launch_pdl(k_resid_restrict<T, true>, grid, dim3(kRRT), 0, s, fine, coarse);
  else
    launch_pdl(k_resid_restrict<T, false>, grid, dim3(kRRT), 0, s, fine, coarse);
  if (!nine) prof_end(BMG_PROF_FINE_RESID, s);
  count_launch();
}

template <typename T>
void launch_interp(const LevelV<T>& fine, const T* xc, bool add_r_over_c, cudaStream_t s, T* out) {
  const int ncx = (fine.nx - 1) / 2, ncy = (fine.ny - 1) / 2;
  const dim3 grid(cdiv(ncx + 1, kTB), ncy + 1);
  const bool finest = fine.SW == nullptr;
  if (finest) prof_begin(BMG_PROF_FINE_INTERP, s);
  launch_pdl(k_interp<T>, grid, dim3(kTB), 0, s, fine, xc, add_r_over_c ? 1 : 0, out ? out : fine.x);
  if (finest) prof_end(BMG_PROF_FINE_INTERP, s);
  count_launch();
}

// Threads of the one-block persistent kernel (environment BMG_COARSE_THREADS,
// a multiple of 32 up to 1024).  Measured on the 255^2 Poisson cycle with
// the coarse kernel on levels 15^2 and below: 127.3 us at 1024 threads,
// 124.9 at 512, 124.7 at 256, 136.3 at 128 (another box: 129.8 and 127.3 at
// 1024 and 512); 512 also keeps wider levels inside the kernel near the
// 1024-thread cost.  The model's calibration probes use the same count.
int coarse_block_threads() {
  static const int n = [] {
    const char* e = std::getenv("BMG_COARSE_THREADS");
    const int v = e && e[0] ? std::atoi(e) : 512;
    return v >= 32 && v <= 1024 && v % 32 == 0 ? v : 512;
  }();
  return n;
}

template <typename T>
void launch_coarse_cycle(Hierarchy* h, const LevelV<T>* dev_levels, int thr, cudaStream_t s) {
  CoarseArgs<T> a;
  a.lev = dev_levels;
  a.thr = thr;
  a.nu1 = h->opt.nu1;
  a.nu2 = h->opt.nu2;
  a.add_rc = h->opt.interp_residual_term;
  a.smoother = h->opt.smoother;
  a.top_nine = (thr < h->L) ? 1 : 0;
  a.chol = h->chol;
  a.idiag = h->chol_idiag;
  a.n0 = h->n0;
  prof_begin(BMG_PROF_COARSE, s);
  if (a.smoother != BMG_SMOOTH_POINT)
    launch_pdl(k_coarse_cycle_line<T>, dim3(1), dim3(512), 0, s, a);
  else if (h->coarse_ctas > 1)
    launch_cluster_kernel<T>(h->coarse_ctas, s, a);
  else
    launch_pdl(k_coarse_cycle<T>, dim3(1), dim3(coarse_block_threads()), 0, s, a);
  prof_end(BMG_PROF_COARSE, s);
  count_launch();
}

void launch_fine_norm(Hierarchy* h, const double* x, const double* b, int what, double tol,
                      cudaStream_t s, bool in_graph) {
  (void)tol;
  const LevelV<double>& L = h->d.back();
  prof_begin(BMG_PROF_NORM, s);
  launch_pdl(k_fine_norm<false>, dim3(h->npartials), dim3(kNormThreads), 0, s, L, x, b, what,
             h->partials);
  launch_pdl(k_norm_final, dim3(1), dim3(kNormThreads), 0, s, (const double*)h->partials,
             h->npartials, h->sc, what, h->hist, h->cond, in_graph ? 1 : 0);
  prof_end(BMG_PROF_NORM, s);
  count_launch(2);
}

void launch_refine_residual(Hierarchy* h, double tol, cudaStream_t s, bool in_graph) {
  (void)tol;
  launch_pdl(k_refine_residual<false>, dim3(h->npartials), dim3(kNormThreads), 0, s, h->d.back(),
             h->f.back(), (const Scalars*)h->sc, h->partials);
  launch_pdl(k_norm_final, dim3(1), dim3(kNormThreads), 0, s, (const double*)h->partials,
             h->npartials, h->sc, 1, h->hist, h->cond, in_graph ? 1 : 0);
  count_launch(2);
}

void launch_norm_final(Hierarchy* h, cudaStream_t s, bool in_graph, int n) {
  launch_pdl(k_norm_final, dim3(1), dim3(kNormThreads), 0, s, (const double*)h->partials,
             n > 0 ? n : h->npartials, h->sc, 1, h->hist, h->cond, in_graph ? 1 : 0);
  count_launch();
}

void launch_refine_update(Hierarchy* h, cudaStream_t s) {
  const LevelV<double>& L = h->d.back();
  launch_pdl(k_refine_update, dim3(cdiv((L.nx + 1) / 2, kTB), L.ny), dim3(kTB), 0, s, L, h->f.back(),
             (const Scalars*)h->sc);
  count_launch();
}

template void launch_residual<double>(const LevelV<double>&, bool, const double*, const double*,
                                      double*, cudaStream_t);
template void launch_residual<float>(const LevelV<float>&, bool, const float*, const float*,
                                     float*, cudaStream_t);
template void launch_restrict<double>(const LevelV<double>&, const double*, LevelV<double>, bool,
                                      cudaStream_t);
template void launch_restrict<float>(const LevelV<float>&, const float*, LevelV<float>, bool,
                                     cudaStream_t);
template void launch_resid_restrict<double>(const LevelV<double>&, bool, LevelV<double>,
                                            cudaStream_t);
template void launch_resid_restrict<float>(const LevelV<float>&, bool, LevelV<float>,
                                           cudaStream_t);
template void launch_interp<double>(const LevelV<double>&, const double*, bool, cudaStream_t,
                                    double*);
template void launch_interp<float>(const LevelV<float>&, const float*, bool, cudaStream_t, float*);
template void launch_coarse_cycle<double>(Hierarchy*, const LevelV<double>*, int, cudaStream_t);
template void launch_coarse_cycle<float>(Hierarchy*, const LevelV<float>*, int, cudaStream_t);

}  // namespace bmg
