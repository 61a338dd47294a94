// V-cycle kernels (Algorithm 1): multicolour Gauss-Seidel, residual,
// restriction R = P^T, interpolate-and-correct, the coarsest direct solve,
// the persistent kernel that runs every level below the schedule threshold
// inside one thread block (the single-GPU reading of the coarse-grid
// redistribution of Section 2.2 / Algorithm 2), residual norms with the
// device-side stop test, and the FP64 kernels of iterative refinement.
#include "bmg_internal.h"

#include <cmath>

namespace bmg {

namespace {

constexpr int kTB = 128;
inline int cdiv(long a, long b) { return int((a + b - 1) / b); }

// A colour is a set of parity sub-lattices; bit (2*pj + pi) stands for the
// points whose 0-based row index j-1 has parity pj and column i-1 parity pi.
// Red-black: red = {(0,0),(1,1)} = (i + j) even, black = {(0,1),(1,0)}.
// Four colours, in the order (i mod 2, j mod 2) = (1,1), (0,1), (1,0), (0,0)
// (1-based): sub-lattices (0,0), (0,1), (1,0), (1,1).
__host__ __device__ constexpr unsigned rb_mask(int c) { return c == 0 ? 0x9u : 0x6u; }
__host__ __device__ constexpr unsigned four_mask(int c) { return 1u << c; }

template <typename T, bool NINE>
__global__ void k_residual(LevelV<T> L, const T* __restrict__ x, const T* __restrict__ b,
                           T* __restrict__ r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int j = blockIdx.y + 1;
  if (i > L.nx) return;
  const int o = j * L.pitch + i;
  r[o] = resid_value<T, NINE>(L, x, b[o], o);
}

template <typename T>
__global__ void k_restrict(LevelV<T> F, const T* __restrict__ r, LevelV<T> Cc, int zero_x) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int J = blockIdx.y + 1;
  if (I > Cc.nx) return;
  const int c = J * Cc.pitch + I;
  const int f = 2 * J * F.pitch + 2 * I;
  Cc.b[c] = restrict_value<T>(F.P, Cc.pitch, r, F.pitch, c, f);
  if (zero_x) Cc.x[c] = T(0);
}

template <typename T>
__global__ void k_interp(LevelV<T> F, const T* __restrict__ xc, int add_rc, T* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int j = blockIdx.y + 1;
  if (i > F.nx) return;
  const int o = j * F.pitch + i;
  T corr = interp_value<T>(F.P, F.cpitch, xc, i, j);
  // Section 3 interpolation equations: + r/C at points that are not coarse
  // points (r is the residual computed after pre-smoothing).
  if (add_rc && ((i | j) & 1)) corr = fma(F.r[o], F.iC[o], corr);
  out[o] = F.x[o] + corr;
}

// ---------------------------------------------------------------------------
// Persistent coarse sub-cycle: one thread block runs Algorithm 1 on levels
// 0 .. thr-1, starting from b_{thr-1} and leaving x_{thr-1}.  Phases are
// separated by __syncthreads(); the per-point arithmetic is the same as in
// the full-grid kernels, so the result does not depend on the threshold.
// ---------------------------------------------------------------------------

template <typename T>
struct CoarseArgs {
  const LevelV<T>* lev;      // device array of level views
  int thr;                   // levels 0 .. thr-1 run here
  int nu1, nu2, add_rc;
  int top_nine;              // is level thr-1 9-point (else red-black)
  const double* chol;        // N0 x N0 lower factor
  const double* idiag;       // 1 / L[i][i]
  int n0;
};

template <typename T, bool NINE>
__device__ void blk_colour(const LevelV<T>& L, unsigned mask) {
  const int hx = (L.nx + 1) >> 1, hy = (L.ny + 1) >> 1;
  for (int t = threadIdx.x; t < hx * hy; t += blockDim.x) {
    const int ii = t % hx, jj = t / hx;
#pragma unroll
    for (int pj = 0; pj < 2; ++pj) {
#pragma unroll
      for (int pi = 0; pi < 2; ++pi) {
        if (!(mask & (1u << (2 * pj + pi)))) continue;
        const int i = 1 + pi + 2 * ii, j = 1 + pj + 2 * jj;
        if (i > L.nx || j > L.ny) continue;
        const int o = j * L.pitch + i;
        L.x[o] = gs_value<T, NINE>(L, L.x, L.b[o], o);
      }
    }
  }
  __syncthreads();
}

template <typename T, bool NINE>
__device__ void blk_relax(const LevelV<T>& L, int nu, bool reverse) {
  const int nc = NINE ? 4 : 2;
  for (int s = 0; s < nu; ++s) {
    for (int k = 0; k < nc; ++k) {
      const int c = reverse ? nc - 1 - k : k;
      blk_colour<T, NINE>(L, NINE ? four_mask(c) : rb_mask(c));
    }
  }
}

template <typename T, bool NINE>
__device__ void blk_residual(const LevelV<T>& L) {
  for (int t = threadIdx.x; t < L.nx * L.ny; t += blockDim.x) {
    const int i = t % L.nx + 1, j = t / L.nx + 1;
    const int o = j * L.pitch + i;
    L.r[o] = resid_value<T, NINE>(L, L.x, L.b[o], o);
  }
  __syncthreads();
}

template <typename T>
__device__ void blk_restrict(const LevelV<T>& F, const LevelV<T>& Cc) {
  for (int t = threadIdx.x; t < Cc.nx * Cc.ny; t += blockDim.x) {
    const int I = t % Cc.nx + 1, J = t / Cc.nx + 1;
    const int c = J * Cc.pitch + I;
    Cc.b[c] = restrict_value<T>(F.P, Cc.pitch, F.r, F.pitch, c, 2 * J * F.pitch + 2 * I);
    Cc.x[c] = T(0);
  }
  __syncthreads();
}

template <typename T>
__device__ void blk_interp(const LevelV<T>& F, const T* xc, int add_rc) {
  for (int t = threadIdx.x; t < F.nx * F.ny; t += blockDim.x) {
    const int i = t % F.nx + 1, j = t / F.nx + 1;
    const int o = j * F.pitch + i;
    T corr = interp_value<T>(F.P, F.cpitch, xc, i, j);
    if (add_rc && ((i | j) & 1)) corr = fma(F.r[o], F.iC[o], corr);
    F.x[o] = F.x[o] + corr;
  }
  __syncthreads();
}

// x_0 = A_0^{-1} b_0 with the stored factor (forward then backward
// substitution, column-oriented, in FP64 shared memory).
template <typename T>
__device__ void blk_coarse_solve(const LevelV<T>& L0, const double* __restrict__ lo,
                                 const double* __restrict__ idiag, int n) {
  __shared__ double v[BMG_MAX_COARSEST];
  const int nx = L0.nx;
  for (int r = threadIdx.x; r < n; r += blockDim.x)
    v[r] = double(L0.b[(r / nx + 1) * L0.pitch + r % nx + 1]);
  __syncthreads();
  if (n <= 64) {
    if (threadIdx.x == 0) {
      for (int j = 0; j < n; ++j) {
        const double y = v[j] * idiag[j];
        v[j] = y;
        for (int i = j + 1; i < n; ++i) v[i] = fma(-lo[size_t(i) * n + j], y, v[i]);
      }
      for (int j = n - 1; j >= 0; --j) {
        const double xj = v[j] * idiag[j];
        v[j] = xj;
        for (int i = 0; i < j; ++i) v[i] = fma(-lo[size_t(j) * n + i], xj, v[i]);
      }
    }
    __syncthreads();
  } else {
    for (int j = 0; j < n; ++j) {
      const double y = v[j] * idiag[j];
      __syncthreads();
      if (threadIdx.x == 0) v[j] = y;
      for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x)
        v[i] = fma(-lo[size_t(i) * n + j], y, v[i]);
      __syncthreads();
    }
    for (int j = n - 1; j >= 0; --j) {
      const double xj = v[j] * idiag[j];
      __syncthreads();
      if (threadIdx.x == 0) v[j] = xj;
      for (int i = threadIdx.x; i < j; i += blockDim.x) v[i] = fma(-lo[size_t(j) * n + i], xj, v[i]);
      __syncthreads();
    }
  }
  for (int r = threadIdx.x; r < n; r += blockDim.x)
    L0.x[(r / nx + 1) * L0.pitch + r % nx + 1] = T(v[r]);
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(1024) k_coarse_cycle(CoarseArgs<T> a) {
  for (int l = a.thr - 1; l >= 1; --l) {
    const LevelV<T> L = a.lev[l];
    const bool nine = (l < a.thr - 1) || a.top_nine;
    if (nine) {
      blk_relax<T, true>(L, a.nu1, false);
      blk_residual<T, true>(L);
    } else {
      blk_relax<T, false>(L, a.nu1, false);
      blk_residual<T, false>(L);
    }
    blk_restrict<T>(L, a.lev[l - 1]);
  }
  blk_coarse_solve<T>(a.lev[0], a.chol, a.idiag, a.n0);
  for (int l = 1; l < a.thr; ++l) {
    const LevelV<T> L = a.lev[l];
    const bool nine = (l < a.thr - 1) || a.top_nine;
    blk_interp<T>(L, a.lev[l - 1].x, a.add_rc);
    if (nine)
      blk_relax<T, true>(L, a.nu2, true);
    else
      blk_relax<T, false>(L, a.nu2, true);
  }
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
                                                             Scalars* sc, int what, double* hist) {
  double acc = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) acc += partials[k];
  acc = block_sum(acc);
  if (threadIdx.x != 0) return;
  if (what == 0) {
    sc->bnorm2 = acc;
    sc->rnorm2 = acc;
    return;
  }
  sc->scale2 = sc->rnorm2;
  sc->rnorm2 = acc;
  const double rel = sqrt(acc / sc->bnorm2);
  sc->rel = rel;
  if (sc->cycles < BMG_MAX_HISTORY) hist[sc->cycles] = rel;
  const bool finite = isfinite(rel);
  if (!finite) sc->err |= DEV_NAN;
  const int go = (finite && rel > sc->tol && sc->cycles < sc->max_cycles && sc->err == 0) ? 1 : 0;
  sc->go = go;
  sc->cycles += go;
}

// FP32_REFINE: r = b - A x in FP64 on the finest level (partials of ||r||^2)
// and the FP32 right-hand side r / ||r_prev|| of the next FP32 V-cycle; the
// FP32 fine iterate is reset to zero.
template <bool NINE>
__global__ void __launch_bounds__(kNormThreads) k_refine_residual(LevelV<double> L, LevelV<float> F,
                                                                  const Scalars* sc,
                                                                  double* partials) {
  const double inv = 1.0 / sqrt(sc->rnorm2);
  double acc = 0.0;
  for (int j = blockIdx.x + 1; j <= L.ny; j += gridDim.x) {
    for (int i = threadIdx.x + 1; i <= L.nx; i += blockDim.x) {
      const int o = j * L.pitch + i;
      const double r = resid_value<double, NINE>(L, L.x, L.b[o], o);
      acc = fma(r, r, acc);
      const int of = j * F.pitch + i;
      F.b[of] = float(r * inv);
      F.x[of] = 0.0f;
    }
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// x += ||r_prev|| * e  (e the FP32 correction).
__global__ void k_refine_update(LevelV<double> L, LevelV<float> F, const Scalars* sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int j = blockIdx.y + 1;
  if (i > L.nx) return;
  const double s = sqrt(sc->scale2);
  const int o = j * L.pitch + i;
  L.x[o] = fma(s, double(F.x[j * F.pitch + i]), L.x[o]);
}

}  // namespace

// ---------------------------------------------------------------------------
// Launch wrappers
// ---------------------------------------------------------------------------

template <typename T>
void launch_residual(const LevelV<T>& L, bool nine, const T* x, const T* b, T* r,
                     cudaStream_t s) {
  const dim3 grid(cdiv(L.nx, kTB), L.ny);
  if (!nine) prof_begin(BMG_PROF_FINE_RESID, s);
  if (nine)
    k_residual<T, true><<<grid, kTB, 0, s>>>(L, x, b, r);
  else
    k_residual<T, false><<<grid, kTB, 0, s>>>(L, x, b, r);
  if (!nine) prof_end(BMG_PROF_FINE_RESID, s);
  count_launch();
}

template <typename T>
void launch_restrict(const LevelV<T>& fine, const T* r, LevelV<T> coarse, bool zero_x,
                     cudaStream_t s) {
  const dim3 grid(cdiv(coarse.nx, kTB), coarse.ny);
  k_restrict<T><<<grid, kTB, 0, s>>>(fine, r, coarse, zero_x ? 1 : 0);
  count_launch();
}

template <typename T>
void launch_interp(const LevelV<T>& fine, const T* xc, bool add_r_over_c, cudaStream_t s, T* out) {
  const dim3 grid(cdiv(fine.nx, kTB), fine.ny);
  const bool finest = fine.SW == nullptr;
  if (finest) prof_begin(BMG_PROF_FINE_INTERP, s);
  k_interp<T><<<grid, kTB, 0, s>>>(fine, xc, add_r_over_c ? 1 : 0, out ? out : fine.x);
  if (finest) prof_end(BMG_PROF_FINE_INTERP, s);
  count_launch();
}

template <typename T>
void launch_coarse_cycle(Hierarchy* h, const LevelV<T>* dev_levels, int thr, cudaStream_t s) {
  CoarseArgs<T> a;
  a.lev = dev_levels;
  a.thr = thr;
  a.nu1 = h->opt.nu1;
  a.nu2 = h->opt.nu2;
  a.add_rc = h->opt.interp_residual_term;
  a.top_nine = (thr < h->L) ? 1 : 0;
  a.chol = h->chol;
  a.idiag = h->chol_idiag;
  a.n0 = h->n0;
  prof_begin(BMG_PROF_COARSE, s);
  k_coarse_cycle<T><<<1, 1024, 0, s>>>(a);
  prof_end(BMG_PROF_COARSE, s);
  count_launch();
}

void launch_fine_norm(Hierarchy* h, const double* x, const double* b, int what, double tol,
                      cudaStream_t s) {
  (void)tol;
  const LevelV<double>& L = h->d.back();
  prof_begin(BMG_PROF_NORM, s);
  k_fine_norm<false><<<h->npartials, kNormThreads, 0, s>>>(L, x, b, what, h->partials);
  k_norm_final<<<1, kNormThreads, 0, s>>>(h->partials, h->npartials, h->sc, what, h->hist);
  prof_end(BMG_PROF_NORM, s);
  count_launch(2);
}

void launch_refine_residual(Hierarchy* h, double tol, cudaStream_t s) {
  (void)tol;
  k_refine_residual<false><<<h->npartials, kNormThreads, 0, s>>>(h->d.back(), h->f.back(), h->sc,
                                                                 h->partials);
  k_norm_final<<<1, kNormThreads, 0, s>>>(h->partials, h->npartials, h->sc, 1, h->hist);
  count_launch(2);
}

void launch_refine_update(Hierarchy* h, cudaStream_t s) {
  const LevelV<double>& L = h->d.back();
  k_refine_update<<<dim3(cdiv(L.nx, kTB), L.ny), kTB, 0, s>>>(L, h->f.back(), h->sc);
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
template void launch_interp<double>(const LevelV<double>&, const double*, bool, cudaStream_t,
                                    double*);
template void launch_interp<float>(const LevelV<float>&, const float*, bool, cudaStream_t, float*);
template void launch_coarse_cycle<double>(Hierarchy*, const LevelV<double>*, int, cudaStream_t);
template void launch_coarse_cycle<float>(Hierarchy*, const LevelV<float>*, int, cudaStream_t);

}  // namespace bmg
