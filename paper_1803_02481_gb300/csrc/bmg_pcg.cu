// Conjugate gradients on the finest operator, preconditioned by one
// symmetric V(nu, nu) cycle of Algorithm 1 from a zero initial guess (on the
// FP64 levels, or on the FP32 hierarchy of BMG_FP32_REFINE; an
// extension: the paper iterates V-cycles; with nu1 = nu2, the colours of the
// post-smoothing reversed, R = P^T and an exact coarsest solve, the cycle is
// a symmetric positive definite preconditioner).
//
// The vectors live on the finest FP64 level: the level's b plane holds the
// residual r (it is the V-cycle's right-hand side), its x plane z = M^{-1} r
// (the V-cycle's output), and Hierarchy::pcg_x, pcg_b, pcg_p, pcg_q hold the
// iterate, the right-hand side, the search direction and A p.  Every kernel
// walks the level with a fixed grid, fixed per-thread order and a fixed
// reduction tree (deterministic dot products); one thread then turns the
// partial sums into the scalars (alpha, beta, or the stop test of
// k_norm_final, which also drives the solve graph's WHILE node).
#include "bmg_internal.h"

namespace bmg {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double pcg_block_sum(double v) {
  __shared__ double red[kThreads / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = v;
  __syncthreads();
  v = lane < kThreads / 32 ? red[lane] : 0.0;
  if (w == 0) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  }
  return v;
}

// Visits every interior point of the finest level: rows blockIdx.x + 1,
// + gridDim.x, ...; columns threadIdx.x + 1, + blockDim.x, ...
template <class F>
__device__ __forceinline__ double for_points(const LevelV<double>& L, F f) {
  double acc = 0.0;
  for (int j = blockIdx.x + 1; j <= L.ny; j += gridDim.x)
    for (int i = threadIdx.x + 1; i <= L.nx; i += blockDim.x) acc = f(j * L.pitch + i, acc);
  return pcg_block_sum(acc);
}

// r = b - A x (r in L.b), z = 0 (L.x), partials of r.r.
__global__ void __launch_bounds__(kThreads) k_pcg_init(LevelV<double> L,
                                                       const double* __restrict__ x,
                                                       const double* __restrict__ b,
                                                       double* __restrict__ partials) {
  const double s = for_points(L, [&](int o, double acc) {
    const double r = resid_value<double, false>(L, x, b[o], o);
    L.b[o] = r;
    if (L.PR[PR_B]) L.PR[PR_B][o] = r * L.iC[o];   // prescaled level: b/C too
    L.x[o] = 0.0;
    return fma(r, r, acc);
  });
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// q = A p (the negated residual of p for b = 0), partials of p.q.
__global__ void __launch_bounds__(kThreads) k_pcg_ap(LevelV<double> L,
                                                     const double* __restrict__ p,
                                                     double* __restrict__ q,
                                                     double* __restrict__ partials) {
  const double s = for_points(L, [&](int o, double acc) {
    const double qv = -resid_value<double, false>(L, p, 0.0, o);
    q[o] = qv;
    return fma(p[o], qv, acc);
  });
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// x += alpha p, r -= alpha q, z = 0, partials of r.r.
__global__ void __launch_bounds__(kThreads) k_pcg_xr(LevelV<double> L, double* __restrict__ x,
                                                     const double* __restrict__ p,
                                                     const double* __restrict__ q,
                                                     const Scalars* __restrict__ sc,
                                                     double* __restrict__ partials) {
  const double a = sc->alpha;
  const double s = for_points(L, [&](int o, double acc) {
    x[o] = fma(a, p[o], x[o]);
    const double r = fma(-a, q[o], L.b[o]);
    L.b[o] = r;
    if (L.PR[PR_B]) L.PR[PR_B][o] = r * L.iC[o];
    L.x[o] = 0.0;
    return fma(r, r, acc);
  });
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// partials of r.z
__global__ void __launch_bounds__(kThreads) k_pcg_rz(LevelV<double> L,
                                                     double* __restrict__ partials) {
  const double s = for_points(L, [&](int o, double acc) { return fma(L.b[o], L.x[o], acc); });
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// p = z + beta p
__global__ void __launch_bounds__(kThreads) k_pcg_p(LevelV<double> L, double* __restrict__ p,
                                                    const Scalars* __restrict__ sc) {
  const double beta = sc->beta;
  for (int j = blockIdx.x + 1; j <= L.ny; j += gridDim.x)
    for (int i = threadIdx.x + 1; i <= L.nx; i += blockDim.x) {
      const int o = j * L.pitch + i;
      p[o] = fma(beta, p[o], L.x[o]);
    }
}

// One thread block sums the partials; what 0: rz = sum, beta = 0 (first
// direction); 1: alpha = rz / sum (sum = p.q); 2: beta = sum / rz, rz = sum
// (sum = r.z of the new residual).  A zero denominator gives 0.
__global__ void __launch_bounds__(kThreads) k_pcg_scalar(const double* __restrict__ partials,
                                                         int n, Scalars* sc, int what) {
  double acc = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) acc += partials[k];
  acc = pcg_block_sum(acc);
  if (threadIdx.x != 0) return;
  if (what == 0) {
    sc->rz = acc;
    sc->beta = 0.0;
  } else if (what == 1) {
    sc->alpha = acc != 0.0 ? sc->rz / acc : 0.0;
  } else {
    sc->beta = sc->rz != 0.0 ? acc / sc->rz : 0.0;
    sc->rz = acc;
  }
}

// FP32 preconditioner: the FP32 finest level's right-hand side r / ||r||
// and x32 = 0 (||r|| of the latest residual: sc->inv, sc->rnorm, set once by
// the norm's final kernel); after the FP32 cycle z = ||r|| e.
__global__ void k_pcg_cast(LevelV<double> L, LevelV<float> F, const Scalars* __restrict__ sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1, j = blockIdx.y + 1;
  if (i > L.nx) return;
  const int of = j * F.pitch + i;
  F.b[of] = float(L.b[j * L.pitch + i] * sc->inv);
  F.x[of] = 0.0f;
}

__global__ void k_pcg_uncast(LevelV<double> L, LevelV<float> F, const Scalars* __restrict__ sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1, j = blockIdx.y + 1;
  if (i > L.nx) return;
  L.x[j * L.pitch + i] = sc->rnorm * double(F.x[j * F.pitch + i]);
}

}  // namespace

void launch_pcg_precond(Hierarchy* h, cudaStream_t s) {
  if (h->opt.precision != BMG_FP32_REFINE) {
    // the PCG kernels left z = 0 in the finest x plane
    enqueue_vcycle<double>(h, h->d, h->dlev64, h->threshold, s, -1, false, true);
    return;
  }
  LevelV<double>& F = h->d.back();
  const dim3 g((F.nx + kThreads - 1) / kThreads, F.ny);
  k_pcg_cast<<<g, kThreads, 0, s>>>(F, h->f.back(), h->sc);
  // (the cast zeroed the FP32 fine iterate)
  enqueue_vcycle<float>(h, h->f, h->dlev32, h->threshold, s, -1, false, true);
  k_pcg_uncast<<<g, kThreads, 0, s>>>(F, h->f.back(), h->sc);
  count_launch(2);
}

void launch_pcg_init(Hierarchy* h, cudaStream_t s, bool in_graph) {
  LevelV<double>& F = h->d.back();
  prof_begin(BMG_PROF_KRYLOV, s);
  k_pcg_init<<<h->npartials, kThreads, 0, s>>>(F, h->pcg_x, h->pcg_b, h->partials);
  launch_norm_final(h, s, in_graph);
  prof_end(BMG_PROF_KRYLOV, s);
  count_launch();
}

void launch_pcg_ap(Hierarchy* h, cudaStream_t s) {
  LevelV<double>& F = h->d.back();
  prof_begin(BMG_PROF_KRYLOV, s);
  k_pcg_ap<<<h->npartials, kThreads, 0, s>>>(F, h->pcg_p, h->pcg_q, h->partials);
  k_pcg_scalar<<<1, kThreads, 0, s>>>(h->partials, h->npartials, h->sc, 1);
  prof_end(BMG_PROF_KRYLOV, s);
  count_launch(2);
}

void launch_pcg_xr(Hierarchy* h, cudaStream_t s, bool in_graph) {
  LevelV<double>& F = h->d.back();
  prof_begin(BMG_PROF_KRYLOV, s);
  k_pcg_xr<<<h->npartials, kThreads, 0, s>>>(F, h->pcg_x, h->pcg_p, h->pcg_q, h->sc,
                                             h->partials);
  launch_norm_final(h, s, in_graph);
  prof_end(BMG_PROF_KRYLOV, s);
  count_launch();
}

void launch_pcg_rz(Hierarchy* h, bool first, cudaStream_t s) {
  LevelV<double>& F = h->d.back();
  prof_begin(BMG_PROF_KRYLOV, s);
  k_pcg_rz<<<h->npartials, kThreads, 0, s>>>(F, h->partials);
  k_pcg_scalar<<<1, kThreads, 0, s>>>(h->partials, h->npartials, h->sc, first ? 0 : 2);
  prof_end(BMG_PROF_KRYLOV, s);
  count_launch(2);
}

void launch_pcg_p(Hierarchy* h, cudaStream_t s) {
  LevelV<double>& F = h->d.back();
  prof_begin(BMG_PROF_KRYLOV, s);
  k_pcg_p<<<h->npartials, kThreads, 0, s>>>(F, h->pcg_p, h->sc);
  prof_end(BMG_PROF_KRYLOV, s);
  count_launch();
}

}  // namespace bmg
