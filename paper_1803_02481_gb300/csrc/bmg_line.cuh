// Zebra line Gauss-Seidel: the per-line arithmetic shared by the full-grid
// kernels (bmg_line.cu) and the persistent coarse sub-cycle, so a level gives
// the same bits whichever of them smooths it.
//
// Section 2 names alternating line smoothing as what anisotropy calls for;
// Section 7 leaves line smoothers to future work.  Every line of one colour
// (odd lines first, 1-based) is solved exactly: a tridiagonal system whose
// off-diagonals are the couplings along the line and whose right-hand side
// holds b and the current values of the two neighbouring lines.
//
// A line of n points is cut into blocks of kLineM - 1 interior points
// separated by single separator points (line positions kLineM, 2 kLineM, ...).
// With the separator values fixed, each block is an independent tridiagonal
// system, so the solve has three data-parallel steps:
//   1. per block: g = T_blk^{-1} d_blk (forward and back substitution with
//      the block's LU factors);
//   2. per line: the Schur complement system on the separators, tridiagonal,
//      solved serially with its own LU factors;
//   3. per interior point: x = g + v x_left_sep + w x_right_sep, v and w the
//      block's responses to unit separator values (the "spikes").
// The LU factors, the spikes and the Schur factors depend only on the
// operator and are computed once at setup (bmg_line.cu).
#pragma once

#include "bmg_internal.h"

namespace bmg {

// Geometry of the lines of one direction: DIR 0 = x-lines (the rows, points
// along x, implicit in the W couplings), DIR 1 = y-lines (the columns,
// implicit in the S couplings).  Point k (1-based, 0 and n + 1 are ghosts) of
// line q (1-based) sits at plane offset q * ls + k * es (b, x and the
// couplings), and its factors and scratch at fbase(q) + k * fes: the plane
// layout for x-lines, and for y-lines the colour-compacted layout, where the
// columns of one colour are side by side (so a step along the lines of a
// colour reads contiguous words).
struct LineGeo {
  int n, nl, es, ls, fes;
};

template <int DIR, typename T>
__host__ __device__ __forceinline__ LineGeo line_geo(const LevelV<T>& L) {
  return DIR == 0 ? LineGeo{L.nx, L.ny, 1, L.pitch, 1}
                  : LineGeo{L.ny, L.nx, L.pitch, 1, L.ycp};
}

template <int DIR, typename T>
__host__ __device__ __forceinline__ int line_fbase(const LevelV<T>& L, int q) {
  return DIR == 0 ? q * L.pitch : ((q - 1) & 1) * L.yhalf + ((q - 1) >> 1);
}

// The scratch of a direction: the r plane for x-lines, the compact plane
// for y-lines.
template <int DIR, typename T>
__device__ __forceinline__ T* line_scratch(const LevelV<T>& L) {
  return DIR == 0 ? L.r : L.ys;
}

// Number of lines of colour c (0: odd lines q = 1, 3, ...; 1: even lines).
__host__ __device__ __forceinline__ int line_count(int nl, int c) { return (nl - c + 1) >> 1; }

// The coupling a_k between point k and point k - 1 of a line.
template <int DIR, typename T>
__device__ __forceinline__ const T* line_coupling(const LevelV<T>& L) {
  return DIR == 0 ? L.W : L.S;
}

// Right-hand side of a line's system at plane offset o: b plus every
// coupling that leaves the line times the current iterate x.
template <typename T, int DIR, bool NINE>
__device__ __forceinline__ T line_rhs(const LevelV<T>& L, const T* __restrict__ x, int o) {
  const int p = L.pitch;
  T d = L.b[o];
  if (DIR == 0) {
    d = fma(L.S[o], x[o - p], d);
    d = fma(L.S[o + p], x[o + p], d);
  } else {
    d = fma(L.W[o], x[o - 1], d);
    d = fma(L.W[o + 1], x[o + 1], d);
  }
  if (NINE) {
    d = fma(L.SW[o], x[o - p - 1], d);
    d = fma(L.NW[o + 1 - p], x[o + 1 - p], d);
    d = fma(L.NW[o], x[o + p - 1], d);
    d = fma(L.SW[o + 1 + p], x[o + 1 + p], d);
  }
  return d;
}

// Forward and back substitution of one block of len points: ld(e, d, mu,
// iu, ca) fetches point e's right-hand side and factors (all fetched before
// the first substitution), st(e, g) stores its solution; returns the
// solutions of the first and last point.
template <typename T, class LD, class ST>
__device__ __forceinline__ void block_subst(int len, LD ld, ST st, T& gfirst, T& glast) {
  T dv[kLineM - 1], mv[kLineM - 1], iv[kLineM - 1], cv[kLineM - 1];
#pragma unroll
  for (int e = 0; e < kLineM - 1; ++e)
    if (e < len) ld(e, dv[e], mv[e], iv[e], cv[e]);
  T prev = T(0);
#pragma unroll
  for (int e = 0; e < kLineM - 1; ++e) {
    if (e < len) {
      prev = fma(mv[e], prev, dv[e]);
      dv[e] = prev;
    }
  }
  T next = T(0);
  glast = T(0);
#pragma unroll
  for (int e = kLineM - 2; e >= 0; --e) {
    if (e < len) {
      next = fma(cv[e], next, dv[e] * iv[e]);
      if (e == len - 1) glast = next;
      st(e, next);
    }
  }
  gfirst = next;
}

// Step 1 for block bb of line q: the scratch G holds d on entry and g on
// exit.  The forward multiplier of a block's first point and the
// back-substitution coefficient of its last point are stored as 0, so every
// point takes the same two fused multiply-adds.  The full-grid variant loads
// the block's four inputs into registers first (all loads in flight at
// once), then also hands the separators their block values: d_s + a_s g_{s-1}
// of the separator after the block and g_{s+1} of the one before it (SP_RL,
// SP_GF).  The INMEM variant (the register-bound persistent kernel) keeps
// the forward values in G itself; the values are the same either way.
template <typename T, int DIR, bool INMEM = false>
__device__ __forceinline__ void line_block_solve(const LevelV<T>& L, int q, int bb) {
  const LineGeo g = line_geo<DIR>(L);
  const int k0 = bb * kLineM + 1;
  const int len = min(kLineM - 1, g.n - k0 + 1);
  if (len <= 0) return;
  const T* __restrict__ mu = L.LF[DIR][LF_MU];
  const T* __restrict__ iu = L.LF[DIR][LF_IU];
  const T* __restrict__ ca = L.LF[DIR][LF_CA];
  T* G = line_scratch<DIR>(L);
  const int f0 = line_fbase<DIR>(L, q) + k0 * g.fes;
  if constexpr (!INMEM) {
    T gfirst, glast;
    block_subst<T>(
        len,
        [&](int e, T& d, T& m, T& i, T& c) {
          const int f = f0 + e * g.fes;
          d = G[f];
          m = mu[f];
          i = iu[f];
          c = ca[f];
        },
        [&](int e, T v) { G[f0 + e * g.fes] = v; }, gfirst, glast);
    // the separators on either side (their compact slots)
    if (k0 + len <= g.n && len == kLineM - 1) {
      const int os = q * g.ls + (k0 + len) * g.es;
      L.SP[DIR][SP_RL][q * L.spp[DIR] + bb] =
          fma(line_coupling<DIR>(L)[os], glast, G[f0 + len * g.fes]);
    }
    if (bb > 0) L.SP[DIR][SP_GF][q * L.spp[DIR] + bb - 1] = gfirst;
  } else {
    T prev = T(0);
    for (int e = 0; e < len; ++e) {
      const int f = f0 + e * g.fes;
      prev = fma(mu[f], prev, G[f]);
      G[f] = prev;
    }
    T next = T(0);
    for (int e = len - 1; e >= 0; --e) {
      const int f = f0 + e * g.fes;
      next = fma(ca[f], next, G[f] * iu[f]);
      G[f] = next;
    }
  }
}

// Step 2, the Schur system on the separators of a line, tridiagonal with
// precomputed LU factors: forward y_t = mu_t y_{t-1} + rhs_t, back
// x_t = ca_t x_{t+1} + y_t / u_t.  A chain of FP64 fused multiply-adds is
// latency-bound, so each substitution runs in two levels: the separators
// form groups of sgl; every group substitutes from a zero carry (yh, xh);
// the carries between groups follow serially (one step per group, using the
// products P and Q of the group's multipliers); a fix-up adds each group's
// carry times P or Q.  Every implementation (one thread per line here, one
// thread per group in the full-grid kernel) performs these same operations:
//   rhs_t = (d_s + a_s g_{s-1}) + a_{s+1} g_{s+1}  (a_{n+1} = 0, ghost G = 0)
//   yh_t  = fma(mu_t, yh_{t-1}, rhs_t),  yh = 0 before a group
//   c_0 = 0,  c_{g+1} = fma(P_end(g), c_g, yh_end(g))
//   a_t   = fma(P_t, c_g, yh_t) * iu_t
//   xh_t  = fma(ca_t, xh_{t+1}, a_t),    xh = 0 after a group
//   e_{G-1} = 0,  e_{g-1} = fma(Q_start(g), e_g, xh_start(g))
//   x_t   = fma(Q_t, e_g, xh_t).
template <typename T, int DIR>
__device__ void line_sep_serial(const LevelV<T>& L, int q, T* __restrict__ xo) {
  const LineGeo g = line_geo<DIR>(L);
  const int nsep = g.n / kLineM;
  if (nsep == 0) return;
  const int sp = q * L.spp[DIR];
  const T* __restrict__ mu = L.SP[DIR][SP_MU] + sp;
  const T* __restrict__ iu = L.SP[DIR][SP_IU] + sp;
  const T* __restrict__ ca = L.SP[DIR][SP_CA] + sp;
  const T* __restrict__ P = L.SP[DIR][SP_P] + sp;
  const T* __restrict__ Q = L.SP[DIR][SP_Q] + sp;
  T* h = L.SP[DIR][SP_RL] + sp;         // partial values
  const T* A = line_coupling<DIR>(L);
  const T* G = line_scratch<DIR>(L);
  const int base = q * g.ls, fb = line_fbase<DIR>(L, q), gl = L.sgl[DIR];
  // forward, group by group, then each group's carry, fix-up and backward
  // partial substitution
  T c = T(0);
  for (int t0 = 0; t0 < nsep; t0 += gl) {
    const int t1 = min(t0 + gl, nsep);
    T yh = T(0);
    for (int t = t0; t < t1; ++t) {
      const int ks = (t + 1) * kLineM;
      const int os = base + ks * g.es, fs = fb + ks * g.fes;
      const T r = fma(A[os], G[fs - g.fes], G[fs]);
      yh = fma(mu[t], yh, fma(A[os + g.es], G[fs + g.fes], r));
      h[t] = yh;
    }
    const T cg = c;
    c = fma(P[t1 - 1], cg, yh);
    T xh = T(0);
    for (int t = t1 - 1; t >= t0; --t) {
      xh = fma(ca[t], xh, fma(P[t], cg, h[t]) * iu[t]);
      h[t] = xh;
    }
  }
  // backward carries and fix-up, last group first
  T e = T(0);
  for (int t0 = (nsep - 1) / gl * gl; t0 >= 0; t0 -= gl) {
    const int t1 = min(t0 + gl, nsep);
    for (int t = t0; t < t1; ++t) xo[base + (t + 1) * kLineM * g.es] = fma(Q[t], e, h[t]);
    e = fma(Q[t0], e, h[t0]);
  }
}

// Step 3 at interior point k of line q: the block's g plus the spikes times
// the separator values on either side (line position 0 or n + 1 where the
// block has no separator there: a ghost, whose value is 0).
template <typename T, int DIR>
__device__ __forceinline__ void line_final(const LevelV<T>& L, const LineGeo& g, int q, int k,
                                           T* __restrict__ xo) {
  const int kl = (k / kLineM) * kLineM;
  const int kr = min(kl + kLineM, g.n + 1);
  const int f = line_fbase<DIR>(L, q) + k * g.fes;
  const T v = L.LF[DIR][LF_V][f], w = L.LF[DIR][LF_W][f];
  const T xl = xo[q * g.ls + kl * g.es], xr = xo[q * g.ls + kr * g.es];
  xo[q * g.ls + k * g.es] = fma(w, xr, fma(v, xl, line_scratch<DIR>(L)[f]));
}

// One colour of one direction by a whole thread block (the persistent coarse
// sub-cycle), in place on L.x, with the same arithmetic as the full-grid
// kernels.
template <typename T, int DIR, bool NINE>
__device__ void blk_line_colour(const LevelV<T>& L, int colour) {
  const LineGeo g = line_geo<DIR>(L);
  const int nlc = line_count(g.nl, colour);
  T* G = line_scratch<DIR>(L);
  for (int t = threadIdx.x; t < nlc * g.n; t += blockDim.x) {
    const int q = 2 * (t / g.n) + colour + 1, k = t % g.n + 1;
    G[line_fbase<DIR>(L, q) + k * g.fes] = line_rhs<T, DIR, NINE>(L, L.x, q * g.ls + k * g.es);
  }
  __syncthreads();
  const int nb = g.n / kLineM + 1;
  for (int t = threadIdx.x; t < nlc * nb; t += blockDim.x)
    line_block_solve<T, DIR, true>(L, 2 * (t / nb) + colour + 1, t % nb);
  __syncthreads();
  for (int t = threadIdx.x; t < nlc; t += blockDim.x)
    line_sep_serial<T, DIR>(L, 2 * t + colour + 1, L.x);
  __syncthreads();
  for (int t = threadIdx.x; t < nlc * g.n; t += blockDim.x) {
    const int q = 2 * (t / g.n) + colour + 1, k = t % g.n + 1;
    if (k % kLineM != 0) line_final<T, DIR>(L, g, q, k, L.x);
  }
  __syncthreads();
}

// The (direction, colour) steps of one line sweep: x-lines, y-lines or both
// (x then y), colours 0 then 1; reversed for post-smoothing.
__host__ __device__ __forceinline__ int line_steps(int smoother, bool reverse, int* dir,
                                                   int* colour) {
  int n = 0;
  if (smoother == BMG_SMOOTH_XLINE || smoother == BMG_SMOOTH_ALTLINE) {
    dir[n] = 0, colour[n++] = 0;
    dir[n] = 0, colour[n++] = 1;
  }
  if (smoother == BMG_SMOOTH_YLINE || smoother == BMG_SMOOTH_ALTLINE) {
    dir[n] = 1, colour[n++] = 0;
    dir[n] = 1, colour[n++] = 1;
  }
  if (reverse) {
    for (int a = 0, b = n - 1; a < b; ++a, --b) {
      const int d = dir[a], c = colour[a];
      dir[a] = dir[b], colour[a] = colour[b];
      dir[b] = d, colour[b] = c;
    }
  }
  return n;
}

template <typename T, bool NINE>
__device__ void blk_line_relax(const LevelV<T>& L, int nu, bool reverse, int smoother) {
  int dir[4], colour[4];
  const int n = line_steps(smoother, reverse, dir, colour);
  for (int s = 0; s < nu; ++s)
    for (int k = 0; k < n; ++k) {
      if (dir[k] == 0)
        blk_line_colour<T, 0, NINE>(L, colour[k]);
      else
        blk_line_colour<T, 1, NINE>(L, colour[k]);
    }
}

}  // namespace bmg
