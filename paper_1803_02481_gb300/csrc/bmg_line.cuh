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
// line q (1-based) sits at plane offset q * ls + k * es.
struct LineGeo {
  int n, nl, es, ls;
};

template <int DIR, typename T>
__host__ __device__ __forceinline__ LineGeo line_geo(const LevelV<T>& L) {
  return DIR == 0 ? LineGeo{L.nx, L.ny, 1, L.pitch} : LineGeo{L.ny, L.nx, L.pitch, 1};
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

// Step 1 for block bb of line q: G holds d on entry and g on exit.  The
// forward multiplier of a block's first point and the back-substitution
// coefficient of its last point are stored as 0, so every point takes the
// same two fused multiply-adds.  The forward values stay in registers, or
// (INMEM, for the register-bound persistent kernel) in G itself; the values
// are the same either way.
template <typename T, int DIR, bool INMEM = false>
__device__ __forceinline__ void line_block_solve(const LevelV<T>& L, int q, int bb) {
  const LineGeo g = line_geo<DIR>(L);
  const int k0 = bb * kLineM + 1;
  const int len = min(kLineM - 1, g.n - k0 + 1);
  if (len <= 0) return;
  const T* __restrict__ mu = L.LF[DIR][LF_MU];
  const T* __restrict__ iu = L.LF[DIR][LF_IU];
  const T* __restrict__ ca = L.LF[DIR][LF_CA];
  T* G = L.r;
  const int o0 = q * g.ls + k0 * g.es;
  if constexpr (INMEM) {
    T prev = T(0);
    for (int e = 0; e < len; ++e) {
      const int o = o0 + e * g.es;
      prev = fma(mu[o], prev, G[o]);
      G[o] = prev;
    }
    T next = T(0);
    for (int e = len - 1; e >= 0; --e) {
      const int o = o0 + e * g.es;
      next = fma(ca[o], next, G[o] * iu[o]);
      G[o] = next;
    }
  } else {
    T y[kLineM - 1];
    T prev = T(0);
#pragma unroll
    for (int e = 0; e < kLineM - 1; ++e) {
      if (e < len) {
        const int o = o0 + e * g.es;
        prev = fma(mu[o], prev, G[o]);
        y[e] = prev;
      }
    }
    T next = T(0);
#pragma unroll
    for (int e = kLineM - 2; e >= 0; --e) {
      if (e < len) {
        const int o = o0 + e * g.es;
        next = fma(ca[o], next, y[e] * iu[o]);
        G[o] = next;
      }
    }
  }
}

// Right-hand side of the Schur system at the separator at offset os:
// d_s + a_s g_{s-1} + a_{s+1} g_{s+1} (a_{n+1} = 0 and the ghost of G is 0).
template <typename T, int DIR>
__device__ __forceinline__ T line_sep_rhs(const LevelV<T>& L, int es, int os) {
  const T* A = line_coupling<DIR>(L);
  const T* G = L.r;
  const T r = fma(A[os], G[os - es], G[os]);
  return fma(A[os + es], G[os + es], r);
}

// Step 2 for line q by one thread: forward substitution (y overwrites d_s in
// G), then back substitution writing the separator values into xo.
template <typename T, int DIR>
__device__ void line_sep_serial(const LevelV<T>& L, int q, T* __restrict__ xo) {
  const LineGeo g = line_geo<DIR>(L);
  const int nsep = g.n / kLineM;
  const T* __restrict__ mu = L.LF[DIR][LF_MU];
  const T* __restrict__ iu = L.LF[DIR][LF_IU];
  const T* __restrict__ ca = L.LF[DIR][LF_CA];
  T* G = L.r;
  const int base = q * g.ls, step = kLineM * g.es;
  T y = T(0);
  for (int t = 0; t < nsep; ++t) {
    const int os = base + (t + 1) * step;
    y = fma(mu[os], y, line_sep_rhs<T, DIR>(L, g.es, os));
    G[os] = y;
  }
  T xn = T(0);
  for (int t = nsep - 1; t >= 0; --t) {
    const int os = base + (t + 1) * step;
    xn = fma(ca[os], xn, G[os] * iu[os]);
    xo[os] = xn;
  }
}

// Step 3 at interior point k of line q (plane offset o): the block's g plus
// the spikes times the separator values on either side (line position 0 or
// n + 1 where the block has no separator there: a ghost, whose value is 0).
template <typename T, int DIR>
__device__ __forceinline__ void line_final(const LevelV<T>& L, const LineGeo& g, int q, int k,
                                           T* __restrict__ xo) {
  const int kl = (k / kLineM) * kLineM;
  const int kr = min(kl + kLineM, g.n + 1);
  const int o = q * g.ls + k * g.es;
  const T v = L.LF[DIR][LF_V][o], w = L.LF[DIR][LF_W][o];
  const T xl = xo[q * g.ls + kl * g.es], xr = xo[q * g.ls + kr * g.es];
  xo[o] = fma(w, xr, fma(v, xl, L.r[o]));
}

// One colour of one direction by a whole thread block (the persistent coarse
// sub-cycle), in place on L.x, with the same arithmetic as the full-grid
// kernels.
template <typename T, int DIR, bool NINE>
__device__ void blk_line_colour(const LevelV<T>& L, int colour) {
  const LineGeo g = line_geo<DIR>(L);
  const int nlc = line_count(g.nl, colour);
  for (int t = threadIdx.x; t < nlc * g.n; t += blockDim.x) {
    const int q = 2 * (t / g.n) + colour + 1, k = t % g.n + 1;
    const int o = q * g.ls + k * g.es;
    L.r[o] = line_rhs<T, DIR, NINE>(L, L.x, o);
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
