// 3D BoxMG V-cycle (include/boxmg3d.h): assembly, operator-induced
// interpolation, Galerkin coarse operators, multicolour Gauss-Seidel,
// residual, restriction, interpolation, dense coarsest solve, and the solve
// loop as one CUDA graph per cycle.
//
// Layout: every grid quantity is a plane of (nz + 2) x (ny + 2) rows of px
// doubles with a one-cell zero ghost layer; point (i, j, k) (1-based) at
// (k * (ny + 2) + j) * px + i, px >= nx + 2 a multiple of 16 (128-byte rows).
// An operator is symmetric: its diagonal C, 1/C, and the negated
// off-diagonals a_d = -A[p, p + d] for the 13 "negative" offsets d (dk = -1;
// or dk = 0, dj = -1; or (-1, 0, 0)); the coupling to +d is a_{-d} of the
// neighbour at p + d.  Couplings to points outside the grid are 0.
// Interpolation into a level: 8 planes on that level's grid, the weight of
// each fine point to its parent corners (plane 4 cz + 2 cy + cx; per
// direction a fine point at odd 1-based i has parents (i-1)/2 (c = 0) and
// (i+1)/2 (c = 1), at even i the single parent i/2 (c = 0)).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <new>
#include <vector>

#include "bmg_internal.h"
#include "boxmg3d.h"

namespace bmg3 {

using bmg::count_launch;
using bmg::griddep_wait;
using bmg::set_last_error;

constexpr int NA = 13;    // stored couplings per point
constexpr int NPW3 = 8;   // interpolation weight planes
constexpr int kT = 128;   // threads along x
constexpr int kNormBlocks = 4 * 152;
constexpr int kNormThreads = 256;

// A level's planes in FP64 (the hierarchy) or FP32 (the V-cycles of
// FP32 refinement: the FP64 operator and interpolation rounded once).
template <typename T>
struct Lev3T {
  int nx, ny, nz, px, py;
  T *C, *iC, *A[NA];
  T *x, *b, *r;
  T *P[NPW3];
};
using Lev3 = Lev3T<double>;
using Lev3f = Lev3T<float>;

template <typename T>
__host__ __device__ __forceinline__ int off3(const Lev3T<T>& L, int di, int dj, int dk) {
  return (dk * L.py + dj) * L.px + di;
}
template <typename T>
__host__ __device__ __forceinline__ int idx3(const Lev3T<T>& L, int i, int j, int k) {
  return (k * L.py + j) * L.px + i;
}
__host__ __device__ __forceinline__ bool is_neg(int di, int dj, int dk) {
  return dk < 0 || (dk == 0 && (dj < 0 || (dj == 0 && di < 0)));
}
// storage index of a negative offset
__host__ __device__ __forceinline__ int neg_index(int di, int dj, int dk) {
  if (dk == -1) return (dj + 1) * 3 + (di + 1);
  if (dj == -1) return 9 + (di + 1);
  return 12;
}
// a_d at point o (negated off-diagonal to o + d)
template <typename T>
__device__ __forceinline__ T coupling(const Lev3T<T>& L, int o, int di, int dj, int dk) {
  if (is_neg(di, dj, dk)) return L.A[neg_index(di, dj, dk)][o];
  return L.A[neg_index(-di, -dj, -dk)][o + off3(L, di, dj, dk)];
}

enum { E3_BADK = 1, E3_BADDEN = 2, E3_NOTSPD = 4 };

// ---------------------------------------------------------------------------
// Assembly: harmonic faces, 2k on boundary faces; the diagonal summed in the
// order x faces (east, west, west wall, east wall), then y, then z.
// ---------------------------------------------------------------------------

__device__ __forceinline__ double hmean(double lo, double hi) { return 2.0 * lo * hi / (lo + hi); }

__global__ void k3_assemble(const double* __restrict__ k, Lev3 L, int* err) {
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x, j0 = blockIdx.y, k0 = blockIdx.z;
  if (i0 >= L.nx) return;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const size_t sxy = size_t(nx) * ny;
  const size_t q = size_t(k0) * sxy + size_t(j0) * nx + i0;
  const double kc = k[q];
  if (!(kc > 0.0) || !(kc < INFINITY)) atomicOr(err, E3_BADK);
  const double aE = i0 < nx - 1 ? hmean(kc, k[q + 1]) : 0.0;
  const double aW = i0 > 0 ? hmean(k[q - 1], kc) : 0.0;
  const double aN = j0 < ny - 1 ? hmean(kc, k[q + nx]) : 0.0;
  const double aS = j0 > 0 ? hmean(k[q - nx], kc) : 0.0;
  const double aU = k0 < nz - 1 ? hmean(kc, k[q + sxy]) : 0.0;
  const double aD = k0 > 0 ? hmean(k[q - sxy], kc) : 0.0;
  double c = 0.0;
  c = __dadd_rn(c, aE);
  c = __dadd_rn(c, aW);
  c = __dadd_rn(c, i0 == 0 ? 2.0 * kc : 0.0);
  c = __dadd_rn(c, i0 == nx - 1 ? 2.0 * kc : 0.0);
  c = __dadd_rn(c, aN);
  c = __dadd_rn(c, aS);
  c = __dadd_rn(c, j0 == 0 ? 2.0 * kc : 0.0);
  c = __dadd_rn(c, j0 == ny - 1 ? 2.0 * kc : 0.0);
  c = __dadd_rn(c, aU);
  c = __dadd_rn(c, aD);
  c = __dadd_rn(c, k0 == 0 ? 2.0 * kc : 0.0);
  c = __dadd_rn(c, k0 == nz - 1 ? 2.0 * kc : 0.0);
  const int o = idx3(L, i0 + 1, j0 + 1, k0 + 1);
  L.C[o] = c;
  L.iC[o] = 1.0 / c;
  L.A[neg_index(-1, 0, 0)][o] = aW;
  L.A[neg_index(0, -1, 0)][o] = aS;
  L.A[neg_index(0, 0, -1)][o] = aD;
}

// ---------------------------------------------------------------------------
// Interpolation weights of the fine level F, one pass per number of
// directions in which a point lies between coarse points (0: coarse points,
// 1: edge, 2: face, 3: cell centre points; each pass reads the weights of
// the passes before it).  Operation order as the oracle's: couplings in
// offset order (dk, dj, di) ascending, products and sums unfused.
// ---------------------------------------------------------------------------

// The weights of fine point (i, j, k) if it belongs to the pass.
__device__ void weights_point(const Lev3& F, int i, int j, int k, int pass, int* err) {
  const int fr[3] = {i & 1, j & 1, k & 1};    // 1: between coarse points in that direction
  const int nb = fr[0] + fr[1] + fr[2];
  if (nb != pass) return;
  const int o = idx3(F, i, j, k);
  if (nb == 0) {
    F.P[0][o] = 1.0;
    return;
  }
  // couplings with the lumping of non-M-matrix rows
  double a[27];
  const double C = F.C[o];
  double sum = 0.0, neg = 0.0;
  for (int dk = -1; dk <= 1; ++dk)
    for (int dj = -1; dj <= 1; ++dj)
      for (int di = -1; di <= 1; ++di) {
        const int t = (dk + 1) * 9 + (dj + 1) * 3 + (di + 1);
        if (t == 13) {
          a[t] = 0.0;
          continue;
        }
        const double v = coupling(F, o, di, dj, dk);
        sum = __dadd_rn(sum, v);
        neg = __dadd_rn(neg, fmin(v, 0.0));
        a[t] = fmax(v, 0.0);
      }
  const double sigma = __dsub_rn(C, sum);
  const double ceff = __dsub_rn(__dsub_rn(C, neg), fmin(sigma, 0.0));
  // collapse the directions the point is coarse-aligned in
  double coll[27];
  for (int t = 0; t < 27; ++t) coll[t] = 0.0;
  double den = ceff;
  for (int dk = -1; dk <= 1; ++dk)
    for (int dj = -1; dj <= 1; ++dj)
      for (int di = -1; di <= 1; ++di) {
        const int t = (dk + 1) * 9 + (dj + 1) * 3 + (di + 1);
        if (t == 13) continue;
        const int pi = fr[0] ? di : 0, pj = fr[1] ? dj : 0, pk = fr[2] ? dk : 0;
        const int tp = (pk + 1) * 9 + (pj + 1) * 3 + (pi + 1);
        if (tp == 13)
          den = __dsub_rn(den, a[t]);
        else
          coll[tp] = __dadd_rn(coll[tp], a[t]);
      }
  if (!(den > 0.0)) {
    atomicOr(err, E3_BADDEN);
    return;
  }
  // weight to each parent: sum over collapsed neighbours of coll times the
  // neighbour's weight to the same coarse point
  for (int m = 0; m < NPW3; ++m) {
    const int mc[3] = {m & 1, (m >> 1) & 1, (m >> 2) & 1};
    if ((mc[0] && !fr[0]) || (mc[1] && !fr[1]) || (mc[2] && !fr[2])) continue;
    // collapsed couplings live only at offsets that vary in the directions
    // the point lies between coarse points (integer bounds instead of an
    // FP64 test per neighbour; the skipped terms are exact zeros)
    double w = 0.0;
    for (int dk = -fr[2]; dk <= fr[2]; ++dk)
      for (int dj = -fr[1]; dj <= fr[1]; ++dj)
        for (int di = -fr[0]; di <= fr[0]; ++di) {
          const int t = (dk + 1) * 9 + (dj + 1) * 3 + (di + 1);
          if (t == 13) continue;
          const int dd[3] = {di, dj, dk};
          int gslot = 0;
          bool ok = true;
          for (int s = 0; s < 3; ++s) {
            if (!fr[s]) continue;                      // dd[s] == 0 here
            if (dd[s] == -1) ok = ok && mc[s] == 0;    // neighbour at the lower parent
            else if (dd[s] == 1) ok = ok && mc[s] == 1;
            else gslot |= mc[s] << s;                  // still between: same parent
          }
          if (!ok) continue;
          const double wn = F.P[gslot][o + off3(F, di, dj, dk)];
          w = __dadd_rn(w, __dmul_rn(coll[t], wn));
        }
    F.P[m][o] = w / den;
  }
}

// One thread per pair of points i = 2t + 1, 2t + 2 of a row (j and k fixed
// per block): the points of one pass then fill whole warps.
__global__ void k3_interp_weights(Lev3 F, int pass, int* err) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y + 1, k = blockIdx.z + 1;
  if (2 * t + 1 <= F.nx) weights_point(F, 2 * t + 1, j, k, pass, err);
  if (2 * t + 2 <= F.nx) weights_point(F, 2 * t + 2, j, k, pass, err);
}

// ---------------------------------------------------------------------------
// Galerkin product: one thread per coarse point computes its 14 stored
// entries from the definition A_c(I, I + d) = sum_f sum_g P(f, I) A(f, g)
// P(g, I + d) over fine f in the support of I and g in that of I + d.
// ---------------------------------------------------------------------------

// slot of fine point 2 I + e (e in -1..1 per direction) for parent I
__device__ __forceinline__ int support_slot(int ex, int ey, int ez) {
  return (ex == -1 ? 1 : 0) | ((ey == -1 ? 1 : 0) << 1) | ((ez == -1 ? 1 : 0) << 2);
}

// One thread per coarse point and stored entry (blockIdx.y = 14 (J - 1) + e):
// a block's threads share the entry, so their loops run in step.
__global__ void k3_rap(Lev3 F, Lev3 Cc, int* err) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x + 1, J = blockIdx.y / 14 + 1, K = blockIdx.z + 1;
  if (I > Cc.nx) return;
  const int oc = idx3(Cc, I, J, K);
  {
    const int e = blockIdx.y % 14;
    int di = 0, dj = 0, dk = 0;
    if (e > 0) {
      const int m = e - 1;
      if (m < 9) {
        dk = -1;
        dj = m / 3 - 1;
        di = m % 3 - 1;
      } else if (m < 12) {
        dj = -1;
        di = m - 10;
      } else {
        di = -1;
      }
    }
    const int I2 = I + di, J2 = J + dj, K2 = K + dk;
    double val = 0.0;
    if (I2 >= 1 && J2 >= 1 && K2 >= 1 && I2 <= Cc.nx && J2 <= Cc.ny && K2 <= Cc.nz) {
      // per direction only the pairs (e, h) with g = e + h - 2d in -1..1 can
      // contribute (fine g in the support of I + d); the loops visit exactly
      // those, in the order of the full 3 x 3 x 3 x 3 x 3 x 3 enumeration
      auto lo = [](int e, int d) { return max(-1, -1 - e + 2 * d); };
      auto hi = [](int e, int d) { return min(1, 1 - e + 2 * d); };
      for (int ez = -1; ez <= 1; ++ez)
        for (int ey = -1; ey <= 1; ++ey)
          for (int ex = -1; ex <= 1; ++ex) {
            if (lo(ex, di) > hi(ex, di) || lo(ey, dj) > hi(ey, dj) || lo(ez, dk) > hi(ez, dk))
              continue;
            const int fi = 2 * I + ex, fj = 2 * J + ey, fk = 2 * K + ez;
            if (fi > F.nx || fj > F.ny || fk > F.nz) continue;
            const int of = idx3(F, fi, fj, fk);
            // no test for zero weights: they add exact zeros, and an FP64
            // compare costs as much as the multiply-add on this part
            const double wf = F.P[support_slot(ex, ey, ez)][of];
            double s = 0.0;
            for (int hz = lo(ez, dk); hz <= hi(ez, dk); ++hz)
              for (int hy = lo(ey, dj); hy <= hi(ey, dj); ++hy)
                for (int hx = lo(ex, di); hx <= hi(ex, di); ++hx) {
                  const int gx = ex + hx - 2 * di, gy = ey + hy - 2 * dj, gz = ez + hz - 2 * dk;
                  const int gi = fi + hx, gj = fj + hy, gk = fk + hz;
                  if (gi < 1 || gj < 1 || gk < 1 || gi > F.nx || gj > F.ny || gk > F.nz) continue;
                  const int og = idx3(F, gi, gj, gk);
                  const double wg = F.P[support_slot(gx, gy, gz)][og];
                  const double afg =
                      (hx | hy | hz) == 0 ? F.C[of] : -coupling(F, of, hx, hy, hz);
                  s = fma(afg, wg, s);
                }
            val = fma(wf, s, val);
          }
    }
    if (e == 0) {
      if (!(val > 0.0) || !(val < INFINITY)) atomicOr(err, E3_NOTSPD);
      Cc.C[oc] = val;
      Cc.iC[oc] = 1.0 / val;
    } else {
      Cc.A[e - 1][oc] = -val;
    }
  }
}

// ---------------------------------------------------------------------------
// Smoothing, residual, restriction, interpolation
// ---------------------------------------------------------------------------

template <bool SEVEN, typename T>
__device__ __forceinline__ T nb_sum(const Lev3T<T>& L, const T* __restrict__ x, int o) {
  T s = T(0);
  if (SEVEN) {
    const int sx = 1, sy = L.px, sz = L.py * L.px;
    s = fma(L.A[12][o], x[o - sx], s);
    s = fma(L.A[12][o + sx], x[o + sx], s);
    s = fma(L.A[10][o], x[o - sy], s);
    s = fma(L.A[10][o + sy], x[o + sy], s);
    s = fma(L.A[4][o], x[o - sz], s);
    s = fma(L.A[4][o + sz], x[o + sz], s);
  } else {
#pragma unroll
    for (int dk = -1; dk <= 1; ++dk)
#pragma unroll
      for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
        for (int di = -1; di <= 1; ++di) {
          if (di == 0 && dj == 0 && dk == 0) continue;
          const int d = off3(L, di, dj, dk);
          s = fma(coupling(L, o, di, dj, dk), x[o + d], s);
        }
  }
  return s;
}

// A forward sweep from x = 0 (a coarse level after its restriction, the
// finest level of FP32 refinement or of a PCG preconditioner cycle): a point
// of colour c sees nonzero x only at neighbours of colours updated before c
// in the same sweep.  A neighbour at (di, dj, dk) differs from the point in
// colour by the parity flips f = 4|dk| + 2|dj| + |di| (eight colours), so
// its colour c ^ f precedes c exactly when the highest bit of f is set in
// c; with two colours (parity of i + j + k) every neighbour of colour 1 is
// of colour 0 and colour 0 has none.  nb_sum_zero skips the other terms:
// fma(a, 0, s) = s, so the sum equals nb_sum's (up to the sign of a zero).
__host__ __device__ constexpr bool zero_term3(int c, int di, int dj, int dk) {
  return (dk ? (c & 4) != 0 : dj ? (c & 2) != 0 : (c & 1) != 0);
}
// Checked by brute force over every colour and offset: the rule above keeps
// exactly the neighbours whose colour (c with the offset's parities flipped)
// precedes c, 0, 2, 6, 8, 18, 20, 24, 26 of them for colours 0..7.
constexpr bool zero_terms3_ok() {
  const int want[8] = {0, 2, 6, 8, 18, 20, 24, 26};
  for (int c = 0; c < 8; ++c) {
    int n = 0;
    for (int dk = -1; dk <= 1; ++dk)
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
          if (!di && !dj && !dk) continue;
          const int nb = c ^ ((dk ? 4 : 0) | (dj ? 2 : 0) | (di ? 1 : 0));
          if (zero_term3(c, di, dj, dk) != (nb < c)) return false;
          n += zero_term3(c, di, dj, dk) ? 1 : 0;
        }
    if (n != want[c]) return false;
  }
  return true;
}
static_assert(zero_terms3_ok(), "zero-start neighbour rule");

template <int C, typename T>
__device__ __forceinline__ T nb_sum27_zero(const Lev3T<T>& L, const T* __restrict__ x, int o) {
  T s = T(0);
#pragma unroll
  for (int dk = -1; dk <= 1; ++dk)
#pragma unroll
    for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
      for (int di = -1; di <= 1; ++di) {
        if (di == 0 && dj == 0 && dk == 0) continue;
        if (!zero_term3(C, di, dj, dk)) continue;
        const int d = off3(L, di, dj, dk);
        s = fma(coupling(L, o, di, dj, dk), x[o + d], s);
      }
  return s;
}

// One colour of a sweep, in place.  SEVEN: red-black, colour (i + j + k)
// parity (0-based); else colour 4 (k mod 2) + 2 (j mod 2) + (i mod 2).
// ZERO (SEVEN, forward sweep of a zero iterate): colour 0 has no nonzero
// neighbour, x = (b + 0) / C.
template <bool SEVEN, typename T, bool ZERO = false>
__global__ void k3_gs(Lev3T<T> L, int colour) {
  griddep_wait();
  const int ih = blockIdx.x * blockDim.x + threadIdx.x;
  int i0, j0, k0;
  if (SEVEN) {
    j0 = blockIdx.y;
    k0 = blockIdx.z;
    i0 = 2 * ih + ((j0 + k0 + colour) & 1);
  } else {
    j0 = 2 * blockIdx.y + ((colour >> 1) & 1);
    k0 = 2 * blockIdx.z + (colour >> 2);
    i0 = 2 * ih + (colour & 1);
  }
  if (i0 >= L.nx || j0 >= L.ny || k0 >= L.nz) return;
  const int o = idx3(L, i0 + 1, j0 + 1, k0 + 1);
  if (ZERO && colour == 0)
    L.x[o] = (L.b[o] + T(0)) * L.iC[o];
  else
    L.x[o] = (L.b[o] + nb_sum<SEVEN>(L, L.x, o)) * L.iC[o];
}

// Two colours of an eight-colour sweep in one launch: colours 2m and 2m + 1
// (the same parities of j and k, (cj, ck) = (m & 1, m >> 1)) differ only in the
// parity of i, so a point of one has neighbours of the other only within its
// own x-row; every other neighbour is of colours 2m + 2 .. 7 (forward) or
// 0 .. 2m - 1 (reverse), untouched by this launch.  One thread block per row:
// the first colour of the row, a barrier, the second.  Each point update is
// that of k3_gs<false>, so a sweep gives the same bits as eight launches.
template <typename T>
__global__ void __launch_bounds__(kT) k3_gs27_pair(Lev3T<T> L, int m, int reverse) {
  griddep_wait();
  const int j0 = 2 * blockIdx.x + (m & 1), k0 = 2 * blockIdx.y + (m >> 1);   // 0-based
  if (j0 >= L.ny || k0 >= L.nz) return;
  const int base = idx3(L, 0, j0 + 1, k0 + 1);
  for (int h = 0; h < 2; ++h) {
    const int ci = reverse ? 1 - h : h;
    for (int i0 = 2 * threadIdx.x + ci; i0 < L.nx; i0 += 2 * kT) {
      const int o = base + i0 + 1;
      L.x[o] = (L.b[o] + nb_sum<false>(L, L.x, o)) * L.iC[o];
    }
    __syncthreads();
  }
}

// The colour pair 2M, 2M + 1 of a forward 27-point sweep of a zero iterate
// (k3_gs27_pair's layout; each colour with only the terms nb_sum27_zero
// keeps).
template <int C, typename T>
__device__ __forceinline__ void gs27_row_zero(const Lev3T<T>& L, int base) {
  for (int i0 = 2 * threadIdx.x + (C & 1); i0 < L.nx; i0 += 2 * kT) {
    const int o = base + i0 + 1;
    L.x[o] = (L.b[o] + nb_sum27_zero<C>(L, L.x, o)) * L.iC[o];
  }
}

template <typename T, int M>
__global__ void __launch_bounds__(kT) k3_gs27_pair_zero(Lev3T<T> L) {
  griddep_wait();
  const int j0 = 2 * blockIdx.x + (M & 1), k0 = 2 * blockIdx.y + (M >> 1);   // 0-based
  if (j0 >= L.ny || k0 >= L.nz) return;
  const int base = idx3(L, 0, j0 + 1, k0 + 1);
  gs27_row_zero<2 * M>(L, base);
  __syncthreads();
  gs27_row_zero<2 * M + 1>(L, base);
  __syncthreads();
}

template <bool SEVEN, typename T>
__global__ void k3_residual(Lev3T<T> L) {
  griddep_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1, j = blockIdx.y + 1, k = blockIdx.z + 1;
  if (i > L.nx) return;
  const int o = idx3(L, i, j, k);
  L.r[o] = fma(-L.C[o], L.x[o], L.b[o]) + nb_sum<SEVEN>(L, L.x, o);
}

// b_c(I) = sum over the fine support of I of P(f, I) r(f); x_c = 0.
template <typename T>
__global__ void k3_restrict(Lev3T<T> F, Lev3T<T> Cc) {
  griddep_wait();
  const int I = blockIdx.x * blockDim.x + threadIdx.x + 1, J = blockIdx.y + 1, K = blockIdx.z + 1;
  if (I > Cc.nx) return;
  T s = T(0);
  for (int ez = -1; ez <= 1; ++ez)
    for (int ey = -1; ey <= 1; ++ey)
      for (int ex = -1; ex <= 1; ++ex) {
        const int fi = 2 * I + ex, fj = 2 * J + ey, fk = 2 * K + ez;
        if (fi > F.nx || fj > F.ny || fk > F.nz) continue;
        const int of = idx3(F, fi, fj, fk);
        s = fma(F.P[support_slot(ex, ey, ez)][of], F.r[of], s);
      }
  const int oc = idx3(Cc, I, J, K);
  Cc.b[oc] = s;
  Cc.x[oc] = T(0);
}

// x(f) += sum over f's parents of P(f, I) x_c(I).  A point has 1, 2, 4 or 8
// parents by the parities of i, j, k; each thread takes one point of each
// parity of i in turn (j and k are fixed per block), so the lanes of a warp
// always follow the same parents.
template <typename T>
__device__ __forceinline__ void interp_point(const Lev3T<T>& F, const Lev3T<T>& Cc, int i, int j, int k) {
  const int o = idx3(F, i, j, k);
  T s = T(0);
  for (int m = 0; m < NPW3; ++m) {
    const int cx = m & 1, cy = (m >> 1) & 1, cz = m >> 2;
    if ((cx && !(i & 1)) || (cy && !(j & 1)) || (cz && !(k & 1))) continue;
    const int I = (i & 1) ? (i - 1) / 2 + cx : i / 2;
    const int J = (j & 1) ? (j - 1) / 2 + cy : j / 2;
    const int K = (k & 1) ? (k - 1) / 2 + cz : k / 2;
    s = fma(F.P[m][o], Cc.x[idx3(Cc, I, J, K)], s);
  }
  F.x[o] += s;
}

template <typename T>
__global__ void k3_interp(Lev3T<T> F, Lev3T<T> Cc) {
  griddep_wait();
  const int t = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y + 1, k = blockIdx.z + 1;
  if (2 * t + 1 <= F.nx) interp_point(F, Cc, 2 * t + 1, j, k);
  if (2 * t + 2 <= F.nx) interp_point(F, Cc, 2 * t + 2, j, k);
}

// ---------------------------------------------------------------------------
// Norms (fixed grid, fixed order: deterministic) and the stop test
// ---------------------------------------------------------------------------

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[kNormThreads / 32];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = v;
  __syncthreads();
  v = lane < kNormThreads / 32 ? red[lane] : 0.0;
  if (w == 0)
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// what 0: ||b||^2; 1: ||b - A x||^2 (7-point finest level)
__global__ void k3_norm(Lev3 L, int what, double* __restrict__ partials) {
  griddep_wait();
  double acc = 0.0;
  const int n = L.nx * L.ny * L.nz;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int i = t % L.nx + 1, rest = t / L.nx, j = rest % L.ny + 1, k = rest / L.ny + 1;
    const int o = idx3(L, i, j, k);
    double v = L.b[o];
    if (what) v = fma(-L.C[o], L.x[o], v) + nb_sum<true>(L, L.x, o);
    acc = fma(v, v, acc);
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// The first sweep of a cycle on the finest (7-point) level, carrying the
// stop test of the cycle before it.  That cycle ended with a post-smoothing
// sweep in reverse colour order, whose last colour is colour 0; nothing has
// changed x since, so recomputing a colour-0 point gives the same bits and
// the sweep's first colour is a copy.  Its second colour updates each
// colour-1 point from its (unchanged) colour-0 neighbours, and
// C (x_new - x_old) there is the residual b - A x of the iterate the sweep
// reads (zero at colour 0 in the same evaluation).  Out of place: x is left
// as it was (the previous cycle's result, returned if the test stops the
// loop) and the swept iterate goes to `out`; the squared residual is summed
// per block into partials.  One thread per pair of points of a row (one of
// each colour), in k3_norm's fixed grid and order.
__global__ void __launch_bounds__(kNormThreads) k3_gs_norm(Lev3 L, double* __restrict__ out,
                                                           double* __restrict__ partials) {
  griddep_wait();
  const int hx = (L.nx + 1) / 2;
  const long n = long(hx) * L.ny * L.nz;
  double acc = 0.0;
  for (long t = long(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += long(gridDim.x) * blockDim.x) {
    const int ih = int(t % hx);
    const long rest = t / hx;
    const int j = int(rest % L.ny) + 1, k = int(rest / L.ny) + 1;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int i = 2 * ih + 1 + e;
      if (i > L.nx) continue;
      const int o = idx3(L, i, j, k);
      if (((i + j + k - 3) & 1) == 0) {
        out[o] = L.x[o];
        continue;
      }
      const double xn = (L.b[o] + nb_sum<true>(L, L.x, o)) * L.iC[o];
      out[o] = xn;
      const double r = L.C[o] * (xn - L.x[o]);
      acc = fma(r, r, acc);
    }
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

struct Scal3 {
  double bnorm2, rnorm2;
  double scale;             // FP32 refinement: the norm the FP32 right-hand side was divided by
  double rz, alpha, beta;   // PCG scalars
  double rnorm, rinv;       // sqrt(rnorm2) and its inverse (0 for a zero residual)
  int err;                  // E3_* bits set by setup kernels
};

__global__ void k3_norm_final(const double* __restrict__ partials, int n, Scal3* sc, int what) {
  griddep_wait();
  double acc = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) acc += partials[k];
  acc = block_sum(acc);
  if (threadIdx.x == 0) {
    if (what) {
      sc->rnorm2 = acc;
      sc->rnorm = sqrt(acc);
      sc->rinv = acc > 0.0 ? 1.0 / sc->rnorm : 0.0;
    }
    else
      sc->bnorm2 = acc;
  }
}

// ---------------------------------------------------------------------------
// FP32 V-cycles inside FP64 refinement (the mixed-precision extension on the
// 3D path): each step solves A e = r / ||r|| approximately with one FP32
// V-cycle from e = 0 and updates x += ||r|| e in FP64; the residual and the
// stop test stay FP64 on the finest level.
// ---------------------------------------------------------------------------

// r = b - A x on the FP64 finest level (the arithmetic of k3_norm, whose grid
// and summation order it shares), r^2 summed into block partials, and the
// FP32 finest level's right-hand side b32 = r / ||r_prev|| (the latest
// residual norm, sc->rnorm2) with x32 = 0.
__global__ void k3_refine_residual(Lev3 L, Lev3f Lf, const Scal3* __restrict__ sc,
                                   double* __restrict__ partials) {
  griddep_wait();
  const double inv = sc->rnorm2 > 0.0 ? 1.0 / sqrt(sc->rnorm2) : 0.0;
  double acc = 0.0;
  const int n = L.nx * L.ny * L.nz;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int i = t % L.nx + 1, rest = t / L.nx, j = rest % L.ny + 1, k = rest / L.ny + 1;
    const int o = idx3(L, i, j, k), of = idx3(Lf, i, j, k);
    const double v = fma(-L.C[o], L.x[o], L.b[o]) + nb_sum<true>(L, L.x, o);
    Lf.b[of] = float(v * inv);
    Lf.x[of] = 0.0f;
    acc = fma(v, v, acc);
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// The new residual norm; the previous one becomes the scale the right-hand
// side just cast was divided by.
__global__ void k3_refine_norm_final(const double* __restrict__ partials, int n, Scal3* sc) {
  griddep_wait();
  double acc = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) acc += partials[k];
  acc = block_sum(acc);
  if (threadIdx.x == 0) {
    sc->scale = sqrt(sc->rnorm2);
    sc->rnorm2 = acc;
  }
}

// x += scale * e on the finest level.
__global__ void k3_refine_update(Lev3 L, Lev3f Lf, const Scal3* __restrict__ sc) {
  griddep_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1, j = blockIdx.y + 1, k = blockIdx.z + 1;
  if (i > L.nx) return;
  const int o = idx3(L, i, j, k);
  L.x[o] = fma(sc->scale, double(Lf.x[idx3(Lf, i, j, k)]), L.x[o]);
}

// The FP32 copy of a level: operator, 1/C and interpolation rounded once
// from FP64, every plane whole (ring included).
__global__ void k3_downcast(Lev3 V, Lev3f F, int with_p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
  if (i > V.nx + 1) return;
  const int o = idx3(V, i, j, k), of = idx3(F, i, j, k);
  F.C[of] = float(V.C[o]);
  F.iC[of] = float(V.iC[o]);
  for (int m = 0; m < NA; ++m) F.A[m][of] = float(V.A[m][o]);
  if (with_p)
    for (int m = 0; m < NPW3; ++m) F.P[m][of] = float(V.P[m][o]);
}

// ---------------------------------------------------------------------------
// Conjugate gradients on the finest operator preconditioned by one symmetric
// V(nu, nu) cycle from zero (nu1 = nu2, post-smoothing colours reversed,
// R = P^T, exact coarsest solve: a symmetric positive definite M), in the
// textbook order of the oracle.  The finest level's b plane holds the
// residual r (the V-cycle's right-hand side) and its x plane z = M^{-1} r;
// the iterate X, the right-hand side B, the direction P and Q = A P are
// planes of their own.  Every kernel visits the points in k3_norm's grid and
// order, so the dot products are deterministic.
// ---------------------------------------------------------------------------

template <class Fn>
__device__ __forceinline__ double pcg_points(const Lev3& F, Fn f) {
  double acc = 0.0;
  const int n = F.nx * F.ny * F.nz;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int i = t % F.nx + 1, rest = t / F.nx, j = rest % F.ny + 1, k = rest / F.ny + 1;
    acc = f(idx3(F, i, j, k), acc);
  }
  return block_sum(acc);
}

// r = B - A X (in F.b), z = 0 (F.x), partials of r.r
__global__ void k3_pcg_init(Lev3 F, const double* __restrict__ X, const double* __restrict__ B,
                            double* __restrict__ partials) {
  const double sum = pcg_points(F, [&](int o, double acc) {
    const double r = fma(-F.C[o], X[o], B[o]) + nb_sum<true>(F, X, o);
    F.b[o] = r;
    F.x[o] = 0.0;
    return fma(r, r, acc);
  });
  if (threadIdx.x == 0) partials[blockIdx.x] = sum;
}

// Q = A P (the negated residual of P for a zero right-hand side), partials of P.Q
__global__ void k3_pcg_ap(Lev3 F, const double* __restrict__ P, double* __restrict__ Q,
                          double* __restrict__ partials) {
  griddep_wait();
  const double sum = pcg_points(F, [&](int o, double acc) {
    const double q = -(fma(-F.C[o], P[o], 0.0) + nb_sum<true>(F, P, o));
    Q[o] = q;
    return fma(P[o], q, acc);
  });
  if (threadIdx.x == 0) partials[blockIdx.x] = sum;
}

// X += alpha P, r -= alpha Q, z = 0, partials of r.r
__global__ void k3_pcg_xr(Lev3 F, double* __restrict__ X, const double* __restrict__ P,
                          const double* __restrict__ Q, const Scal3* __restrict__ sc,
                          double* __restrict__ partials) {
  griddep_wait();
  const double a = sc->alpha;
  const double sum = pcg_points(F, [&](int o, double acc) {
    X[o] = fma(a, P[o], X[o]);
    const double r = fma(-a, Q[o], F.b[o]);
    F.b[o] = r;
    F.x[o] = 0.0;
    return fma(r, r, acc);
  });
  if (threadIdx.x == 0) partials[blockIdx.x] = sum;
}

// partials of r.z
__global__ void k3_pcg_rz(Lev3 F, double* __restrict__ partials) {
  griddep_wait();
  const double sum = pcg_points(F, [&](int o, double acc) { return fma(F.b[o], F.x[o], acc); });
  if (threadIdx.x == 0) partials[blockIdx.x] = sum;
}

// P = z + beta P
__global__ void k3_pcg_p(Lev3 F, double* __restrict__ P, const Scal3* __restrict__ sc) {
  griddep_wait();
  const double beta = sc->beta;
  pcg_points(F, [&](int o, double acc) {
    P[o] = fma(beta, P[o], F.x[o]);
    return acc;
  });
}

// One block sums the partials; what 0: rz = sum, beta = 0 (first
// direction); 1: alpha = rz / sum (sum = P.Q); 2: beta = sum / rz, rz = sum
// (sum = r.z of the new residual).  A zero denominator gives 0.
__global__ void k3_pcg_scalar(const double* __restrict__ partials, int n, Scal3* sc, int what) {
  griddep_wait();
  double acc = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) acc += partials[k];
  acc = block_sum(acc);
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

// FP32 preconditioner: the FP32 finest level's right-hand side r / s and
// x32 = 0, s = ||r|| of the latest residual (sc->rnorm, sc->rinv, set once by
// k3_norm_final); then z = s e.
__global__ void k3_pcg_cast(Lev3 F, Lev3f Ff, const Scal3* __restrict__ sc) {
  griddep_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1, j = blockIdx.y + 1, k = blockIdx.z + 1;
  if (i > F.nx) return;
  const int of = idx3(Ff, i, j, k);
  Ff.b[of] = float(F.b[idx3(F, i, j, k)] * sc->rinv);
  Ff.x[of] = 0.0f;
}
__global__ void k3_pcg_uncast(Lev3 F, Lev3f Ff, const Scal3* __restrict__ sc) {
  griddep_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1, j = blockIdx.y + 1, k = blockIdx.z + 1;
  if (i > F.nx) return;
  F.x[idx3(F, i, j, k)] = sc->rnorm * double(Ff.x[idx3(Ff, i, j, k)]);
}

// ---------------------------------------------------------------------------
// Coarsest level: dense matrix and Cholesky factor (one block), solve
// ---------------------------------------------------------------------------

__global__ void k3_coarse_factor(Lev3 L0, double* __restrict__ lo, double* __restrict__ idiag,
                                 int* err) {
  const int nx = L0.nx, ny = L0.ny, n = nx * L0.ny * L0.nz;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) lo[e] = 0.0;
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const int i = r % nx + 1, j = (r / nx) % ny + 1, k = r / (nx * ny) + 1;
    const int o = idx3(L0, i, j, k);
    lo[size_t(r) * n + r] = L0.C[o];
    for (int dk = -1; dk <= 1; ++dk)
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
          if ((di | dj | dk) == 0) continue;
          const int i2 = i + di, j2 = j + dj, k2 = k + dk;
          if (i2 < 1 || j2 < 1 || k2 < 1 || i2 > nx || j2 > ny || k2 > L0.nz) continue;
          const int c = ((k2 - 1) * ny + (j2 - 1)) * nx + (i2 - 1);
          lo[size_t(r) * n + c] = -coupling(L0, o, di, dj, dk);
        }
  }
  __syncthreads();
  // right-looking Cholesky, lower triangle, row-major
  for (int c = 0; c < n; ++c) {
    __shared__ double piv;
    if (threadIdx.x == 0) {
      const double d = lo[size_t(c) * n + c];
      if (!(d > 0.0)) atomicOr(err, E3_NOTSPD);
      piv = sqrt(fmax(d, 1e-300));
      lo[size_t(c) * n + c] = piv;
      idiag[c] = 1.0 / piv;
    }
    __syncthreads();
    for (int r = c + 1 + threadIdx.x; r < n; r += blockDim.x) lo[size_t(r) * n + c] /= piv;
    __syncthreads();
    for (int e = threadIdx.x; e < (n - c - 1) * (n - c - 1); e += blockDim.x) {
      const int r = c + 1 + e / (n - c - 1), q = c + 1 + e % (n - c - 1);
      if (q <= r) lo[size_t(r) * n + q] -= lo[size_t(r) * n + c] * lo[size_t(q) * n + c];
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void k3_coarse_solve(Lev3T<T> L0, const double* __restrict__ lo,
                                const double* __restrict__ idiag) {
  griddep_wait();
  __shared__ double v[BMG_MAX_COARSEST];
  const int nx = L0.nx, ny = L0.ny, n = nx * ny * L0.nz;
  for (int r = threadIdx.x; r < n; r += blockDim.x)
    v[r] = double(L0.b[idx3(L0, r % nx + 1, (r / nx) % ny + 1, r / (nx * ny) + 1)]);
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const double y = v[j] * idiag[j];
    __syncthreads();
    if (threadIdx.x == 0) v[j] = y;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) v[i] = fma(-lo[size_t(i) * n + j], y, v[i]);
    __syncthreads();
  }
  for (int j = n - 1; j >= 0; --j) {
    const double xj = v[j] * idiag[j];
    __syncthreads();
    if (threadIdx.x == 0) v[j] = xj;
    for (int i = threadIdx.x; i < j; i += blockDim.x) v[i] = fma(-lo[size_t(j) * n + i], xj, v[i]);
    __syncthreads();
  }
  for (int r = threadIdx.x; r < n; r += blockDim.x)
    L0.x[idx3(L0, r % nx + 1, (r / nx) % ny + 1, r / (nx * ny) + 1)] = T(v[r]);
}

// dense (nz, ny, nx) <-> plane interior
__global__ void k3_pack(const double* __restrict__ src, double* __restrict__ dst, Lev3 L) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
  if (i >= L.nx) return;
  dst[idx3(L, i + 1, j + 1, k + 1)] = src[(size_t(k) * L.ny + j) * L.nx + i];
}
__global__ void k3_unpack(const double* __restrict__ src, double* __restrict__ dst, Lev3 L) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
  if (i >= L.nx) return;
  dst[(size_t(k) * L.ny + j) * L.nx + i] = src[idx3(L, i + 1, j + 1, k + 1)];
}

inline int cdiv(long a, long b) { return int((a + b - 1) / b); }
template <typename T>
inline dim3 grid_pts(const Lev3T<T>& L) { return dim3(cdiv(L.nx, kT), L.ny, L.nz); }

}  // namespace bmg3

using namespace bmg3;

struct bmg3_hierarchy {
  int L = 0;
  bmg_options opt{};
  std::vector<Lev3> lv;           // lv[0] coarsest ... lv[L-1] finest
  std::vector<Lev3f> lv32;        // FP32 copies (BMG_FP32_REFINE), else empty
  bool refine = false;            // FP32 V-cycles inside FP64 refinement
  bool pcg = false;               // BMG_SOLVER_PCG: CG preconditioned by the V-cycle
  double *pX = nullptr, *pB = nullptr, *pP = nullptr, *pQ = nullptr;   // PCG planes (finest layout)
  cudaGraph_t pcg_graph[2] = {nullptr, nullptr};          // first iteration, later ones
  cudaGraphExec_t pcg_exec[2] = {nullptr, nullptr};
  void* arena = nullptr;
  double *chol = nullptr, *chol_idiag = nullptr, *partials = nullptr;
  Scal3* sc = nullptr;
  Scal3* sc_host = nullptr;
  int* err = nullptr;
  int n0 = 0;
  int gs27_pairs = 1;             // 27-point sweeps as four colour-pair launches (1) or
                                  // eight colour launches (0; environment BMG3_GS27_PAIRS)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t gstream = nullptr;   // stream the graph was built for
  // FP64 V-cycles with the stop test in the next cycle's first fine sweep
  // (k3_gs_norm; environment BMG3_FUSED_NORM=0 at setup turns it off): the
  // finest iterate alternates between lv[L-1].x and x2, one step graph per
  // direction
  bool fused = false;
  double* x2 = nullptr;
  cudaGraph_t fgraph[2] = {nullptr, nullptr};
  cudaGraphExec_t fexec[2] = {nullptr, nullptr};
  double setup_ms = 0.0;
};

namespace {

double now_ms() {
  using clk = std::chrono::steady_clock;
  return std::chrono::duration<double, std::milli>(clk::now().time_since_epoch()).count();
}

void free3(bmg3_hierarchy* h) {
  if (!h) return;
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  for (int g = 0; g < 2; ++g) {
    if (h->fexec[g]) cudaGraphExecDestroy(h->fexec[g]);
    if (h->fgraph[g]) cudaGraphDestroy(h->fgraph[g]);
    if (h->pcg_exec[g]) cudaGraphExecDestroy(h->pcg_exec[g]);
    if (h->pcg_graph[g]) cudaGraphDestroy(h->pcg_graph[g]);
  }
  if (h->arena) cudaFree(h->arena);
  if (h->sc_host) cudaFreeHost(h->sc_host);
  delete h;
}

// One V(nu1, nu2) cycle (Algorithm 1), then ||b - A x||^2 of the finest level.
// One V(nu1, nu2) cycle (Algorithm 1) on the levels `lv` (FP64, or the FP32
// copies of FP32 refinement).
// skip_first: the finest level's first pre-smoothing sweep was already
// issued (k3_gs_norm).
// top_zero: the finest iterate is zero on entry (every coarser level's is
// after its restriction); the first forward sweep of a zero iterate takes
// the zero-start kernels (environment BMG_ZERO_START=0 turns them off).
template <typename T>
void enqueue_vcycle3(bmg3_hierarchy* h, std::vector<Lev3T<T>>& lv, cudaStream_t s,
                     bool skip_first = false, bool top_zero = false) {
  const int L = h->L;
  static const bool zero_start = [] {
    const char* e = std::getenv("BMG_ZERO_START");
    return !(e && e[0] == '0');
  }();
  auto sweep = [&](int l, int nu, bool reverse, bool zero) {
    const Lev3T<T>& V = lv[l];
    const bool seven = l == L - 1;
    const int nc = seven ? 2 : 8;
    for (int it = 0; it < nu; ++it) {
      const bool z = zero && zero_start && it == 0 && !reverse;
      if (seven) bmg::prof_begin(BMG_PROF_FINE_SMOOTH, s);
      if (!seven && h->gs27_pairs && z) {
        const dim3 g0((V.ny + 1) / 2, (V.nz + 1) / 2), g1(V.ny / 2, (V.nz + 1) / 2),
            g2((V.ny + 1) / 2, V.nz / 2), g3(V.ny / 2, V.nz / 2);
        bmg::launch_pdl(k3_gs27_pair_zero<T, 0>, g0, dim3(kT), 0, s, V);
        bmg::launch_pdl(k3_gs27_pair_zero<T, 1>, g1, dim3(kT), 0, s, V);
        bmg::launch_pdl(k3_gs27_pair_zero<T, 2>, g2, dim3(kT), 0, s, V);
        bmg::launch_pdl(k3_gs27_pair_zero<T, 3>, g3, dim3(kT), 0, s, V);
        count_launch(4);
        continue;
      }
      if (!seven && h->gs27_pairs) {
        for (int p0 = 0; p0 < 4; ++p0) {
          const int m = reverse ? 3 - p0 : p0;
          bmg::launch_pdl(k3_gs27_pair<T>, dim3((V.ny + 1 - (m & 1)) / 2, (V.nz + 1 - (m >> 1)) / 2), dim3(kT), 0, s, V, m, reverse ? 1 : 0);
          count_launch();
        }
        continue;
      }
      for (int c0 = 0; c0 < nc; ++c0) {
        const int c = reverse ? nc - 1 - c0 : c0;
        if (seven && z)
          bmg::launch_pdl(k3_gs<true, T, true>, dim3(cdiv((V.nx + 1) / 2, kT), V.ny, V.nz), dim3(kT), 0, s, V, c);
        else if (seven)
          bmg::launch_pdl(k3_gs<true, T>, dim3(cdiv((V.nx + 1) / 2, kT), V.ny, V.nz), dim3(kT), 0, s, V, c);
        else
          bmg::launch_pdl(k3_gs<false, T>, dim3(cdiv((V.nx + 1) / 2, kT), (V.ny + 1) / 2, (V.nz + 1) / 2), dim3(kT), 0, s, V, c);
        count_launch();
      }
      if (seven) bmg::prof_end(BMG_PROF_FINE_SMOOTH, s);
    }
  };
  bmg::NvtxRange cycle_range("vcycle3d", L - 1);
  for (int l = L - 1; l >= 1; --l) {
    bmg::NvtxRange r("restrict_leg", l);
    const Lev3T<T>& V = lv[l];
    sweep(l, h->opt.nu1 - (skip_first && l == L - 1 ? 1 : 0), false,
          !(skip_first && l == L - 1) && (l < L - 1 || top_zero));
    if (l == L - 1)
      bmg::launch_pdl(k3_residual<true, T>, dim3(grid_pts(V)), dim3(kT), 0, s, V);
    else
      bmg::launch_pdl(k3_residual<false, T>, dim3(grid_pts(V)), dim3(kT), 0, s, V);
    bmg::launch_pdl(k3_restrict<T>, dim3(grid_pts(lv[l - 1])), dim3(kT), 0, s, V, lv[l - 1]);
    count_launch(2);
  }
  bmg::launch_pdl(k3_coarse_solve<T>, dim3(1), dim3(256), 0, s, lv[0], h->chol, h->chol_idiag);
  count_launch();
  for (int l = 1; l < L; ++l) {
    bmg::NvtxRange r("interp_leg", l);
    bmg::launch_pdl(k3_interp<T>, dim3(cdiv((lv[l].nx + 1) / 2, kT), lv[l].ny, lv[l].nz), dim3(kT), 0, s, lv[l], lv[l - 1]);
    count_launch();
    sweep(l, h->opt.nu2, true, false);
  }
}

// FP32 refinement: the residual of the current x as the next FP32
// right-hand side, and its norm (the stop test).
void enqueue_refine_residual(bmg3_hierarchy* h, cudaStream_t s) {
  bmg::launch_pdl(k3_refine_residual, dim3(kNormBlocks), dim3(kNormThreads), 0, s, h->lv[h->L - 1], h->lv32[h->L - 1], h->sc, h->partials);
  bmg::launch_pdl(k3_refine_norm_final, dim3(1), dim3(kNormThreads), 0, s, h->partials, kNormBlocks, h->sc);
  count_launch(2);
}

// One step of the solve: a V-cycle and the stop test's residual norm, copied
// to the host.  FP64: the cycle on x, then ||b - A x||^2.  FP32 refinement:
// the FP32 cycle on the FP32 right-hand side, x += scale e, then the next
// right-hand side and ||b - A x||^2.
void enqueue_step(bmg3_hierarchy* h, cudaStream_t s) {
  const int L = h->L;
  if (h->refine) {
    // the refinement residual zeroed the FP32 finest iterate
    enqueue_vcycle3<float>(h, h->lv32, s, false, true);
    const Lev3& F = h->lv[L - 1];
    bmg::launch_pdl(k3_refine_update, dim3(grid_pts(F)), dim3(kT), 0, s, F, h->lv32[L - 1], h->sc);
    count_launch();
    enqueue_refine_residual(h, s);
  } else {
    enqueue_vcycle3<double>(h, h->lv, s);
    bmg::launch_pdl(k3_norm, dim3(kNormBlocks), dim3(kNormThreads), 0, s, h->lv[L - 1], 1, h->partials);
    bmg::launch_pdl(k3_norm_final, dim3(1), dim3(kNormThreads), 0, s, h->partials, kNormBlocks, h->sc, 1);
    count_launch(2);
  }
  cudaMemcpyAsync(h->sc_host, h->sc, sizeof(Scal3), cudaMemcpyDeviceToHost, s);
}

// The finest level's first pre-smoothing sweep (two colour launches, in
// place): the start of the first cycle of a fused solve.
void enqueue_first_sweep3(bmg3_hierarchy* h, cudaStream_t s) {
  const Lev3& V = h->lv[h->L - 1];
  bmg::prof_begin(BMG_PROF_FINE_SMOOTH, s);
  for (int c = 0; c < 2; ++c)
    bmg::launch_pdl(k3_gs<true, double>, dim3(cdiv((V.nx + 1) / 2, kT), V.ny, V.nz), dim3(kT), 0, s, V, c);
  bmg::prof_end(BMG_PROF_FINE_SMOOTH, s);
  count_launch(2);
}

// One step of a fused solve (h->fused): the rest of a cycle on the finest
// iterate in `in` (its first pre-sweep done), then the next cycle's first
// sweep from `in` into `out` with the stop test of `in`, copied to the host.
void enqueue_fused_step(bmg3_hierarchy* h, double* in, double* out, cudaStream_t s) {
  const int L = h->L;
  std::vector<Lev3> lv = h->lv;
  lv[L - 1].x = in;
  enqueue_vcycle3<double>(h, lv, s, true);
  bmg::prof_begin(BMG_PROF_NORM, s);
  bmg::launch_pdl(k3_gs_norm, dim3(kNormBlocks), dim3(kNormThreads), 0, s, lv[L - 1], out, h->partials);
  bmg::launch_pdl(k3_norm_final, dim3(1), dim3(kNormThreads), 0, s, h->partials, kNormBlocks, h->sc, 1);
  bmg::prof_end(BMG_PROF_NORM, s);
  count_launch(2);
  cudaMemcpyAsync(h->sc_host, h->sc, sizeof(Scal3), cudaMemcpyDeviceToHost, s);
}

// z = M^{-1} r: one V-cycle on the residual held in the finest level's b
// plane, from z = 0 in its x plane; on the FP32 copies (BMG_FP32_REFINE)
// with r / ||r|| cast down and z = ||r|| e cast back.
void enqueue_precond(bmg3_hierarchy* h, cudaStream_t s) {
  const int L = h->L;
  if (h->refine) {
    const Lev3& F = h->lv[L - 1];
    bmg::launch_pdl(k3_pcg_cast, dim3(grid_pts(F)), dim3(kT), 0, s, F, h->lv32[L - 1], h->sc);
    enqueue_vcycle3<float>(h, h->lv32, s, false, true);   // the cast zeroed z
    bmg::launch_pdl(k3_pcg_uncast, dim3(grid_pts(F)), dim3(kT), 0, s, F, h->lv32[L - 1], h->sc);
    count_launch(2);
  } else {
    enqueue_vcycle3<double>(h, h->lv, s, false, true);    // z = 0 from the update
  }
}

// One PCG iteration after a failed stop test: z = M^{-1} r, r.z (the first
// iteration takes p = z), p = z + beta p, q = A p, alpha, x += alpha p,
// r -= alpha q, ||r||^2 for the stop test, copied to the host.
void enqueue_pcg_iter(bmg3_hierarchy* h, bool first, cudaStream_t s) {
  const Lev3& F = h->lv[h->L - 1];
  enqueue_precond(h, s);
  bmg::launch_pdl(k3_pcg_rz, dim3(kNormBlocks), dim3(kNormThreads), 0, s, F, h->partials);
  bmg::launch_pdl(k3_pcg_scalar, dim3(1), dim3(kNormThreads), 0, s, h->partials, kNormBlocks, h->sc, first ? 0 : 2);
  bmg::launch_pdl(k3_pcg_p, dim3(kNormBlocks), dim3(kNormThreads), 0, s, F, h->pP, h->sc);
  bmg::launch_pdl(k3_pcg_ap, dim3(kNormBlocks), dim3(kNormThreads), 0, s, F, h->pP, h->pQ, h->partials);
  bmg::launch_pdl(k3_pcg_scalar, dim3(1), dim3(kNormThreads), 0, s, h->partials, kNormBlocks, h->sc, 1);
  bmg::launch_pdl(k3_pcg_xr, dim3(kNormBlocks), dim3(kNormThreads), 0, s, F, h->pX, h->pP, h->pQ, h->sc, h->partials);
  bmg::launch_pdl(k3_norm_final, dim3(1), dim3(kNormThreads), 0, s, h->partials, kNormBlocks, h->sc, 1);
  count_launch(7);
  cudaMemcpyAsync(h->sc_host, h->sc, sizeof(Scal3), cudaMemcpyDeviceToHost, s);
}

// Records fn(stream) as a graph (on a private stream) and instantiates it.
template <class Fn>
bool record_graph(cudaGraph_t* g, cudaGraphExec_t* e, Fn fn) {
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return false;
  bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) fn(cs);
  ok = cudaStreamEndCapture(cs, g) == cudaSuccess && ok;
  ok = ok && cudaGraphInstantiate(e, *g, 0) == cudaSuccess;
  cudaStreamDestroy(cs);
  if (!ok) cudaGetLastError();
  return ok;
}

// The PCG solve of bmg3_solve (BMG_SOLVER_PCG).
int solve_pcg(bmg3_hierarchy* h, const double* b, double* x, double tol, cudaStream_t s, int* iters,
              double* rel_out) {
  const Lev3& F = h->lv[h->L - 1];
  const dim3 g = dim3(cdiv(F.nx, kT), F.ny, F.nz);
  k3_pack<<<g, kT, 0, s>>>(b, h->pB, F);
  k3_pack<<<g, kT, 0, s>>>(b, F.b, F);
  k3_pack<<<g, kT, 0, s>>>(x, h->pX, F);
  k3_norm<<<kNormBlocks, kNormThreads, 0, s>>>(F, 0, h->partials);
  k3_norm_final<<<1, kNormThreads, 0, s>>>(h->partials, kNormBlocks, h->sc, 0);
  k3_pcg_init<<<kNormBlocks, kNormThreads, 0, s>>>(F, h->pX, h->pB, h->partials);
  k3_norm_final<<<1, kNormThreads, 0, s>>>(h->partials, kNormBlocks, h->sc, 1);
  count_launch(7);
  if (cudaMemcpyAsync(h->sc_host, h->sc, sizeof(Scal3), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return BMG_ECUDA;
  const double bn2 = h->sc_host->bnorm2;
  double rel = bn2 > 0.0 ? std::sqrt(h->sc_host->rnorm2 / bn2) : 0.0;
  int it = 0, rc = BMG_OK;
  if (bn2 == 0.0) {
    cudaMemsetAsync(x, 0, sizeof(double) * size_t(F.nx) * F.ny * F.nz, s);
    *iters = 0;
    *rel_out = 0.0;
    return cudaStreamSynchronize(s) == cudaSuccess ? BMG_OK : BMG_ECUDA;
  }
  const bool use_graph = !bmg::prof_active();
  if (use_graph && !h->pcg_exec[0]) {
    for (int k = 0; k < 2; ++k)
      if (!record_graph(&h->pcg_graph[k], &h->pcg_exec[k],
                        [&](cudaStream_t cs) { enqueue_pcg_iter(h, k == 0, cs); }))
        return BMG_ECUDA;
  }
  while (rel > tol && it < h->opt.max_cycles) {
    if (use_graph) {
      if (cudaGraphLaunch(h->pcg_exec[it == 0 ? 0 : 1], s) != cudaSuccess) return BMG_ECUDA;
    } else {
      enqueue_pcg_iter(h, it == 0, s);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return BMG_ECUDA;
    ++it;
    rel = std::sqrt(h->sc_host->rnorm2 / bn2);
    if (!std::isfinite(rel)) {
      rc = BMG_ENAN;
      break;
    }
  }
  if (!rc && rel > tol) rc = BMG_ENOCONV;
  k3_unpack<<<g, kT, 0, s>>>(h->pX, x, F);
  count_launch();
  if (cudaStreamSynchronize(s) != cudaSuccess) return BMG_ECUDA;
  *iters = it;
  *rel_out = rel;
  return rc;
}

int check_err(bmg3_hierarchy* h, cudaStream_t s) {
  if (cudaMemcpyAsync(h->sc_host, h->sc, sizeof(Scal3), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return BMG_ECUDA;
  const int e = h->sc_host->err;
  if (e & E3_BADK) {
    set_last_error("3D setup: a coefficient k is not finite and positive");
    return BMG_EINVAL;
  }
  if (e & E3_BADDEN) {
    set_last_error("3D setup: an interpolation denominator is not positive");
    return BMG_EINVAL;
  }
  if (e & E3_NOTSPD) {
    set_last_error("3D setup: a coarse operator is not positive definite");
    return BMG_EINVAL;
  }
  return BMG_OK;
}

}  // namespace

extern "C" {

int bmg3_setup(const double* k, int nx, int ny, int nz, const bmg_options* opt_in,
               bmg_stream_t stream, bmg3_hierarchy** out) {
  if (!out) return BMG_EINVAL;
  *out = nullptr;
  if (!k || nx < 2 || ny < 2 || nz < 2) return BMG_EINVAL;
  bmg_options opt;
  bmg_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (opt.nu1 < 0 || opt.nu2 < 0 || opt.nu1 + opt.nu2 < 1 || opt.max_cycles < 0 ||
      (opt.precision != BMG_FP64 && opt.precision != BMG_FP32_REFINE) || opt.smoother != BMG_SMOOTH_POINT ||
      (opt.solver != BMG_SOLVER_VCYCLE && !(opt.solver == BMG_SOLVER_PCG && opt.nu1 == opt.nu2)) ||
      opt.interp_residual_term || opt.aniso_r != 1.0 ||
      opt.cell_aspect != 1.0 || opt.bc_beta[0] >= 0.0 || opt.bc_beta[1] >= 0.0 ||
      opt.bc_beta[2] >= 0.0 || opt.bc_beta[3] >= 0.0 || opt.log_coefficients) {
    set_last_error("3D setup: options other than nu1, nu2, max_cycles, precision and solver must be the "
                   "defaults (BMG_SOLVER_PCG needs nu1 == nu2)");
    return BMG_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const double t0 = now_ms();
  std::vector<int> sx{nx}, sy{ny}, sz{nz};
  while (std::min({sx.back(), sy.back(), sz.back()}) > 3) {
    sx.push_back(sx.back() / 2);
    sy.push_back(sy.back() / 2);
    sz.push_back(sz.back() / 2);
  }
  bmg3_hierarchy* h = new (std::nothrow) bmg3_hierarchy();
  if (!h) return BMG_ENOMEM;
  h->opt = opt;
  if (const char* e = std::getenv("BMG3_GS27_PAIRS")) h->gs27_pairs = std::atoi(e) != 0;
  h->L = int(sx.size());
  const int L = h->L;
  h->n0 = sx.back() * sy.back() * sz.back();
  if (h->n0 > BMG_MAX_COARSEST) {
    set_last_error("3D setup: the coarsest level would hold %d unknowns (at most %d)", h->n0,
                   BMG_MAX_COARSEST);
    delete h;
    return BMG_EINVAL;
  }
  h->lv.assign(L, Lev3{});
  // sizes, then one zeroed arena
  size_t total = 0;
  auto reserve = [&](size_t bytes) {
    const size_t o = total;
    total += (bytes + 255) & ~size_t(255);
    return o;
  };
  std::vector<size_t> offs;
  for (int l = 0; l < L; ++l) {
    Lev3& V = h->lv[l];
    const int src = L - 1 - l;
    V.nx = sx[src];
    V.ny = sy[src];
    V.nz = sz[src];
    V.px = (V.nx + 2 + 15) / 16 * 16;
    V.py = V.ny + 2;
    const size_t pb = size_t(V.nz + 2) * V.py * V.px * sizeof(double);
    const int nplanes = 2 + NA + 3 + (l >= 1 ? NPW3 : 0);
    for (int p = 0; p < nplanes; ++p) offs.push_back(reserve(pb));
  }
  h->refine = opt.precision == BMG_FP32_REFINE;
  std::vector<size_t> offs32;
  if (h->refine) {
    h->lv32.assign(L, Lev3f{});
    for (int l = 0; l < L; ++l) {
      Lev3f& W = h->lv32[l];
      const Lev3& V = h->lv[l];
      W.nx = V.nx;
      W.ny = V.ny;
      W.nz = V.nz;
      W.px = (V.nx + 2 + 31) / 32 * 32;
      W.py = V.ny + 2;
      const size_t pb = size_t(W.nz + 2) * W.py * W.px * sizeof(float);
      const int nplanes = 2 + NA + 3 + (l >= 1 ? NPW3 : 0);
      for (int p = 0; p < nplanes; ++p) offs32.push_back(reserve(pb));
    }
  }
  h->pcg = opt.solver == BMG_SOLVER_PCG;
  size_t o_pcg = 0;
  if (h->pcg) {
    const Lev3& Ff = h->lv[L - 1];
    const size_t pbf = size_t(Ff.nz + 2) * Ff.py * Ff.px * sizeof(double);
    o_pcg = reserve(pbf);
    for (int q = 1; q < 4; ++q) reserve(pbf);
  }
  {
    const char* e = std::getenv("BMG3_FUSED_NORM");
    h->fused = !h->pcg && !h->refine && opt.nu1 >= 1 && opt.nu2 >= 1 && !(e && e[0] == '0');
  }
  size_t o_x2 = 0;
  if (h->fused) {
    const Lev3& Ff = h->lv[L - 1];
    o_x2 = reserve(size_t(Ff.nz + 2) * Ff.py * Ff.px * sizeof(double));
  }
  const size_t o_chol = reserve(sizeof(double) * size_t(h->n0) * h->n0);
  const size_t o_idiag = reserve(sizeof(double) * h->n0);
  const size_t o_part = reserve(sizeof(double) * kNormBlocks);
  const size_t o_sc = reserve(sizeof(Scal3));
  if (cudaMalloc(&h->arena, total) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return BMG_ENOMEM;
  }
  if (cudaMallocHost(&h->sc_host, sizeof(Scal3)) != cudaSuccess) {
    free3(h);
    return BMG_ENOMEM;
  }
  char* base = static_cast<char*>(h->arena);
  size_t pi = 0;
  for (int l = 0; l < L; ++l) {
    Lev3& V = h->lv[l];
    auto next = [&]() { return reinterpret_cast<double*>(base + offs[pi++]); };
    V.C = next();
    V.iC = next();
    for (int m = 0; m < NA; ++m) V.A[m] = next();
    V.x = next();
    V.b = next();
    V.r = next();
    for (int m = 0; m < NPW3; ++m) V.P[m] = l >= 1 ? next() : nullptr;
  }
  size_t qi = 0;
  for (int l = 0; l < int(h->lv32.size()); ++l) {
    Lev3f& W = h->lv32[l];
    auto next = [&]() { return reinterpret_cast<float*>(base + offs32[qi++]); };
    W.C = next();
    W.iC = next();
    for (int m = 0; m < NA; ++m) W.A[m] = next();
    W.x = next();
    W.b = next();
    W.r = next();
    for (int m = 0; m < NPW3; ++m) W.P[m] = l >= 1 ? next() : nullptr;
  }
  if (h->pcg) {
    const Lev3& Ff = h->lv[L - 1];
    const size_t pbf = (size_t(Ff.nz + 2) * Ff.py * Ff.px * sizeof(double) + 255) & ~size_t(255);
    h->pX = reinterpret_cast<double*>(base + o_pcg);
    h->pB = reinterpret_cast<double*>(base + o_pcg + pbf);
    h->pP = reinterpret_cast<double*>(base + o_pcg + 2 * pbf);
    h->pQ = reinterpret_cast<double*>(base + o_pcg + 3 * pbf);
  }
  if (h->fused) h->x2 = reinterpret_cast<double*>(base + o_x2);
  h->chol = reinterpret_cast<double*>(base + o_chol);
  h->chol_idiag = reinterpret_cast<double*>(base + o_idiag);
  h->partials = reinterpret_cast<double*>(base + o_part);
  h->sc = reinterpret_cast<Scal3*>(base + o_sc);
  h->err = &h->sc->err;
  if (cudaMemsetAsync(h->arena, 0, total, s) != cudaSuccess) {
    free3(h);
    return BMG_ECUDA;
  }
  const Lev3& F = h->lv[L - 1];
  k3_assemble<<<dim3(cdiv(F.nx, kT), F.ny, F.nz), kT, 0, s>>>(k, F, h->err);
  count_launch();
  for (int l = L - 1; l >= 1; --l) {
    const Lev3& V = h->lv[l];
    for (int pass = 0; pass <= 3; ++pass) {
      k3_interp_weights<<<dim3(cdiv((V.nx + 1) / 2, kT), V.ny, V.nz), kT, 0, s>>>(V, pass, h->err);
      count_launch();
    }
    {
      const Lev3& Cc = h->lv[l - 1];
      k3_rap<<<dim3(cdiv(Cc.nx, kT), 14 * Cc.ny, Cc.nz), kT, 0, s>>>(V, Cc, h->err);
    }
    count_launch();
  }
  k3_coarse_factor<<<1, 512, 0, s>>>(h->lv[0], h->chol, h->chol_idiag, h->err);
  count_launch();
  for (int l = 0; l < int(h->lv32.size()); ++l) {
    const Lev3& V = h->lv[l];
    k3_downcast<<<dim3(cdiv(V.nx + 2, kT), V.ny + 2, V.nz + 2), kT, 0, s>>>(V, h->lv32[l], l >= 1 ? 1 : 0);
    count_launch();
  }
  if (cudaGetLastError() != cudaSuccess) {
    free3(h);
    return BMG_ECUDA;
  }
  int rc = check_err(h, s);
  if (rc) {
    free3(h);
    return rc;
  }
  h->setup_ms = now_ms() - t0;
  *out = h;
  return BMG_OK;
}

int bmg3_solve(bmg3_hierarchy* h, const double* b, double* x, double tol, bmg_info* info,
               bmg_stream_t stream) {
  if (!h || !b || !x || !(tol >= 0.0)) return BMG_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const double t0 = now_ms();
  if (h->pcg) {
    int it = 0;
    double rel = 0.0;
    const int rc = solve_pcg(h, b, x, tol, s, &it, &rel);
    if (info) {
      info->cycles = it;
      info->threshold = 0;
      info->rel_resid = rel;
      info->setup_ms = h->setup_ms;
      info->solve_ms = now_ms() - t0;
      info->coarse_ctas = 1;
    }
    return rc;
  }
  const Lev3& F = h->lv[h->L - 1];
  const dim3 g = dim3(cdiv(F.nx, kT), F.ny, F.nz);
  k3_pack<<<g, kT, 0, s>>>(b, F.b, F);
  k3_pack<<<g, kT, 0, s>>>(x, F.x, F);
  k3_norm<<<kNormBlocks, kNormThreads, 0, s>>>(F, 0, h->partials);
  k3_norm_final<<<1, kNormThreads, 0, s>>>(h->partials, kNormBlocks, h->sc, 0);
  k3_norm<<<kNormBlocks, kNormThreads, 0, s>>>(F, 1, h->partials);
  k3_norm_final<<<1, kNormThreads, 0, s>>>(h->partials, kNormBlocks, h->sc, 1);
  count_launch(6);
  if (cudaMemcpyAsync(h->sc_host, h->sc, sizeof(Scal3), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return BMG_ECUDA;
  const double bn2 = h->sc_host->bnorm2;
  int cycles = 0;
  double rel = bn2 > 0.0 ? std::sqrt(h->sc_host->rnorm2 / bn2) : 0.0;
  int rc = BMG_OK;
  if (bn2 == 0.0) {
    cudaMemsetAsync(x, 0, sizeof(double) * size_t(F.nx) * F.ny * F.nz, s);
  } else if (h->fused) {
    // step k (1, 2, ...) works on the iterate in x (k odd) or x2 (k even)
    // and sweeps it into the other; after K steps the result is step K's
    // input (x for K = 0)
    double* buf[2] = {F.x, h->x2};
    const bool use_graph = !bmg::prof_active();
    if (use_graph && !h->fexec[0]) {
      for (int p = 0; p < 2; ++p)
        if (!record_graph(&h->fgraph[p], &h->fexec[p],
                          [&](cudaStream_t cs) { enqueue_fused_step(h, buf[p], buf[1 - p], cs); }))
          return BMG_ECUDA;
    }
    if (rel > tol && h->opt.max_cycles > 0) enqueue_first_sweep3(h, s);
    while (rel > tol && cycles < h->opt.max_cycles) {
      const int p = cycles & 1;
      if (use_graph) {
        if (cudaGraphLaunch(h->fexec[p], s) != cudaSuccess) return BMG_ECUDA;
      } else {
        enqueue_fused_step(h, buf[p], buf[1 - p], s);
      }
      if (cudaStreamSynchronize(s) != cudaSuccess) return BMG_ECUDA;
      ++cycles;
      rel = std::sqrt(h->sc_host->rnorm2 / bn2);
      if (!std::isfinite(rel)) {
        rc = BMG_ENAN;
        break;
      }
    }
    if (!rc && rel > tol) rc = BMG_ENOCONV;
    k3_unpack<<<g, kT, 0, s>>>(cycles == 0 ? F.x : buf[(cycles - 1) & 1], x, F);
    count_launch();
  } else {
    // one cycle as a graph, recorded on a private stream (stream launches
    // while kernel classes are being timed)
    const bool use_graph = !bmg::prof_active();
    if (use_graph && !h->gexec) {
      cudaStream_t cs;
      if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return BMG_ECUDA;
      bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) enqueue_step(h, cs);
      ok = cudaStreamEndCapture(cs, &h->graph) == cudaSuccess && ok;
      ok = ok && cudaGraphInstantiate(&h->gexec, h->graph, 0) == cudaSuccess;
      cudaStreamDestroy(cs);
      if (!ok) {
        cudaGetLastError();
        return BMG_ECUDA;
      }
    }
    // FP32 refinement: the first right-hand side is the initial residual
    if (h->refine && rel > tol && h->opt.max_cycles > 0) enqueue_refine_residual(h, s);
    while (rel > tol && cycles < h->opt.max_cycles) {
      if (use_graph) {
        if (cudaGraphLaunch(h->gexec, s) != cudaSuccess) return BMG_ECUDA;
      } else {
        enqueue_step(h, s);
      }
      if (cudaStreamSynchronize(s) != cudaSuccess) return BMG_ECUDA;
      ++cycles;
      rel = std::sqrt(h->sc_host->rnorm2 / bn2);
      if (!std::isfinite(rel)) {
        rc = BMG_ENAN;
        break;
      }
    }
    if (!rc && rel > tol) rc = BMG_ENOCONV;
    k3_unpack<<<g, kT, 0, s>>>(F.x, x, F);
    count_launch();
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return BMG_ECUDA;
  if (info) {
    info->cycles = cycles;
    info->threshold = 0;
    info->rel_resid = rel;
    info->setup_ms = h->setup_ms;
    info->solve_ms = now_ms() - t0;
    info->coarse_ctas = 1;
  }
  return rc;
}

void bmg3_destroy(bmg3_hierarchy* h) { free3(h); }

int bmg3_num_levels(const bmg3_hierarchy* h, int* n) {
  if (!h || !n) return BMG_EINVAL;
  *n = h->L;
  return BMG_OK;
}

int bmg3_level_shape(const bmg3_hierarchy* h, int level, int* nx, int* ny, int* nz) {
  if (!h || level < 0 || level >= h->L || !nx || !ny || !nz) return BMG_EINVAL;
  *nx = h->lv[level].nx;
  *ny = h->lv[level].ny;
  *nz = h->lv[level].nz;
  return BMG_OK;
}

static int copy_planes(const Lev3& V, double* const* planes, int np, double* out) {
  const size_t pb = size_t(V.nz + 2) * V.py * V.px;
  std::vector<double> buf(pb);
  const size_t n = size_t(V.nx) * V.ny * V.nz;
  for (int p = 0; p < np; ++p) {
    if (cudaMemcpy(buf.data(), planes[p], pb * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      return BMG_ECUDA;
    for (int k = 0; k < V.nz; ++k)
      for (int j = 0; j < V.ny; ++j)
        for (int i = 0; i < V.nx; ++i)
          out[p * n + (size_t(k) * V.ny + j) * V.nx + i] = buf[idx3(V, i + 1, j + 1, k + 1)];
  }
  return BMG_OK;
}

int bmg3_level_stencil(const bmg3_hierarchy* h, int level, double* host_out) {
  if (!h || level < 0 || level >= h->L || !host_out) return BMG_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return BMG_ECUDA;
  const Lev3& V = h->lv[level];
  double* planes[1 + NA];
  planes[0] = V.C;
  for (int m = 0; m < NA; ++m) planes[1 + m] = V.A[m];
  return copy_planes(V, planes, 1 + NA, host_out);
}

int bmg3_level_interp(const bmg3_hierarchy* h, int level, double* host_out) {
  if (!h || level < 1 || level >= h->L || !host_out) return BMG_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return BMG_ECUDA;
  const Lev3& V = h->lv[level];
  return copy_planes(V, V.P, NPW3, host_out);
}

}  // extern "C"
