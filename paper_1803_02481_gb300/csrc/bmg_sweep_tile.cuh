// Tile body of the one-kernel multicolour Gauss-Seidel sweep, shared by the
// single-problem and the batched kernels.
//
// A thread block owns a TX x TY tile.  It loads the old iterate on the tile
// plus a halo of NC columns and 2 rows into shared memory, then relaxes the
// colours in order: colour k (0-based) is updated on the tile grown by
// (colour_grow_x(NC, k), colour_grow_y(NC, k)) cells, so the last colour's
// neighbours of earlier colours are all available without reading another
// block's new values.  The points a block relaxes outside its tile are
// recomputed by the neighbouring block from the same old values, so every
// block sees exactly what an in-place sweep would see.  The new iterate goes
// to a second buffer (old and new never alias); only the tile is written.
// Per-point arithmetic is gs_load/gs_apply.
#pragma once

#include "bmg_internal.h"

namespace bmg {

// Sub-lattice masks of the colours in sweep order (bit 2*pj + pi: 0-based
// row parity pj, column parity pi), 4 bits per colour.
__host__ __device__ constexpr unsigned rb_order(bool reverse) { return reverse ? 0x96u : 0x69u; }
__host__ __device__ constexpr unsigned four_order(bool reverse) {
  return reverse ? 0x1248u : 0x8421u;
}

// Growth of colour phase k of nc (2: rb_order, 4: four_order, either
// direction) for a sweep that relaxes each tile once.  A later phase reads
// an earlier phase's points at offsets whose x part is +-1 exactly when the
// two sub-lattices differ in column parity and whose y part is +-1 exactly
// when they differ in row parity; the earlier phase must cover the later
// one's region grown by those amounts.  Red-black: (1, 1), (0, 0).  Four
// colours (0,0), (0,1), (1,0), (1,1) of (row, column) parities or the
// reverse: (3, 1), (2, 1), (1, 0), (0, 0).  Every phase needs old values one
// cell beyond its region: nc halo columns and 2 halo rows.
__host__ __device__ constexpr int colour_grow_x(int nc, int k) { return nc - 1 - k; }
__host__ __device__ constexpr int colour_grow_y(int nc, int k) {
  return nc == 4 ? (k < 2 ? 1 : 0) : nc - 1 - k;
}
constexpr int kColourHaloRows = 2;

// A forward sweep (rb_order(false), four_order(false)) from x = 0: phase k
// sees nonzero x only at points of the colours updated before it in the same
// sweep.  Neighbour-term mask of phase k (the bits of gs_apply_masked): the
// point's (row, column) parities are (k >> 1, k & 1) with four colours; a
// neighbour differing in (row, column) parity by (dr, dc) has colour
// 2 (pr ^ dr) + (pc ^ dc), and counts if that colour comes before k.  With
// two colours the second phase's neighbours are all of the first.
__host__ __device__ constexpr unsigned zero_start_mask(bool nine, int k) {
  if (!nine) return k == 0 ? 0u : 0x0Fu;
  return ((2 * (k >> 1) + ((k & 1) ^ 1) < k) ? 0x03u : 0u) |
         ((2 * ((k >> 1) ^ 1) + (k & 1) < k) ? 0x0Cu : 0u) |
         ((2 * ((k >> 1) ^ 1) + ((k & 1) ^ 1) < k) ? 0xF0u : 0u);
}
static_assert(zero_start_mask(true, 0) == 0u && zero_start_mask(true, 1) == 0x03u &&
                  zero_start_mask(true, 2) == 0xFCu && zero_start_mask(true, 3) == 0xFFu,
              "four-colour zero-start masks");

// NRM (5-point, forward order, double): the sweep that carries the stop test
// (the same argument as the TMA sweep's: after a reverse-order sweep the
// first colour's update is a no-op, so that phase is skipped, and the second
// phase's C (x_new - x_old) is the residual of the iterate read); the squared
// residual is summed per block into nrm[by * gridDim.x + bx].
template <typename T, bool NINE, int TX, int TY, int NT, int UB = (NINE ? 3 : 1), bool NRM = false>
__device__ __forceinline__ void sweep_tile(const LevelV<T>& L, const T* __restrict__ xin,
                                           T* __restrict__ xout, unsigned order, int bx, int by,
                                           double* __restrict__ nrm = nullptr) {
  static_assert(!NRM || (!NINE && UB == 1), "the fused stop test is a red-black sweep");
  double nacc = 0.0;
  constexpr int NC = NINE ? 4 : 2;
  constexpr int H = NC, HY = kColourHaloRows;   // halo columns, halo rows
  constexpr int SX = TX + 2 * H, SY = TY + 2 * HY;
  __shared__ T xs[SY * SX];
  const int nx = L.nx, ny = L.ny, p = L.pitch;
  // domain coordinates of shared-memory cell (0, 0)
  const int ib = bx * TX + 1 - H;
  const int jb = by * TY + 1 - HY;

  for (int e = threadIdx.x; e < SX * SY; e += NT) {
    const int r = e / SX, c = e - r * SX;
    const int i = ib + c, j = jb + r;
    T v = T(0);
    if (i >= 0 && i <= nx + 1 && j >= 0 && j <= ny + 1) v = xin[j * p + i];
    xs[e] = v;
  }
  __syncthreads();

#pragma unroll
  for (int k = 0; k < NC; ++k) {
    if (NRM && k == 0) continue;
    const unsigned mask = (order >> (4 * k)) & 0xFu;
    const int gx = colour_grow_x(NC, k), gy = colour_grow_y(NC, k);
    const int r0 = HY - gy, r1 = HY + TY + gy;   // region rows [r0, r1)
    const int c0 = H - gx, c1 = H + TX + gx;
#pragma unroll
    for (int sl = 0; sl < 4; ++sl) {
      if (!(mask & (1u << sl))) continue;
      const int pj = sl >> 1, pi = sl & 1;
      // first region row/col whose 0-based domain index has the right parity
      const int rf = r0 + ((pj + 1 - jb - r0) & 1);
      const int cf = c0 + ((pi + 1 - ib - c0) & 1);
      const int nr = (r1 - rf + 1) >> 1, ncol = (c1 - cf + 1) >> 1;
      const int npts = nr * ncol;
      // U points per thread per step: all their coefficient loads are issued
      // before any update, so the loads overlap instead of serialising (a
      // win for the 9-point stencil; for 5 points the extra registers cost
      // more occupancy than the overlap gains, measured).
      constexpr int U = UB;
      for (int t0 = threadIdx.x; t0 < npts; t0 += NT * U) {
        GsCoef<T, NINE> cf_[U];
        T cc[U];
        int sp[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int t = t0 + u * NT;
          const int rr = t / ncol;
          const int r = rf + 2 * rr, c = cf + 2 * (t - rr * ncol);
          const int i = ib + c, j = jb + r;
          ok[u] = t < npts && i >= 1 && i <= nx && j >= 1 && j <= ny;
          sp[u] = r * SX + c;
          if (ok[u]) {
            const int o = j * p + i;
            cf_[u] = gs_load<T, NINE>(L, o, __ldg(L.b + o));
            if (NRM) cc[u] = __ldg(L.C + o);
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (!ok[u]) continue;
          T* xp = xs + sp[u];
          const T xn = gs_apply<T, NINE>(cf_[u], [&](int dx, int dy) { return xp[dx + dy * SX]; });
          if (NRM && k == NC - 1) {
            const double rv = double(cc[u]) * double(xn - *xp);
            nacc = fma(rv, rv, nacc);
          }
          *xp = xn;
        }
      }
    }
    __syncthreads();
  }

  for (int e = threadIdx.x; e < TX * TY; e += NT) {
    const int r = e / TX, c = e - r * TX;
    const int i = ib + H + c, j = jb + HY + r;
    if (i <= nx && j <= ny) xout[j * p + i] = xs[(r + HY) * SX + c + H];
  }
  if (NRM) {
    // fixed reduction tree: warps, then warp sums in order
    __shared__ double wsum[NT / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) nacc += __shfl_xor_sync(0xffffffffu, nacc, off);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = nacc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0;
      for (int w = 0; w < NT / 32; ++w) a += wsum[w];
      nrm[by * gridDim.x + bx] = a;
    }
  }
}


}  // namespace bmg
