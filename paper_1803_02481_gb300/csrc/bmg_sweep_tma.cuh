// Persistent, TMA-staged multicolour Gauss-Seidel sweep (smoothing of
// Algorithm 1): red-black on 5-point levels, four colours on 9-point levels.
//
// Persistent blocks (a few per SM) walk the level's TX x TY tiles.  For each
// tile, one thread issues 2-D bulk tensor copies (cp.async.bulk.tensor) of
// the tile plus a halo: the old iterate and the planes 1/C, W, S, b (and SW,
// NW on 9-point levels).  They land in a shared-memory stage and complete on
// that stage's mbarrier.  With two stages, the block relaxes tile t out of
// one while the copies of its next tile fill the other; with one stage,
// the other blocks on the SM do their arithmetic while a block waits.
//
// The relaxation itself is a redundant-halo scheme: colour phase k is
// updated on the tile grown by (GX_k, GY_k) cells, so no block reads another
// block's new values.  The new iterate goes to a second buffer.  Per-point
// arithmetic is gs_apply, as in every other kernel, so the result is
// bit-identical to theirs.
//
// Growth.  A point of a later phase reads the points of an earlier phase at
// offsets (dx, dy) with |dx| = 1 exactly when the two sub-lattices differ in
// column parity and |dy| = 1 exactly when they differ in row parity, so the
// earlier phase must be relaxed on the later phase's region grown by those
// amounts.  Red-black (5-point): (1, 1) then (0, 0).  Four colours in the
// order (0,0), (0,1), (1,0), (1,1) of (row, column) parities, or its reverse:
// (3, 1), (2, 1), (1, 0), (0, 0) -- the first two phases differ from the
// last in column parity, so the growth is mostly along x, and the tile
// needs two halo rows instead of four.
//
// Staged box: rows j0-HY .. j0+TY+HY-1 and columns i0-HA .. i0+TX+HA-1 of
// each plane, (i0, j0) the tile's first interior point; HY = 2 rows and
// HA >= NPH columns (old values one cell beyond the widest phase region).
// HA is a whole number of 16-byte units, which keeps the box's first column
// on a 16-byte boundary (interior rows start on a 128-byte boundary).  Rows and columns
// outside the plane read as zero, the Dirichlet ghost value.
//
// Every wait on an mbarrier gives up after one second: the block then sets
// DEV_TIMEOUT in the error word, waits (again bounded) for its copies in
// flight and returns.
//
// Stop-test residual inside a sweep (NRM, prescaled red-black levels).  Let
// the previous sweep of the level end with colour c, and nothing change the
// iterate since.  Then every point of c satisfies its prescaled equation
// exactly: recomputing its update from the same neighbours gives the same
// bits, so C (x_new - x_old) = 0 there.  A sweep whose phases are
// (c, other colour) therefore leaves c unchanged in its first phase, which it
// skips (the staged values of c, ring included, are already the phase's
// result), and in its second phase C (x_new - x_old) at each point is that
// point's residual b - A x of the iterate before the sweep, evaluated in the
// prescaled form
// C (b/C + sum_X (a_X/C) x_X - x).  The sweep sums its square over the
// tile interiors (every point once) into one partial per block; C is read
// from global memory before the tile's copies are waited for.
#pragma once

#include <cuda.h>

#include "bmg_internal.h"
#include "bmg_sweep_tile.cuh"

namespace bmg {

namespace tma_detail {

__device__ __forceinline__ unsigned saddr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(saddr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(saddr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}

// Waits for the phase of `bar` with the given parity to complete; false
// after about one second (and, should the global timer not advance, after
// 2^32 polls).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint64_t n = 1; !mbar_try_wait(bar, parity); ++n) {
    if (globaltimer_ns() - t0 > 1000000000ull || n > (1ull << 32)) return false;
  }
  return true;
}

// 2-D tiled bulk tensor copy global -> shared, completing on `bar`.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(saddr(bar))
      : "memory");
}

}  // namespace tma_detail

// Halo rows of every staged box (both colour schemes grow by at most one
// row before the last phase; colour_grow_x/y give the growth).
constexpr int kTmaHaloRows = kColourHaloRows;

// Shape of the staged tile.  NPH colour phases (2 on 5-point levels, 4 on
// 9-point levels) need kTmaHaloRows halo rows and at least NPH halo columns;
// HA columns are staged so that the box start stays 16-byte aligned.
template <typename T, bool NINE, int TX, int TY, int NSTAGE = 2, bool PRE = false>
struct TmaTile {
  static constexpr int NPH = NINE ? 4 : 2;                  // colour phases
  static constexpr int ALIGN = int(16 / sizeof(T));        // elements per 16 bytes
  static constexpr int HA = NPH > ALIGN ? NPH : ALIGN;      // halo columns staged on each side
  static constexpr int HY = kTmaHaloRows;                   // halo rows staged above and below
  static constexpr int BW = TX + 2 * HA;                    // box width (elements)
  static constexpr int BH = TY + 2 * HY;                    // box height
  static constexpr int PLANE = BW * BH;                     // elements of one staged plane
  // x, 1/C, W, S, b (, SW, NW); prescaled: x, b/C, W/C, S/C, E/C, N/C
  static constexpr int NPL = PRE ? 6 : (NINE ? 7 : 5);
  static constexpr unsigned STAGE_BYTES = unsigned(NPL * PLANE * sizeof(T));
  static constexpr size_t SMEM = NSTAGE * size_t(STAGE_BYTES);
  static_assert(NSTAGE == 1 || NSTAGE == 2, "one or two stages");
  static_assert(TX % 4 == 0 && TY % 2 == 0, "tile sides keep colours and TMA alignment");
  static_assert(HA % ALIGN == 0 && HA % 2 == 0 && HY % 2 == 0,
                "box start aligned, colour parity kept");
  static_assert(colour_grow_x(NPH, 0) + 1 <= HA && colour_grow_y(NPH, 0) + 1 <= HY,
                "old values staged one cell beyond the widest phase region");
  static_assert(BW <= 256 && BH <= 256, "TMA box sides are at most 256 elements");
  static_assert((BW * sizeof(T)) % 16 == 0, "TMA box rows are multiples of 16 bytes");
  static_assert((PLANE * sizeof(T)) % 128 == 0, "staged planes start 128-byte aligned");
};

// Planes a TMA sweep stages, in their order in a stage (a prescaled level:
// x, b/C, W/C, S/C, E/C, N/C in the slots of x, 1/C, W, S, b, SW).
enum TmaPlane { TP_X = 0, TP_IC, TP_W, TP_S, TP_B, TP_SW, TP_NW };

// PRE: the level is prescaled (5-point only); the seven map parameters then
// carry x, b/C, W/C, S/C, E/C, N/C and an unused one.  NRM (with PRE): the
// second colour phase also sums (C (x_new - x_old))^2, C read from `cdiag`,
// into nrm[blockIdx.x].
// ZERO: a forward sweep whose input iterate is zero (a coarse level after the
// restriction, an FP32 finest level after the refinement residual, the
// finest level of a PCG preconditioner cycle): x is not staged, each phase
// applies only the neighbour terms of the colours updated before it
// (zero_start_mask; on a prescaled level the first phase's value is b/C),
// and the phases write zero at the points of their regions outside the grid
// (the Dirichlet values the staged ghosts would hold) -- the same values as
// the plain sweep of a zero iterate.
template <typename T, bool NINE, int TX, int TY, int NT, int MINB, int NSTAGE, bool PRE = false,
          bool NRM = false, bool ZERO = false>
__global__ void __launch_bounds__(NT, MINB)
    k_sweep_tma(const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap mic,
                const __grid_constant__ CUtensorMap mw, const __grid_constant__ CUtensorMap ms,
                const __grid_constant__ CUtensorMap mb, const __grid_constant__ CUtensorMap msw,
                const __grid_constant__ CUtensorMap mnw, LevelV<T> L, T* __restrict__ xout,
                unsigned order, int* __restrict__ err, const T* __restrict__ cdiag,
                double* __restrict__ nrm) {
  griddep_wait();
  using namespace tma_detail;
  static_assert(!(PRE && NINE), "prescaled levels are 5-point");
  static_assert(!NRM || PRE, "the fused residual is taken on prescaled levels");
  static_assert(!(ZERO && NRM), "the stop-test sweep reads a converging iterate");
  using G = TmaTile<T, NINE, TX, TY, NSTAGE, PRE>;
  constexpr int BW = G::BW, HA = G::HA, HY = G::HY, PL = G::PLANE, NPH = G::NPH;
  // NRM: the last phase relaxes the tile interior; each of its two
  // sub-lattices has (TY / 2) x (TX / 2) points, at most KU per thread
  constexpr int QX = TX / 2, NQ = QX * (TY / 2), KU = (NQ + NT - 1) / NT;
  const unsigned last_mask = (order >> (4 * (NPH - 1))) & 0xFu;
  double nacc = 0.0;
  extern __shared__ __align__(128) unsigned char tma_smem[];
  __shared__ __align__(8) uint64_t bar[2];
  const int nx = L.nx, ny = L.ny, p = L.pitch;
  const int ntx = (nx + TX - 1) / TX;
  const int ntiles = ntx * ((ny + TY - 1) / TY);
  const int tid = threadIdx.x;
  T* const stage0 = reinterpret_cast<T*>(tma_smem);
  // with one stage, both names denote it (stage1 is never selected)
  T* const stage1 = reinterpret_cast<T*>(tma_smem + (NSTAGE == 2 ? G::STAGE_BYTES : 0));

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();

  // Thread 0: stage the box of tile t into stage s.
  auto issue = [&](int s, int t) {
    const int bx = t % ntx, by = t / ntx;
    const int X = bx * TX + 1 - HA + base_shift<T>();   // tensor column of the box start
    const int Y = by * TY + 1 - HY;                     // tensor row (= j) of the box start
    T* d = s ? stage1 : stage0;
    uint64_t* b = &bar[s];
    mbar_expect_tx(b, G::STAGE_BYTES - (ZERO ? unsigned(PL * sizeof(T)) : 0u));
    if (!ZERO) tma_load_2d(d + TP_X * PL, &mx, X, Y, b);
    tma_load_2d(d + TP_IC * PL, &mic, X, Y, b);
    tma_load_2d(d + TP_W * PL, &mw, X, Y, b);
    tma_load_2d(d + TP_S * PL, &ms, X, Y, b);
    tma_load_2d(d + TP_B * PL, &mb, X, Y, b);
    if (PRE) tma_load_2d(d + TP_SW * PL, &msw, X, Y, b);
    if (NINE) {
      tma_load_2d(d + TP_SW * PL, &msw, X, Y, b);
      tma_load_2d(d + TP_NW * PL, &mnw, X, Y, b);
    }
  };

  // Two stages: the copies of the next tile are issued before the current
  // one is relaxed.  One stage: after it (more blocks per SM then overlap
  // one block's copies with another's arithmetic).  Stage s serves
  // iterations it with it % NSTAGE == s; its mbarrier phase is it / NSTAGE.
  int t = blockIdx.x;
  if (tid == 0 && t < ntiles) issue(0, t);
  for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
    const int s = NSTAGE == 2 ? (it & 1) : 0;
    const unsigned parity = unsigned(it / NSTAGE) & 1u;
    const int tn = t + gridDim.x;
    if (NSTAGE == 2 && tid == 0 && tn < ntiles) issue(s ^ 1, tn);
    const int bx = t % ntx, by = t / ntx;
    const int i0 = bx * TX + 1, j0 = by * TY + 1;
    // NRM: C at this thread's points of the last phase (sub-lattice sl,
    // u-th point), zero outside the plane
    T cpre[NRM ? 4 * KU : 1];
    if (NRM) {
#pragma unroll
      for (int sl = 0; sl < 4; ++sl) {
#pragma unroll
        for (int u = 0; u < KU; ++u) {
          const int q = tid + u * NT;
          const int i = i0 + (sl & 1) + 2 * (q % QX), j = j0 + (sl >> 1) + 2 * (q / QX);
          const bool in = (last_mask & (1u << sl)) && q < NQ && i <= nx && j <= ny;
          cpre[sl * KU + u] = in ? __ldg(cdiag + size_t(j) * p + i) : T(0);
        }
      }
    }
    const bool ok = mbar_wait_bounded(&bar[s], parity);
    if (!__syncthreads_and(ok)) {
      if (tid == 0) {
        atomicOr(err, DEV_TIMEOUT);
        // the block's shared memory must outlive its copies in flight
        mbar_wait_bounded(&bar[s], parity);
        if (NSTAGE == 2 && tn < ntiles) mbar_wait_bounded(&bar[s ^ 1], unsigned((it + 1) >> 1) & 1u);
      }
      __syncthreads();
      return;
    }

    T* const sx = s ? stage1 : stage0;
    const T* const sic = sx + TP_IC * PL;
    const T* const sw = sx + TP_W * PL;
    const T* const ss = sx + TP_S * PL;
    const T* const sb = sx + TP_B * PL;
    const T* const ssw = sx + TP_SW * PL;
    const T* const snw = sx + TP_NW * PL;
    // Shared cell (r, c) holds domain point (i0 + c - HA, j0 + r - HY).  With
    // TX, TY, HA and HY even, the 0-based domain parities of (r, c) are
    // (r & 1, c & 1).  Phase k is relaxed on the tile grown by (gx, gy).
#pragma unroll
    for (int k = 0; k < NPH; ++k) {
      // NRM: the first phase would recompute every value of its colour from
      // unchanged neighbours, giving the same bits (see above): skipped
      if (NRM && k == 0) continue;
      if (NRM && k == NPH - 1) {
        // the last phase with the residual of the points it updates
#pragma unroll
        for (int sl = 0; sl < 4; ++sl) {
          if (!(last_mask & (1u << sl))) continue;
#pragma unroll
          for (int u = 0; u < KU; ++u) {
            const int q = tid + u * NT;
            const int c = HA + (sl & 1) + 2 * (q % QX), r = HY + (sl >> 1) + 2 * (q / QX);
            if (q >= NQ || unsigned(i0 + c - HA - 1) >= unsigned(nx) ||
                unsigned(j0 + r - HY - 1) >= unsigned(ny))
              continue;
            const int o = r * BW + c;
            T* xp = sx + o;
            const T xo = *xp;
            const T xn = gs_pre_apply<T>(sic[o], sw[o], sb[o], ss[o], ssw[o],
                                         [&](int dx, int dy) { return xp[dx + dy * BW]; });
            const double rv = double(cpre[sl * KU + u]) * double(xn - xo);
            nacc = fma(rv, rv, nacc);
            *xp = xn;
          }
        }
        __syncthreads();
        continue;
      }
      const unsigned mask = (order >> (4 * k)) & 0xFu;
      const int gx = colour_grow_x(NPH, k), gy = colour_grow_y(NPH, k);
      const int r0 = HY - gy, r1 = HY + TY + gy;
      const int c0 = HA - gx, c1 = HA + TX + gx;
#pragma unroll
      for (int sl = 0; sl < 4; ++sl) {
        if (!(mask & (1u << sl))) continue;
        const int pj = sl >> 1, pi = sl & 1;
        const int rf = r0 + ((pj - r0) & 1);
        const int cf = c0 + ((pi - c0) & 1);
        const int nr = (r1 - rf + 1) >> 1, ncol = (c1 - cf + 1) >> 1;
        const int npts = nr * ncol;
        // point q = rr * ncol + cc of the sub-lattice; q advances by NT, so
        // (rr, cc) advance by (NT / ncol, NT % ncol) with one carry
        const int drr = NT / ncol, dcc = NT - drr * ncol;
        int rr = tid / ncol, cc = tid - rr * ncol;
        for (int q = tid; q < npts; q += NT) {
          const int r = rf + 2 * rr, c = cf + 2 * cc;
          rr += drr;
          cc += dcc;
          if (cc >= ncol) {
            cc -= ncol;
            ++rr;
          }
          // domain point (i, j) = (i0 + c - HA, j0 + r - HY) inside 1..nx, 1..ny
          if (unsigned(i0 + c - HA - 1) >= unsigned(nx) ||
              unsigned(j0 + r - HY - 1) >= unsigned(ny)) {
            if (ZERO) sx[r * BW + c] = T(0);
            continue;
          }
          const int o = r * BW + c;
          if (PRE) {
            T* xp = sx + o;
            // zero start: the first phase's neighbours are all zero, and
            // fma(a, 0, b/C) = b/C
            if (ZERO && zero_start_mask(false, k) == 0u)
              *xp = sic[o];
            else
              *xp = gs_pre_apply<T>(sic[o], sw[o], sb[o], ss[o], ssw[o],
                                    [&](int dx, int dy) { return xp[dx + dy * BW]; });
            continue;
          }
          GsCoef<T, NINE> cf_;
          cf_.b = sb[o];
          cf_.ic = sic[o];
          cf_.w = sw[o];
          cf_.e = sw[o + 1];
          cf_.s = ss[o];
          cf_.n = ss[o + BW];
          if (NINE) {
            cf_.sw = ssw[o];
            cf_.se = snw[o + 1 - BW];
            cf_.nw = snw[o];
            cf_.ne = ssw[o + 1 + BW];
          }
          T* xp = sx + o;
          if (ZERO)
            *xp = gs_apply_masked<T, NINE>(cf_, [&](int dx, int dy) { return xp[dx + dy * BW]; },
                                           zero_start_mask(NINE, k));
          else
            *xp = gs_apply<T, NINE>(cf_, [&](int dx, int dy) { return xp[dx + dy * BW]; });
        }
      }
      __syncthreads();
    }
    for (int e = tid; e < TX * TY; e += NT) {
      const int r = e / TX, c = e - r * TX;
      const int i = i0 + c, j = j0 + r;
      if (i <= nx && j <= ny) xout[j * p + i] = sx[(r + HY) * BW + c + HA];
    }
    // this stage is refilled by the copies issued next
    fence_proxy_async();
    __syncthreads();
    if (NSTAGE == 1 && tid == 0 && tn < ntiles) issue(0, tn);
  }
  if (NRM) {
    // fixed reduction tree: warps, then warp sums in order
    __shared__ double wsum[NT / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) nacc += __shfl_xor_sync(0xffffffffu, nacc, off);
    if ((tid & 31) == 0) wsum[tid >> 5] = nacc;
    __syncthreads();
    if (tid == 0) {
      double a = 0.0;
      for (int w = 0; w < NT / 32; ++w) a += wsum[w];
      nrm[blockIdx.x] = a;
    }
  }
}

}  // namespace bmg
