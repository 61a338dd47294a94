// Persistent coarse sub-cycle (the single-GPU reading of the coarse-grid
// redistribution of Section 2.2 / Algorithm 2): one thread block, or every
// block of one thread-block cluster, runs Algorithm 1 on levels 0 .. thr-1,
// starting from b_{thr-1} and leaving x_{thr-1}, with phases separated by a
// barrier (__syncthreads(), or the hardware cluster barrier) instead of
// kernel launches.  The per-point arithmetic is that of the full-grid
// kernels and the points of one colour are independent, so the result does
// not depend on the threshold or on the number of blocks.  Shared by the
// single-problem kernels and the batched kernel (one block per problem).
#pragma once

#include "bmg_line.cuh"

namespace bmg {

// Who runs a phase and how phases are separated.  BlockTeam: the threads of
// one block.  ClusterTeam: the threads of every block of the cluster, in
// block-rank order; the barrier is barrier.cluster.arrive.release +
// barrier.cluster.wait.acquire, which orders every memory access of the
// cluster's threads before it (global memory included) before every access
// after it.  Every thread of the team reaches every barrier (all loops below
// have team-uniform trip counts), so no barrier can wait forever.
struct BlockTeam {
  static constexpr bool kCluster = false;
  __device__ static int rank() { return 0; }
  __device__ static int index() { return int(threadIdx.x); }
  __device__ static int size() { return int(blockDim.x); }
  __device__ static void sync() { __syncthreads(); }
};

struct ClusterTeam {
  static constexpr bool kCluster = true;
  __device__ static int rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return int(r);
  }
  __device__ static int ranks() {
    unsigned n;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(n));
    return int(n);
  }
  __device__ static int index() { return rank() * int(blockDim.x) + int(threadIdx.x); }
  __device__ static int size() { return ranks() * int(blockDim.x); }
  __device__ static void sync() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
  }
};

// A colour is a set of parity sub-lattices; bit (2*pj + pi) stands for the
// points whose 0-based row index j-1 has parity pj and column i-1 parity pi.
// Red-black: red = {(0,0),(1,1)} = (i + j) even, black = {(0,1),(1,0)}.
// Four colours, in the order (i mod 2, j mod 2) = (1,1), (0,1), (1,0), (0,0)
// (1-based): sub-lattices (0,0), (0,1), (1,0), (1,1).
__host__ __device__ constexpr unsigned rb_mask(int c) { return c == 0 ? 0x9u : 0x6u; }
__host__ __device__ constexpr unsigned four_mask(int c) { return 1u << c; }

template <typename T>
struct CoarseArgs {
  const LevelV<T>* lev;      // device array of level views
  int thr;                   // levels 0 .. thr-1 run here
  int nu1, nu2, add_rc;
  int smoother;              // BMG_SMOOTH_*
  int top_nine;              // is level thr-1 9-point (else red-black)
  const double* chol;        // N0 x N0 lower factor
  const double* idiag;       // 1 / L[i][i]
  int n0;
};

template <typename T, bool NINE, class Team = BlockTeam>
__device__ void blk_colour(const LevelV<T>& L, unsigned mask) {
  const int hx = (L.nx + 1) >> 1, hy = (L.ny + 1) >> 1;
  for (int t = Team::index(); t < hx * hy; t += Team::size()) {
    const int ii = t % hx, jj = t / hx;
#pragma unroll
    for (int pj = 0; pj < 2; ++pj) {
#pragma unroll
      for (int pi = 0; pi < 2; ++pi) {
        if (!(mask & (1u << (2 * pj + pi)))) continue;
        const int i = 1 + pi + 2 * ii, j = 1 + pj + 2 * jj;
        if (i > L.nx || j > L.ny) continue;
        const int o = j * L.pitch + i;
        if (!NINE && sizeof(T) == 8 && L.PR[PR_B])
          L.x[o] = gs_pre_value<T>(L, L.x, o);     // prescaled finest level (FP64 only)
        else
          L.x[o] = gs_value<T, NINE>(L, L.x, L.b[o], o);
      }
    }
  }
  Team::sync();
}

// LINE: the line smoother of a.smoother (compiled into its own kernel, so the
// point-smoother kernel keeps its registers).
template <typename T, bool NINE, bool LINE, class Team = BlockTeam>
__device__ void blk_relax(const LevelV<T>& L, int nu, bool reverse, int smoother) {
  if constexpr (LINE) {
    static_assert(!Team::kCluster, "line smoothing runs in one block");
    blk_line_relax<T, NINE>(L, nu, reverse, smoother);
    return;
  }
  const int nc = NINE ? 4 : 2;
  for (int s = 0; s < nu; ++s) {
    for (int k = 0; k < nc; ++k) {
      const int c = reverse ? nc - 1 - k : k;
      blk_colour<T, NINE, Team>(L, NINE ? four_mask(c) : rb_mask(c));
    }
  }
}

template <typename T, bool NINE, class Team = BlockTeam>
__device__ void blk_residual(const LevelV<T>& L) {
  for (int t = Team::index(); t < L.nx * L.ny; t += Team::size()) {
    const int i = t % L.nx + 1, j = t / L.nx + 1;
    const int o = j * L.pitch + i;
    L.r[o] = resid_value<T, NINE>(L, L.x, L.b[o], o);
  }
  Team::sync();
}

template <typename T, class Team = BlockTeam>
__device__ void blk_restrict(const LevelV<T>& F, const LevelV<T>& Cc) {
  for (int t = Team::index(); t < Cc.nx * Cc.ny; t += Team::size()) {
    const int I = t % Cc.nx + 1, J = t / Cc.nx + 1;
    const int c = J * Cc.pitch + I;
    Cc.b[c] = restrict_value<T>(F.P, Cc.pitch, F.r, F.pitch, c, 2 * J * F.pitch + 2 * I);
    Cc.x[c] = T(0);
  }
  Team::sync();
}

template <typename T, class Team = BlockTeam>
__device__ void blk_interp(const LevelV<T>& F, const T* xc, int add_rc) {
  for (int t = Team::index(); t < F.nx * F.ny; t += Team::size()) {
    const int i = t % F.nx + 1, j = t / F.nx + 1;
    const int o = j * F.pitch + i;
    T corr = interp_value<T>(F.P, F.cpitch, xc, i, j);
    if (add_rc && ((i | j) & 1)) corr = fma(F.r[o], F.iC[o], corr);
    F.x[o] = F.x[o] + corr;
  }
  Team::sync();
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

template <typename T, bool LINE = false, class Team = BlockTeam>
__device__ void coarse_cycle_body(const CoarseArgs<T>& a) {
  for (int l = a.thr - 1; l >= 1; --l) {
    const LevelV<T> L = a.lev[l];
    const bool nine = (l < a.thr - 1) || a.top_nine;
    if (nine) {
      blk_relax<T, true, LINE, Team>(L, a.nu1, false, a.smoother);
      blk_residual<T, true, Team>(L);
    } else {
      blk_relax<T, false, LINE, Team>(L, a.nu1, false, a.smoother);
      blk_residual<T, false, Team>(L);
    }
    blk_restrict<T, Team>(L, a.lev[l - 1]);
  }
  // the coarsest solve is one block's work (block rank 0 of a cluster; its
  // own barriers are block barriers), then the whole team resumes
  if (Team::rank() == 0) blk_coarse_solve<T>(a.lev[0], a.chol, a.idiag, a.n0);
  if constexpr (Team::kCluster) Team::sync();
  for (int l = 1; l < a.thr; ++l) {
    const LevelV<T> L = a.lev[l];
    const bool nine = (l < a.thr - 1) || a.top_nine;
    blk_interp<T, Team>(L, a.lev[l - 1].x, a.add_rc);
    if (nine)
      blk_relax<T, true, LINE, Team>(L, a.nu2, true, a.smoother);
    else
      blk_relax<T, false, LINE, Team>(L, a.nu2, true, a.smoother);
  }
}


}  // namespace bmg
