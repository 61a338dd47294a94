// Zebra line Gauss-Seidel on full grids (the per-line arithmetic is in
// bmg_line.cuh): setup-time factorisation of every line, and one sweep as
// four launches per (direction, colour) step -- right-hand sides, block
// solves, separator chains, final update.
#include <type_traits>

#include "bmg_line.cuh"

namespace bmg {

namespace {

inline int cdiv(long a, long b) { return int((a + b - 1) / b); }

constexpr int kPT = 256;        // threads of the point-parallel kernels
constexpr int kBT = 128;        // threads of the block-parallel kernels

// Point-parallel index space of one colour: the fast grid axis runs along
// the contiguous direction of the plane (the points of a row for x-lines,
// the lines of the colour for y-lines).  Calls f(q, k) for every point.
template <int DIR, class F>
__device__ __forceinline__ void for_colour_points(const LineGeo& g, int colour, F f) {
  const int nlc = line_count(g.nl, colour);
  const int fast = DIR == 0 ? g.n : nlc, slow = DIR == 0 ? nlc : g.n;
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= fast) return;
  for (int b = blockIdx.y; b < slow; b += gridDim.y) {
    const int li = DIR == 0 ? b : a, k = (DIR == 0 ? a : b) + 1;
    f(2 * li + colour + 1, k);
  }
}

template <typename T, int DIR, bool NINE>
__global__ void __launch_bounds__(kPT) k_line_rhs(LevelV<T> L, int colour,
                                                  const T* __restrict__ xs) {
  const LineGeo g = line_geo<DIR>(L);
  T* G = line_scratch<DIR>(L);
  for_colour_points<DIR>(g, colour, [&](int q, int k) {
    G[line_fbase<DIR>(L, q) + k * g.fes] = line_rhs<T, DIR, NINE>(L, xs, q * g.ls + k * g.es);
  });
}

// Block-parallel: the fast axis runs over blocks of a row (x-lines) or over
// the lines of the colour (y-lines).
template <typename T, int DIR>
__global__ void __launch_bounds__(kBT) k_line_blocks(LevelV<T> L, int colour) {
  const LineGeo g = line_geo<DIR>(L);
  const int nlc = line_count(g.nl, colour), nb = g.n / kLineM + 1;
  const int fast = DIR == 0 ? nb : nlc, slow = DIR == 0 ? nlc : nb;
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= fast) return;
  for (int b = blockIdx.y; b < slow; b += gridDim.y) {
    const int li = DIR == 0 ? b : a, bb = DIR == 0 ? a : b;
    line_block_solve<T, DIR>(L, 2 * li + colour + 1, bb);
  }
}

// x-lines: one thread block per segment of kXSeg blocks of a row.  The
// segment's right-hand sides and factors are loaded with contiguous accesses
// into shared memory (one word of padding per block of kLineM points, so the
// threads' block-strided reads hit distinct banks), each thread substitutes
// its block there, and the solutions go back with contiguous stores.
constexpr int kXSeg = 128;
constexpr int kXPts = kXSeg * kLineM;
constexpr int kXPad = kXSeg * (kLineM + 1);

template <typename T>
size_t xblocks_smem() { return 4 * size_t(kXPad) * sizeof(T); }

template <typename T>
__global__ void __launch_bounds__(kXSeg) k_line_blocks_x(LevelV<T> L, int colour) {
  extern __shared__ __align__(16) unsigned char xsm_raw[];
  T* sd = reinterpret_cast<T*>(xsm_raw);
  T* sm = sd + kXPad;
  T* si = sm + kXPad;
  T* sc = si + kXPad;
  const LineGeo g = line_geo<0>(L);
  const int q = 2 * blockIdx.y + colour + 1;
  const int k_base = blockIdx.x * kXPts + 1;      // first point of the segment
  const int o_base = q * g.ls + k_base;
  const T* __restrict__ mu = L.LF[0][LF_MU];
  const T* __restrict__ iu = L.LF[0][LF_IU];
  const T* __restrict__ ca = L.LF[0][LF_CA];
  T* G = L.r;
  const int npts = min(kXPts, g.n - k_base + 1);
  for (int i = threadIdx.x; i < npts; i += kXSeg) {
    const int p = i + i / kLineM, o = o_base + i;
    sd[p] = G[o];
    sm[p] = mu[o];
    si[p] = iu[o];
    sc[p] = ca[o];
  }
  __syncthreads();
  const int j = threadIdx.x;
  const int bb = blockIdx.x * kXSeg + j;
  const int k0 = bb * kLineM + 1;
  const int len = min(kLineM - 1, g.n - k0 + 1);
  if (len > 0) {
    const int pb = j * (kLineM + 1);
    T gfirst, glast;
    block_subst<T>(
        len,
        [&](int e, T& d, T& m, T& iv, T& c) {
          d = sd[pb + e];
          m = sm[pb + e];
          iv = si[pb + e];
          c = sc[pb + e];
        },
        [&](int e, T v) { sd[pb + e] = v; }, gfirst, glast);
    if (k0 + len <= g.n && len == kLineM - 1) {
      const int os = q * g.ls + k0 + len;
      L.SP[0][SP_RL][q * L.spp[0] + bb] = fma(L.W[os], glast, sd[pb + len]);
    }
    if (bb > 0) L.SP[0][SP_GF][q * L.spp[0] + bb - 1] = gfirst;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < npts; i += kXSeg)
    if ((i + 1) % kLineM != 0) G[o_base + i] = sd[i + i / kLineM];
}

// The separators' two-level substitution (line_sep_serial states the
// operations): one thread per group of a line, several lines per thread
// block; each thread substitutes its group from a zero carry, one thread
// per line runs the carries through the groups in shared memory, and each
// thread then fixes up its group.  The right-hand sides come from the
// compact slots the block solves filled.
constexpr int kSepThreads = 256;
constexpr int kSepGroup = 16;   // separators per group held in registers

template <typename T, int DIR>
__global__ void __launch_bounds__(kSepThreads) k_line_seps(LevelV<T> L, int colour, int ngroups,
                                                           T* __restrict__ xo) {
  __shared__ T s_end[kSepThreads], s_pq[kSepThreads], s_c[kSepThreads];
  const int tid = threadIdx.x;
  const LineGeo g = line_geo<DIR>(L);
  const int lpb = kSepThreads / ngroups;               // lines per block
  const int l = tid / ngroups, gi = tid - l * ngroups;
  const int li = blockIdx.x * lpb + l;
  const bool act = l < lpb && li < line_count(g.nl, colour);
  const int nsep = g.n / kLineM, gl = L.sgl[DIR];
  const int t0 = gi * gl, t1 = min(t0 + gl, nsep);
  const int q = 2 * li + colour + 1;
  const int sp = q * L.spp[DIR];
  const T* __restrict__ mu = L.SP[DIR][SP_MU] + sp;
  const T* __restrict__ iu = L.SP[DIR][SP_IU] + sp;
  const T* __restrict__ ca = L.SP[DIR][SP_CA] + sp;
  const T* __restrict__ an = L.SP[DIR][SP_AN] + sp;
  const T* __restrict__ P = L.SP[DIR][SP_P] + sp;
  const T* __restrict__ Q = L.SP[DIR][SP_Q] + sp;
  const T* __restrict__ gf = L.SP[DIR][SP_GF] + sp;
  T* h = L.SP[DIR][SP_RL] + sp;
  // forward partial substitution of the group (groups of kSepGroup: every
  // load of a phase is issued before its substitution starts)
  constexpr int GL = kSepGroup;
  const bool regs = gl == GL;
  const int len = t1 - t0;
  T hv[GL];
  T yh = T(0);
  if (act) {
    if (regs) {
      T mv[GL], rv[GL];
#pragma unroll
      for (int u = 0; u < GL; ++u)
        if (u < len) {
          mv[u] = mu[t0 + u];
          rv[u] = fma(an[t0 + u], gf[t0 + u], h[t0 + u]);
        }
#pragma unroll
      for (int u = 0; u < GL; ++u)
        if (u < len) {
          yh = fma(mv[u], yh, rv[u]);
          hv[u] = yh;
        }
    } else {
      for (int t = t0; t < t1; ++t) {
        yh = fma(mu[t], yh, fma(an[t], gf[t], h[t]));
        h[t] = yh;
      }
    }
    s_end[tid] = yh;
    s_pq[tid] = P[t1 - 1];
  }
  __syncthreads();
  if (act && gi == 0) {
    T c = T(0);
    for (int k = 0; k < ngroups; ++k) {
      const int j = l * ngroups + k;
      const T cg = c;
      s_c[j] = cg;
      c = fma(s_pq[j], cg, s_end[j]);
    }
  }
  __syncthreads();
  // fix-up, scaling and backward partial substitution of the group
  if (act) {
    const T cg = s_c[tid];
    T xh = T(0);
    if (regs) {
      T pv[GL], iv[GL], cv[GL];
#pragma unroll
      for (int u = 0; u < GL; ++u)
        if (u < len) {
          pv[u] = P[t0 + u];
          iv[u] = iu[t0 + u];
          cv[u] = ca[t0 + u];
        }
#pragma unroll
      for (int u = GL - 1; u >= 0; --u)
        if (u < len) {
          xh = fma(cv[u], xh, fma(pv[u], cg, hv[u]) * iv[u]);
          hv[u] = xh;
        }
    } else {
      for (int t = t1 - 1; t >= t0; --t) {
        xh = fma(ca[t], xh, fma(P[t], cg, h[t]) * iu[t]);
        h[t] = xh;
      }
    }
    s_end[tid] = xh;
    s_pq[tid] = Q[t0];
  }
  __syncthreads();
  if (act && gi == 0) {
    T e = T(0);
    for (int k = ngroups - 1; k >= 0; --k) {
      const int j = l * ngroups + k;
      s_c[j] = e;
      e = fma(s_pq[j], e, s_end[j]);
    }
  }
  __syncthreads();
  if (act) {
    const T e = s_c[tid];
    const int base = q * g.ls;
    if (regs) {
#pragma unroll
      for (int u = 0; u < GL; ++u)
        if (u < len) xo[base + (t0 + u + 1) * kLineM * g.es] = fma(Q[t0 + u], e, hv[u]);
    } else {
      for (int t = t0; t < t1; ++t) xo[base + (t + 1) * kLineM * g.es] = fma(Q[t], e, h[t]);
    }
  }
}

template <typename T, int DIR>
__global__ void __launch_bounds__(kPT) k_line_final(LevelV<T> L, int colour,
                                                    T* __restrict__ xo) {
  const LineGeo g = line_geo<DIR>(L);
  for_colour_points<DIR>(g, colour, [&](int q, int k) {
    if (k % kLineM != 0) line_final<T, DIR>(L, g, q, k, xo);
  });
}

// ---------------------------------------------------------------------------
// Setup: factors of every line (both colours), computed in FP64 and stored
// in the level's precision.
// ---------------------------------------------------------------------------

// Per block: LU of the block's tridiagonal matrix (diagonal C, off-diagonals
// -a) and its responses v = T^{-1} (a_first e_first), w = T^{-1} (a_next e_last)
// to unit values of the separators on either side (a_first couples the
// block's first point to the point before it, a_next its last point to the
// point after it; both are 0 at the ends of the line).
template <typename T, int DIR>
__global__ void __launch_bounds__(kBT) k_line_factor_blocks(LevelV<T> L, int* derr) {
  const LineGeo g = line_geo<DIR>(L);
  const int nb = g.n / kLineM + 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nb * g.nl) return;
  const int q = t / nb + 1, bb = t % nb;
  const int k0 = bb * kLineM + 1;
  const int len = min(kLineM - 1, g.n - k0 + 1);
  if (len <= 0) return;
  const T* A = line_coupling<DIR>(L);
  const int o0 = q * g.ls + k0 * g.es;
  const int f0 = line_fbase<DIR>(L, q) + k0 * g.fes;
  double iu[kLineM - 1], ca[kLineM - 1], mu[kLineM - 1];
  double up = 1.0;
  bool bad = false;
#pragma unroll
  for (int e = 0; e < kLineM - 1; ++e) {
    if (e < len) {
      const int o = o0 + e * g.es;
      const double a = double(A[o]), c = double(L.C[o]);
      const double m = e ? a / up : 0.0;
      const double u = c - m * a;
      if (!(u > 0.0) || !(u < INFINITY)) bad = true;
      mu[e] = m;
      iu[e] = 1.0 / u;
      if (e) ca[e - 1] = a * iu[e - 1];
      up = u;
    }
  }
  const double a_first = double(A[o0]);
  const double a_next = double(A[o0 + len * g.es]);
  double yv[kLineM - 1];
  double prev = a_first;
#pragma unroll
  for (int e = 0; e < kLineM - 1; ++e) {
    if (e < len) {
      if (e) prev = mu[e] * prev;
      yv[e] = prev;
    }
  }
  double vn = 0.0, wn = 0.0;
#pragma unroll
  for (int e = kLineM - 2; e >= 0; --e) {
    if (e < len) {
      const int f = f0 + e * g.fes;
      const double cae = e == len - 1 ? 0.0 : ca[e];
      vn = yv[e] * iu[e] + cae * vn;
      wn = (e == len - 1 ? a_next * iu[e] : 0.0) + cae * wn;
      L.LF[DIR][LF_MU][f] = T(mu[e]);
      L.LF[DIR][LF_IU][f] = T(iu[e]);
      L.LF[DIR][LF_CA][f] = T(cae);
      L.LF[DIR][LF_V][f] = T(vn);
      L.LF[DIR][LF_W][f] = T(wn);
    }
  }
  if (bad) atomicOr(derr, DEV_BADLINE);
}

// Per line: the Schur complement on the separators.  With the interior
// points written as g + v x_left + w x_right, the equation of separator s is
//   (C_s - a_s w_{s-1} - a_{s+1} v_{s+1}) x_s - a_s v_{s-1} x_prev
//     - a_{s+1} w_{s+1} x_next = d_s + a_s g_{s-1} + a_{s+1} g_{s+1},
// a tridiagonal system over the separators of the line, factored here.
template <typename T, int DIR>
__global__ void __launch_bounds__(kBT) k_line_factor_seps(LevelV<T> L, int* derr) {
  const LineGeo g = line_geo<DIR>(L);
  const int q = blockIdx.x * blockDim.x + threadIdx.x + 1;
  if (q > g.nl) return;
  const int nsep = g.n / kLineM;
  const T* A = line_coupling<DIR>(L);
  const T* V = L.LF[DIR][LF_V];
  const T* W = L.LF[DIR][LF_W];
  double up = 1.0, uprev_coupling = 0.0;
  bool bad = false;
  for (int t = 0; t < nsep; ++t) {
    const int os = q * g.ls + (t + 1) * kLineM * g.es;
    const int fs = line_fbase<DIR>(L, q) + (t + 1) * kLineM * g.fes;
    const double as = double(A[os]), an = double(A[os + g.es]);
    const double d = double(L.C[os]) - as * double(W[fs - g.fes]) - an * double(V[fs + g.fes]);
    const double lo = as * double(V[fs - g.fes]);   // coupling to the previous separator
    const double hi = an * double(W[fs + g.fes]);   // coupling to the next separator
    const double m = t ? lo / up : 0.0;
    const double u = d - m * uprev_coupling;
    if (!(u > 0.0) || !(u < INFINITY)) bad = true;
    const int c = q * L.spp[DIR] + t;
    L.SP[DIR][SP_MU][c] = T(m);
    L.SP[DIR][SP_IU][c] = T(1.0 / u);
    L.SP[DIR][SP_CA][c] = T(hi / u);
    L.SP[DIR][SP_AN][c] = A[os + g.es];
    up = u;
    uprev_coupling = hi;
  }
  // products of the stored multipliers over each group: P from the group's
  // start to t, Q from t to the group's end
  const int gl = L.sgl[DIR];
  T* mu = L.SP[DIR][SP_MU] + q * L.spp[DIR];
  T* ca = L.SP[DIR][SP_CA] + q * L.spp[DIR];
  T* P = L.SP[DIR][SP_P] + q * L.spp[DIR];
  T* Q = L.SP[DIR][SP_Q] + q * L.spp[DIR];
  double pr = 1.0;
  for (int t = 0; t < nsep; ++t) {
    pr = (t % gl == 0 ? 1.0 : pr) * double(mu[t]);
    P[t] = T(pr);
  }
  for (int t = nsep - 1; t >= 0; --t) {
    pr = (t == nsep - 1 || (t + 1) % gl == 0 ? 1.0 : pr) * double(ca[t]);
    Q[t] = T(pr);
  }
  if (bad) atomicOr(derr, DEV_BADLINE);
}

int grid_y(int slow) { return slow < 65535 ? slow : 65535; }

template <typename T, int DIR, bool NINE>
void line_step(const LevelV<T>& L, int colour, const T* xs, T* xo, cudaStream_t s) {
  const LineGeo g = line_geo<DIR>(L);
  const int nlc = line_count(g.nl, colour);
  if (nlc <= 0) return;
  const int nb = g.n / kLineM + 1;
  {
    const int fast = DIR == 0 ? g.n : nlc, slow = DIR == 0 ? nlc : g.n;
    k_line_rhs<T, DIR, NINE><<<dim3(cdiv(fast, kPT), grid_y(slow)), kPT, 0, s>>>(L, colour, xs);
  }
  if (DIR == 0) {
    k_line_blocks_x<T><<<dim3(cdiv(g.n, kXPts), nlc), kXSeg, xblocks_smem<T>(), s>>>(L, colour);
  } else {
    const int fast = nlc, slow = nb;
    k_line_blocks<T, DIR><<<dim3(cdiv(fast, kBT), grid_y(slow)), kBT, 0, s>>>(L, colour);
  }
  if (g.n >= kLineM) {
    const int nsep = g.n / kLineM, ngroups = cdiv(nsep, L.sgl[DIR]);
    const int lpb = kSepThreads / ngroups;
    k_line_seps<T, DIR><<<cdiv(nlc, lpb), kSepThreads, 0, s>>>(L, colour, ngroups, xo);
  }
  {
    const int fast = DIR == 0 ? g.n : nlc, slow = DIR == 0 ? nlc : g.n;
    k_line_final<T, DIR><<<dim3(cdiv(fast, kPT), grid_y(slow)), kPT, 0, s>>>(L, colour, xo);
  }
  count_launch(g.n >= kLineM ? 4 : 3);
}

}  // namespace

template <typename T>
int launch_line_factor(const LevelV<T>& L, int smoother, int* derr, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_line_blocks_x<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(xblocks_smem<T>())) != cudaSuccess)
      return BMG_ECUDA;
    attr = true;
  }
  auto one = [&](auto dir_tag) {
    constexpr int DIR = decltype(dir_tag)::value;
    const LineGeo g = line_geo<DIR>(L);
    const int nb = g.n / kLineM + 1;
    k_line_factor_blocks<T, DIR><<<cdiv(nb * g.nl, kBT), kBT, 0, s>>>(L, derr);
    k_line_factor_seps<T, DIR><<<cdiv(g.nl, kBT), kBT, 0, s>>>(L, derr);
    count_launch(2);
  };
  if (smoother == BMG_SMOOTH_XLINE || smoother == BMG_SMOOTH_ALTLINE)
    one(std::integral_constant<int, 0>{});
  if (smoother == BMG_SMOOTH_YLINE || smoother == BMG_SMOOTH_ALTLINE)
    one(std::integral_constant<int, 1>{});
  return cudaGetLastError() == cudaSuccess ? 0 : BMG_ECUDA;
}

template <typename T>
void launch_line_sweep(const LevelV<T>& L, bool nine, int smoother, bool reverse, const T* xin,
                       T* xout, cudaStream_t s) {
  int dir[4], colour[4];
  const int n = line_steps(smoother, reverse, dir, colour);
  for (int k = 0; k < n; ++k) {
    // The first step reads the neighbouring lines from xin; every later one
    // from xout, which holds all lines the earlier steps solved.
    const T* xs = k == 0 ? xin : xout;
    if (dir[k] == 0) {
      if (nine)
        line_step<T, 0, true>(L, colour[k], xs, xout, s);
      else
        line_step<T, 0, false>(L, colour[k], xs, xout, s);
    } else {
      if (nine)
        line_step<T, 1, true>(L, colour[k], xs, xout, s);
      else
        line_step<T, 1, false>(L, colour[k], xs, xout, s);
    }
  }
}

template int launch_line_factor<double>(const LevelV<double>&, int, int*, cudaStream_t);
template int launch_line_factor<float>(const LevelV<float>&, int, int*, cudaStream_t);
template void launch_line_sweep<double>(const LevelV<double>&, bool, int, bool, const double*,
                                        double*, cudaStream_t);
template void launch_line_sweep<float>(const LevelV<float>&, bool, int, bool, const float*, float*,
                                       cudaStream_t);

}  // namespace bmg
