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
constexpr int kSepChunk = 256;  // separators per line staged per pass
constexpr int kSepLines = 8;    // lines per thread block of the separator kernel

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

// One line per lane: kSepLines lanes of warp 0 run the separator chains of
// kSepLines lines of the colour at once (an FP64 warp instruction costs the
// same pipe slot however few lanes are active), after all kSepThreads
// threads have staged a chunk of kSepChunk separators of those lines in
// shared memory, transposed to [separator][line] with one word of padding
// per row (the loads run along each line's compact slots; each chain step
// reads consecutive words).  Forward: stage the Schur right-hand sides
// (d_s + a_s g_{s-1}) + a_{s+1} g_{s+1} and the multipliers, run
// y = mu y + rhs, write y back over d_s + a_s g_{s-1}; backward: stage
// y * (1/u) and the coefficients, run x = ca x + y / u, write x to the
// separators.  The arithmetic is that of line_sep_serial.
constexpr int kSepThreads = 128;

template <typename T, int DIR>
__global__ void __launch_bounds__(kSepThreads) k_line_seps(LevelV<T> L, int colour,
                                                           T* __restrict__ xo) {
  __shared__ T sa[kSepChunk][kSepLines + 1], sb[kSepChunk][kSepLines + 1];
  const int tid = threadIdx.x;
  const LineGeo g = line_geo<DIR>(L);
  const int nlc = line_count(g.nl, colour);
  const int li0 = blockIdx.x * kSepLines;
  const int nsep = g.n / kLineM, spp = L.spp[DIR];
  const T* __restrict__ mu = L.SP[DIR][SP_MU];
  const T* __restrict__ iu = L.SP[DIR][SP_IU];
  const T* __restrict__ ca = L.SP[DIR][SP_CA];
  const T* __restrict__ an = L.SP[DIR][SP_AN];
  const T* __restrict__ gf = L.SP[DIR][SP_GF];
  T* rl = L.SP[DIR][SP_RL];
  const int nl_here = min(kSepLines, nlc - li0);
  const bool chain = tid < nl_here;       // one lane per line
  auto slot = [&](int l, int t) { return (2 * (li0 + l) + colour + 1) * spp + t; };
  T y = T(0);
  for (int c0 = 0; c0 < nsep; c0 += kSepChunk) {
    const int cn = min(kSepChunk, nsep - c0);
#pragma unroll 4
    for (int idx = tid; idx < nl_here * cn; idx += kSepThreads) {
      const int l = idx / cn, t = idx - l * cn;
      const int r = slot(l, c0 + t);
      sa[t][l] = fma(an[r], gf[r], rl[r]);
      sb[t][l] = mu[r];
    }
    __syncthreads();
    if (chain) {
      int t = 0;
      for (; t + 8 <= cn; t += 8) {
        T m[8], r[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          m[u] = sb[t + u][tid];
          r[u] = sa[t + u][tid];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          y = fma(m[u], y, r[u]);
          sa[t + u][tid] = y;
        }
      }
      for (; t < cn; ++t) {
        y = fma(sb[t][tid], y, sa[t][tid]);
        sa[t][tid] = y;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int idx = tid; idx < nl_here * cn; idx += kSepThreads) {
      const int l = idx / cn, t = idx - l * cn;
      rl[slot(l, c0 + t)] = sa[t][l];
    }
    __syncthreads();
  }
  T xn = T(0);
  for (int c1 = nsep; c1 > 0; c1 -= kSepChunk) {
    const int c0 = max(0, c1 - kSepChunk), cn = c1 - c0;
#pragma unroll 4
    for (int idx = tid; idx < nl_here * cn; idx += kSepThreads) {
      const int l = idx / cn, t = idx - l * cn;
      const int r = slot(l, c0 + t);
      sa[t][l] = rl[r] * iu[r];
      sb[t][l] = ca[r];
    }
    __syncthreads();
    if (chain) {
      int t = cn - 1;
      for (; t >= 7; t -= 8) {
        T c[8], a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          c[u] = sb[t - u][tid];
          a[u] = sa[t - u][tid];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          xn = fma(c[u], xn, a[u]);
          sa[t - u][tid] = xn;
        }
      }
      for (; t >= 0; --t) {
        xn = fma(sb[t][tid], xn, sa[t][tid]);
        sa[t][tid] = xn;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int idx = tid; idx < nl_here * cn; idx += kSepThreads) {
      const int l = idx / cn, t = idx - l * cn;
      xo[(2 * (li0 + l) + colour + 1) * g.ls + (c0 + t + 1) * kLineM * g.es] = sa[t][l];
    }
    __syncthreads();
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
  if (g.n >= kLineM)
    k_line_seps<T, DIR><<<cdiv(nlc, kSepLines), kSepThreads, 0, s>>>(L, colour, xo);
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
