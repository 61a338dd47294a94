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
constexpr int kSepWarps = 4;    // lines per block of the separator kernel
constexpr int kSepChunk = 256;  // separators staged per pass

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
  for_colour_points<DIR>(g, colour, [&](int q, int k) {
    const int o = q * g.ls + k * g.es;
    L.r[o] = line_rhs<T, DIR, NINE>(L, xs, o);
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

// One warp per line.  The lanes compute the Schur right-hand sides (and the
// products y * (1/u)) of a chunk of separators in parallel into shared
// memory; lane 0 runs the substitution chain through the chunk.  The
// arithmetic is that of line_sep_serial.
template <typename T, int DIR>
__global__ void __launch_bounds__(kSepWarps * 32) k_line_seps(LevelV<T> L, int colour,
                                                              T* __restrict__ xo) {
  __shared__ T sa[kSepWarps][kSepChunk], sb[kSepWarps][kSepChunk];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const LineGeo g = line_geo<DIR>(L);
  const int li = blockIdx.x * kSepWarps + warp;
  if (li >= line_count(g.nl, colour)) return;
  const int nsep = g.n / kLineM;
  const T* __restrict__ mu = L.LF[DIR][LF_MU];
  const T* __restrict__ iu = L.LF[DIR][LF_IU];
  const T* __restrict__ ca = L.LF[DIR][LF_CA];
  T* G = L.r;
  T* a = sa[warp];
  T* c = sb[warp];
  const int base = (2 * li + colour + 1) * g.ls, step = kLineM * g.es;
  T y = T(0);
  for (int c0 = 0; c0 < nsep; c0 += kSepChunk) {
    const int cn = min(kSepChunk, nsep - c0);
    for (int t = lane; t < cn; t += 32) {
      const int os = base + (c0 + t + 1) * step;
      a[t] = line_sep_rhs<T, DIR>(L, g.es, os);
      c[t] = mu[os];
    }
    __syncwarp();
    if (lane == 0)
      for (int t = 0; t < cn; ++t) {
        y = fma(c[t], y, a[t]);
        a[t] = y;
      }
    __syncwarp();
    for (int t = lane; t < cn; t += 32) G[base + (c0 + t + 1) * step] = a[t];
    __syncwarp();
  }
  T xn = T(0);
  for (int c1 = nsep; c1 > 0; c1 -= kSepChunk) {
    const int c0 = max(0, c1 - kSepChunk), cn = c1 - c0;
    for (int t = lane; t < cn; t += 32) {
      const int os = base + (c0 + t + 1) * step;
      a[t] = G[os] * iu[os];
      c[t] = ca[os];
    }
    __syncwarp();
    if (lane == 0)
      for (int t = cn - 1; t >= 0; --t) {
        xn = fma(c[t], xn, a[t]);
        a[t] = xn;
      }
    __syncwarp();
    for (int t = lane; t < cn; t += 32) xo[base + (c0 + t + 1) * step] = a[t];
    __syncwarp();
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
      const int o = o0 + e * g.es;
      const double cae = e == len - 1 ? 0.0 : ca[e];
      vn = yv[e] * iu[e] + cae * vn;
      wn = (e == len - 1 ? a_next * iu[e] : 0.0) + cae * wn;
      L.LF[DIR][LF_MU][o] = T(mu[e]);
      L.LF[DIR][LF_IU][o] = T(iu[e]);
      L.LF[DIR][LF_CA][o] = T(cae);
      L.LF[DIR][LF_V][o] = T(vn);
      L.LF[DIR][LF_W][o] = T(wn);
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
    const double as = double(A[os]), an = double(A[os + g.es]);
    const double d = double(L.C[os]) - as * double(W[os - g.es]) - an * double(V[os + g.es]);
    const double lo = as * double(V[os - g.es]);   // coupling to the previous separator
    const double hi = an * double(W[os + g.es]);   // coupling to the next separator
    const double m = t ? lo / up : 0.0;
    const double u = d - m * uprev_coupling;
    if (!(u > 0.0) || !(u < INFINITY)) bad = true;
    L.LF[DIR][LF_MU][os] = T(m);
    L.LF[DIR][LF_IU][os] = T(1.0 / u);
    L.LF[DIR][LF_CA][os] = T(hi / u);
    L.LF[DIR][LF_V][os] = T(0);
    L.LF[DIR][LF_W][os] = T(0);
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
  {
    const int fast = DIR == 0 ? nb : nlc, slow = DIR == 0 ? nlc : nb;
    k_line_blocks<T, DIR><<<dim3(cdiv(fast, kBT), grid_y(slow)), kBT, 0, s>>>(L, colour);
  }
  if (g.n >= kLineM)
    k_line_seps<T, DIR><<<cdiv(nlc, kSepWarps), kSepWarps * 32, 0, s>>>(L, colour, xo);
  {
    const int fast = DIR == 0 ? g.n : nlc, slow = DIR == 0 ? nlc : g.n;
    k_line_final<T, DIR><<<dim3(cdiv(fast, kPT), grid_y(slow)), kPT, 0, s>>>(L, colour, xo);
  }
  count_launch(g.n >= kLineM ? 4 : 3);
}

}  // namespace

template <typename T>
int launch_line_factor(const LevelV<T>& L, int smoother, int* derr, cudaStream_t s) {
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
