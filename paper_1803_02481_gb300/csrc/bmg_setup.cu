// BoxMG setup kernels (Section 2; discretisation of Section 5):
//   assembly of the 5-point cell-centred FV operator, operator-induced
//   interpolation weights, the Galerkin product P^T A P, the Cholesky factor
//   of the coarsest operator, dense <-> plane copies, and the backward of the
//   assembly (adjoint gradient).
#include "bmg_internal.h"

#include <cmath>

namespace bmg {

namespace {

constexpr int kTB = 256;

inline int cdiv(long a, long b) { return int((a + b - 1) / b); }

// Face coefficient of two square cells (series conductance of the two half
// cells, Section 5 discretisation): 2 k1 k2 / (k1 + k2).
__device__ __forceinline__ double harmonic(double k1, double k2) {
  return 2.0 * k1 * k2 / (k1 + k2);
}

// k of cell q: the input itself, or exp(input) for log-coefficients.
__device__ __forceinline__ double cell_k(const double* __restrict__ k, size_t q, bool log_k) {
  return log_k ? exp(k[q]) : k[q];
}

// Assembly tile: kAX x kAY cells per block, one thread per cell.
constexpr int kAX = 32, kAY = 8;

// Face and cell factors of the assembly: D = diag(k / r, k r) on cells of
// aspect hy / hx.  x faces carry harmonic(k_1 / r, k_2 / r) * hy / hx, y
// faces harmonic(k_1 r, k_2 r) * hx / hy; boundary faces (2 k / r) hy / hx
// and (2 k r) hx / hy.  1 / r and hx / hy come from the host; with
// r = aspect = 1 every factor is an exact 1.
struct AssemblyScale {
  double inv_r, r, aspect, inv_aspect;
  double beta[4];   // west, east, south, north: < 0 Dirichlet, else Robin beta
};

// A boundary face: the Dirichlet coefficient d (wall half a cell away), or
// for a Robin wall (k du/dn + alpha u = 0, beta = alpha times the cell width
// normal to the wall) the series conductance d * beta / (2 k_n + beta);
// beta = 0 is Neumann.
__device__ __forceinline__ double boundary_face(double d, double kn, double beta) {
  return beta < 0.0 ? d : d * (beta / (2.0 * kn + beta));
}

// Writes C, 1/C, W, S of the finest level and a dense copy of k; flags k that
// is not finite and positive.  Each thread forms the west and south faces of
// its cell (each interior face once); the east and north faces come from the
// neighbours through shared memory, the tile's last column and row forming
// the faces beyond it.  The east face of cell q is the same call as the west
// face of cell q+1, so C is what forming all four faces per cell would give.
template <typename T>
__global__ void __launch_bounds__(kAX * kAY) k_assemble(const double* __restrict__ k, int nx,
                                                        int ny, LevelV<T> L,
                                                        double* __restrict__ kcopy, int* derr,
                                                        bool log_k, AssemblyScale f) {
  __shared__ double fw[kAY][kAX + 1];   // west faces, column kAX = east of the tile
  __shared__ double fs[kAY + 1][kAX];   // south faces, row kAY = north of the tile
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i0 = blockIdx.x * kAX + tx;
  const int j0 = blockIdx.y * kAY + ty;
  const bool in = i0 < nx && j0 < ny;
  const size_t q = size_t(j0) * nx + i0;
  double kc = 1.0;
  auto kx = [&](size_t c) { return cell_k(k, c, log_k) * f.inv_r; };
  auto ky = [&](size_t c) { return cell_k(k, c, log_k) * f.r; };
  if (in) {
    kc = cell_k(k, q, log_k);
    if (!(kc > 0.0) || !(kc < INFINITY)) atomicOr(derr, DEV_BADK);
    kcopy[q] = kc;
    const double kxc = kc * f.inv_r, kyc = kc * f.r;
    fw[ty][tx] = i0 > 0 ? harmonic(kx(q - 1), kxc) * f.aspect : 0.0;
    fs[ty][tx] = j0 > 0 ? harmonic(ky(q - nx), kyc) * f.inv_aspect : 0.0;
    if (tx == kAX - 1)
      fw[ty][kAX] = i0 < nx - 1 ? harmonic(kxc, kx(q + 1)) * f.aspect : 0.0;
    if (ty == kAY - 1)
      fs[kAY][tx] = j0 < ny - 1 ? harmonic(kyc, ky(q + nx)) * f.inv_aspect : 0.0;
  }
  __syncthreads();
  if (!in) return;
  const double kxc = kc * f.inv_r, kyc = kc * f.r;
  const double aw = fw[ty][tx], as = fs[ty][tx];
  const double ae = i0 < nx - 1 ? fw[ty][tx + 1] : 0.0;
  const double an = j0 < ny - 1 ? fs[ty + 1][tx] : 0.0;
  // boundary faces, in the order west, east, south, north
  double bw = 0.0;
  if (i0 == 0) bw = bw + boundary_face(2.0 * kxc * f.aspect, kxc, f.beta[0]);
  if (i0 == nx - 1) bw = bw + boundary_face(2.0 * kxc * f.aspect, kxc, f.beta[1]);
  if (j0 == 0) bw = bw + boundary_face(2.0 * kyc * f.inv_aspect, kyc, f.beta[2]);
  if (j0 == ny - 1) bw = bw + boundary_face(2.0 * kyc * f.inv_aspect, kyc, f.beta[3]);
  const double c = (((aw + ae) + as) + an) + bw;
  const int o = (j0 + 1) * L.pitch + (i0 + 1);
  L.C[o] = T(c);
  L.iC[o] = T(1.0 / c);
  L.W[o] = T(aw);
  L.S[o] = T(as);
}

// Fine stencil row at plane offset o, as the interpolation formulas use it:
// negated off-diagonals a_X with a_X < 0 (positive matrix entries) lumped into
// the diagonal and a negative row sum sigma dropped,
//   a_X+ = max(a_X, 0),  C_eff = C - sum_X min(a_X, 0) - min(sigma, 0).
// On M-matrix rows with sigma >= 0 (the whole assembled level) this is the
// plain row.  Sums run in the order W, E, S, N, SW, SE, NW, NE.
template <typename T, bool NINE>
struct St {
  T c, w, e, s, n, sw, se, nw, ne;
  __device__ __forceinline__ St(const LevelV<T>& L, int o) {
    const int p = L.pitch;
    c = L.C[o];
    w = L.W[o];
    e = L.W[o + 1];
    s = L.S[o];
    n = L.S[o + p];
    if (NINE) {
      sw = L.SW[o];
      ne = L.SW[o + 1 + p];
      nw = L.NW[o];
      se = L.NW[o + 1 - p];
    } else {
      sw = se = nw = ne = T(0);
    }
    const T total = ((((((((T(0) + w) + e) + s) + n) + sw) + se) + nw) + ne);
    const T sigma = c - total;
    const T z = T(0);
    const T neg = ((((((((z + fmin(w, z)) + fmin(e, z)) + fmin(s, z)) + fmin(n, z)) + fmin(sw, z)) +
                     fmin(se, z)) + fmin(nw, z)) + fmin(ne, z));
    c = (c - neg) - fmin(sigma, z);
    w = fmax(w, z);
    e = fmax(e, z);
    s = fmax(s, z);
    n = fmax(n, z);
    sw = fmax(sw, z);
    se = fmax(se, z);
    nw = fmax(nw, z);
    ne = fmax(ne, z);
  }
};

// x-edge point: collapse the fine row in y (flux balance along x).
template <typename T, bool NINE>
__device__ __forceinline__ void xedge(const LevelV<T>& L, int o, T& ww, T& we, int* derr,
                                      int lbit) {
  St<T, NINE> a(L, o);
  const T den = (a.c - a.s) - a.n;
  if (!(den > T(0))) atomicOr(derr, DEV_BADDEN | lbit);
  ww = ((a.w + a.sw) + a.nw) / den;
  we = ((a.e + a.se) + a.ne) / den;
}

// y-edge point: collapse the fine row in x.
template <typename T, bool NINE>
__device__ __forceinline__ void yedge(const LevelV<T>& L, int o, T& ws, T& wn, int* derr,
                                      int lbit) {
  St<T, NINE> a(L, o);
  const T den = (a.c - a.w) - a.e;
  if (!(den > T(0))) atomicOr(derr, DEV_BADDEN | lbit);
  ws = ((a.s + a.sw) + a.se) / den;
  wn = ((a.n + a.nw) + a.ne) / den;
}

// One thread per coarse-grid index (I, J), 0 <= I <= ncx, 0 <= J <= ncy
// (ncx = floor(nx / 2)).  Computes the weights of the x-edge point
// (2I+1, 2J), the y-edge point (2I, 2J+1) and the centre point (2I+1, 2J+1)
// where those fine points exist: on an even side the last fine point is a
// coarse point, so column 2I+1 (or row 2J+1) may lie beyond the grid; its
// weights stay zero and nothing is read there.  The centre point's four edge
// neighbours are recomputed here with the same code, so the stored edge
// weights and the ones used for the centre agree bit for bit.
template <typename T, bool NINE>
__global__ void k_interp_weights(LevelV<T> F, int ncx, int ncy, int* derr, int level) {
  const int lbit = 1 << (8 + level);
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y;
  if (I > ncx || J > ncy) return;
  const int p = F.pitch, cp = F.cpitch;
  const int c = J * cp + I;
  const bool col_odd = 2 * I + 1 <= F.nx;   // fine column 2I+1 exists
  const bool row_odd = 2 * J + 1 <= F.ny;   // fine row 2J+1 exists
  T xw0 = 0, xe0 = 0, xw1 = 0, xe1 = 0, ys0 = 0, yn0 = 0, ys1 = 0, yn1 = 0;
  // x-edge (2I+1, 2J) and (2I+1, 2J+2)
  if (col_odd && J >= 1) xedge<T, NINE>(F, (2 * J) * p + 2 * I + 1, xw0, xe0, derr, lbit);
  if (col_odd && J + 1 <= ncy)
    xedge<T, NINE>(F, (2 * J + 2) * p + 2 * I + 1, xw1, xe1, derr, lbit);
  // y-edge (2I, 2J+1) and (2I+2, 2J+1)
  if (row_odd && I >= 1) yedge<T, NINE>(F, (2 * J + 1) * p + 2 * I, ys0, yn0, derr, lbit);
  if (row_odd && I + 1 <= ncx)
    yedge<T, NINE>(F, (2 * J + 1) * p + 2 * I + 2, ys1, yn1, derr, lbit);
  if (col_odd && J >= 1) {
    F.P[XW][c] = xw0;
    F.P[XE][c] = xe0;
  }
  if (row_odd && I >= 1) {
    F.P[YS][c] = ys0;
    F.P[YN][c] = yn0;
  }
  if (!(col_odd && row_odd)) return;
  // centre (2I+1, 2J+1): the fine equation with the edge neighbours replaced
  // by their interpolants.
  St<T, NINE> a(F, (2 * J + 1) * p + 2 * I + 1);
  F.P[CSW][c] = ((a.sw + a.w * ys0) + a.s * xw0) / a.c;
  F.P[CSE][c] = ((a.se + a.e * ys1) + a.s * xe0) / a.c;
  F.P[CNW][c] = ((a.nw + a.w * yn0) + a.n * xw1) / a.c;
  F.P[CNE][c] = ((a.ne + a.e * yn1) + a.n * xe1) / a.c;
}

// Matrix entry A[p, p + (dx, dy)] of the fine operator at plane offset o.
template <typename T, bool NINE>
__device__ __forceinline__ T aentry(const LevelV<T>& L, int o, int dx, int dy) {
  const int p = L.pitch;
  if (dx == 0 && dy == 0) return L.C[o];
  if (dy == 0) return dx < 0 ? -L.W[o] : -L.W[o + 1];
  if (dx == 0) return dy < 0 ? -L.S[o] : -L.S[o + p];
  if (!NINE) return T(0);
  if (dx < 0 && dy < 0) return -L.SW[o];
  if (dx > 0 && dy > 0) return -L.SW[o + 1 + p];
  if (dx < 0 && dy > 0) return -L.NW[o];
  return -L.NW[o + 1 - p];
}

// Galerkin entry A_c[(I,J), (I+DX, J+DY)] = sum_{p near 2I} P(p, I)
// sum_{q near p} A(p, q) P(q, I + D).  Terms whose q lies outside the support
// of P(., I + D) are removed at compile time after unrolling.
template <typename T, bool NINE, int DX, int DY>
__device__ __forceinline__ T rap_entry(const LevelV<T>& F, int I, int J) {
  const int p = F.pitch, cp = F.cpitch;
  const int c = J * cp + I;
  const int ct = (J + DY) * cp + (I + DX);
  T sum = T(0);
#pragma unroll
  for (int py = -1; py <= 1; ++py) {
#pragma unroll
    for (int px = -1; px <= 1; ++px) {
      // fine points beyond an even side do not exist (their weights are 0)
      if (2 * I + px > F.nx || 2 * J + py > F.ny) continue;
      const int o = (2 * J + py) * p + (2 * I + px);
      T inner = T(0);
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const int rx = px + dx - 2 * DX, ry = py + dy - 2 * DY;
          if (rx < -1 || rx > 1 || ry < -1 || ry > 1) continue;
          if (!NINE && dx != 0 && dy != 0) continue;
          inner = fma(aentry<T, NINE>(F, o, dx, dy), pweight<T>(F.P, cp, rx, ry, ct), inner);
        }
      }
      sum = fma(pweight<T>(F.P, cp, px, py, c), inner, sum);
    }
  }
  return sum;
}

// One thread per interior coarse point: the five stored planes of A_{l-1}.
template <typename T, bool NINE>
__global__ void k_rap(LevelV<T> F, LevelV<T> Cc) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int J = blockIdx.y + 1;
  if (I > Cc.nx) return;
  const int o = J * Cc.pitch + I;
  const T cc = rap_entry<T, NINE, 0, 0>(F, I, J);
  Cc.C[o] = cc;
  Cc.iC[o] = T(1) / cc;
  Cc.W[o] = I > 1 ? -rap_entry<T, NINE, -1, 0>(F, I, J) : T(0);
  Cc.S[o] = J > 1 ? -rap_entry<T, NINE, 0, -1>(F, I, J) : T(0);
  Cc.SW[o] = (I > 1 && J > 1) ? -rap_entry<T, NINE, -1, -1>(F, I, J) : T(0);
  Cc.NW[o] = (I > 1 && J < Cc.ny) ? -rap_entry<T, NINE, -1, 1>(F, I, J) : T(0);
}

// Dense A_0 (FP64) from the coarsest planes, then an in-place right-looking
// Cholesky factorisation in one thread block; stores 1/L[i][i] too.
template <typename T>
__global__ void k_coarse_factor(LevelV<T> L0, double* __restrict__ a, double* __restrict__ idiag,
                                int* derr) {
  const int nx = L0.nx, ny = L0.ny, n = nx * ny, p = L0.pitch;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) a[e] = 0.0;
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const int i = r % nx + 1, j = r / nx + 1, o = j * p + i;
    a[size_t(r) * n + r] = double(L0.C[o]);
    auto put = [&](int di, int dj, double v) {
      const int ii = i + di, jj = j + dj;
      if (ii < 1 || ii > nx || jj < 1 || jj > ny) return;
      a[size_t(r) * n + (jj - 1) * nx + (ii - 1)] = -v;
    };
    put(-1, 0, double(L0.W[o]));
    put(1, 0, double(L0.W[o + 1]));
    put(0, -1, double(L0.S[o]));
    put(0, 1, double(L0.S[o + p]));
    if (L0.SW) {
      put(-1, -1, double(L0.SW[o]));
      put(1, 1, double(L0.SW[o + 1 + p]));
      put(-1, 1, double(L0.NW[o]));
      put(1, -1, double(L0.NW[o + 1 - p]));
    }
  }
  __syncthreads();
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      const double d = a[size_t(k) * n + k];
      if (!(d > 0.0)) {
        bad = 1;
        atomicOr(derr, DEV_NOTSPD);
      }
      const double s = sqrt(d > 0.0 ? d : 1.0);
      a[size_t(k) * n + k] = s;
      idiag[k] = 1.0 / s;
    }
    __syncthreads();
    if (bad) return;
    const double inv = idiag[k];
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) a[size_t(i) * n + k] *= inv;
    __syncthreads();
    const int m = n - k - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = k + 1 + e / m, j = k + 1 + e % m;
      if (j <= i) a[size_t(i) * n + j] -= a[size_t(i) * n + k] * a[size_t(j) * n + k];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x)
    if (e % n > e / n) a[e] = 0.0;
}

__global__ void k_downcast(LevelV<double> D, LevelV<float> F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int j = blockIdx.y + 1;
  if (i > D.nx) return;
  const int od = j * D.pitch + i, of = j * F.pitch + i;
  F.C[of] = float(D.C[od]);
  F.iC[of] = float(D.iC[od]);
  F.W[of] = float(D.W[od]);
  F.S[of] = float(D.S[od]);
}

template <typename T>
__global__ void k_pack(const double* __restrict__ src, T* __restrict__ dst, int nx, int pitch) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= nx) return;
  dst[(j + 1) * pitch + i + 1] = T(src[size_t(j) * nx + i]);
}

template <typename T>
__global__ void k_unpack(const T* __restrict__ src, double* __restrict__ dst, int nx, int pitch) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= nx) return;
  dst[size_t(j) * nx + i] = double(src[(j + 1) * pitch + i + 1]);
}

// Backward of the assembly, one thread per cell (dense arrays):
// g_c = -k_c [ sum_faces 2 k_n^2/(k_c + k_n)^2 (u_c - u_n)(lam_c - lam_n)
//              + (#boundary faces) 2 u_c lam_c ].
__global__ void k_assemble_backward(const double* __restrict__ k, const double* __restrict__ u,
                                    const double* __restrict__ lam, double* __restrict__ g,
                                    int nx, int ny) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= nx) return;
  const size_t q = size_t(j) * nx + i;
  const double kc = k[q], uc = u[q], lc = lam[q];
  double acc = 0.0;
  int nb = 0;
  auto face = [&](size_t qn) {
    const double kn = k[qn];
    const double s = kc + kn;
    acc += 2.0 * kn * kn / (s * s) * ((uc - u[qn]) * (lc - lam[qn]));
  };
  if (i > 0) face(q - 1); else ++nb;
  if (i < nx - 1) face(q + 1); else ++nb;
  if (j > 0) face(q - nx); else ++nb;
  if (j < ny - 1) face(q + nx); else ++nb;
  acc += double(nb) * 2.0 * uc * lc;
  g[q] = -kc * acc;
}

}  // namespace

template <typename T>
int launch_assemble(const double* k, int nx, int ny, LevelV<T> L, double* kcopy, int* derr,
                    bool log_k, double r, double aspect, const double* bc_beta, cudaStream_t s) {
  const AssemblyScale f{1.0 / r, r, aspect, 1.0 / aspect,
                        {bc_beta[0], bc_beta[1], bc_beta[2], bc_beta[3]}};
  k_assemble<T><<<dim3(cdiv(nx, kAX), cdiv(ny, kAY)), dim3(kAX, kAY), 0, s>>>(k, nx, ny, L, kcopy,
                                                                            derr, log_k, f);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : BMG_ECUDA;
}

template <typename T>
int launch_interp_weights(const LevelV<T>& fine, bool nine, int* derr, int level, cudaStream_t s) {
  const int ncx = fine.nx / 2, ncy = fine.ny / 2;
  dim3 grid(cdiv(ncx + 1, 128), ncy + 1);
  if (nine)
    k_interp_weights<T, true><<<grid, 128, 0, s>>>(fine, ncx, ncy, derr, level);
  else
    k_interp_weights<T, false><<<grid, 128, 0, s>>>(fine, ncx, ncy, derr, level);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : BMG_ECUDA;
}

template <typename T>
int launch_rap(const LevelV<T>& fine, bool nine, LevelV<T> coarse, cudaStream_t s) {
  dim3 grid(cdiv(coarse.nx, 128), coarse.ny);
  if (nine)
    k_rap<T, true><<<grid, 128, 0, s>>>(fine, coarse);
  else
    k_rap<T, false><<<grid, 128, 0, s>>>(fine, coarse);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : BMG_ECUDA;
}

int launch_coarse_factor(Hierarchy* h, const LevelV<double>* l0d, const LevelV<float>* l0f,
                         cudaStream_t s) {
  int* derr = &h->sc->err;
  if (l0d)
    k_coarse_factor<double><<<1, 512, 0, s>>>(*l0d, h->chol, h->chol_idiag, derr);
  else
    k_coarse_factor<float><<<1, 512, 0, s>>>(*l0f, h->chol, h->chol_idiag, derr);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : BMG_ECUDA;
}

int launch_downcast_fine(const LevelV<double>& d, LevelV<float> f, cudaStream_t s) {
  k_downcast<<<dim3(cdiv(d.nx, kTB), d.ny), kTB, 0, s>>>(d, f);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : BMG_ECUDA;
}

template <typename T>
void launch_pack(const double* src, T* dst, int nx, int ny, int pitch, cudaStream_t s) {
  k_pack<T><<<dim3(cdiv(nx, kTB), ny), kTB, 0, s>>>(src, dst, nx, pitch);
  count_launch();
}

template <typename T>
void launch_unpack(const T* src, double* dst, int nx, int ny, int pitch, cudaStream_t s) {
  k_unpack<T><<<dim3(cdiv(nx, kTB), ny), kTB, 0, s>>>(src, dst, nx, pitch);
  count_launch();
}

void launch_assemble_backward(const double* k, const double* u, const double* lam, double* g,
                              int nx, int ny, cudaStream_t s) {
  k_assemble_backward<<<dim3(cdiv(nx, kTB), ny), kTB, 0, s>>>(k, u, lam, g, nx, ny);
  count_launch();
}

template int launch_assemble<double>(const double*, int, int, LevelV<double>, double*, int*,
                                     bool, double, double, const double*, cudaStream_t);
template int launch_interp_weights<double>(const LevelV<double>&, bool, int*, int, cudaStream_t);
template int launch_interp_weights<float>(const LevelV<float>&, bool, int*, int, cudaStream_t);
template int launch_rap<double>(const LevelV<double>&, bool, LevelV<double>, cudaStream_t);
template int launch_rap<float>(const LevelV<float>&, bool, LevelV<float>, cudaStream_t);
template void launch_pack<double>(const double*, double*, int, int, int, cudaStream_t);
template void launch_pack<float>(const double*, float*, int, int, int, cudaStream_t);
template void launch_unpack<double>(const double*, double*, int, int, int, cudaStream_t);
template void launch_unpack<float>(const float*, double*, int, int, int, cudaStream_t);

}  // namespace bmg
