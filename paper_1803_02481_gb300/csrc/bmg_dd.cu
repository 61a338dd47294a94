// Domain decomposition (Section 2.1) and redistribution (Section 2.2,
// Algorithm 2): one rank's part of a distributed hierarchy.
//
// The ranks form a px x py processor grid; on every distributed level each
// owns a rectangular block of points.  A block is stored like a full level
// (the LevelV layout: interior rows 128-byte aligned, a one-point ring), so
// the ring holds the neighbours' values -- the width-1 halo of Section 2.1 --
// and the full-level kernels (residual, restriction, interpolation and the
// per-point Gauss-Seidel update) run on it unchanged.  The operator and
// interpolation planes of a block, ring included, come from the caller
// (setup scatters them); the vectors' rings are filled by the caller's halo
// exchange through bmg_dd_copy.  The gather level (part level 0) holds only
// the restricted right-hand side and the scattered coarse solution.
//
// Blocks start at 0-based global indices that are multiples of 2^d, d the
// number of coarsenings between the finest and the gather level, so local
// and global parities agree on every level: the colours, the coarse point
// 2I and the restriction and interpolation offsets are the full-level ones.
#include "bmg_internal.h"
#include "bmg_coarse.cuh"

namespace bmg {

namespace {

constexpr int kDT = 128;
constexpr int kDN = 256;

inline int cdiv(long a, long b) { return int((a + b - 1) / b); }

// One colour of multicolour Gauss-Seidel on a block, in place: the points of
// one colour are not coupled, so each update reads only other colours.
template <typename T, bool NINE>
__global__ void k_dd_colour(LevelV<T> L, unsigned mask) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int j = blockIdx.y + 1;
  if (i > L.nx) return;
  const int sub = 2 * ((j - 1) & 1) + ((i - 1) & 1);
  if (!(mask & (1u << sub))) return;
  const int o = j * L.pitch + i;
  L.x[o] = gs_value<T, NINE>(L, L.x, L.b[o], o);
}

__global__ void k_dd_inverse(LevelV<double> L) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int j = blockIdx.y + 1;
  if (i > L.nx) return;
  const int o = j * L.pitch + i;
  L.iC[o] = 1.0 / L.C[o];
}

// Per block row: sum of r^2 and of b^2 over the owned points.
__global__ void __launch_bounds__(kDN) k_dd_row_norms(LevelV<double> L, double* rows) {
  __shared__ double red[2][kDN / 32];
  const int j = blockIdx.x + 1;
  double rr = 0.0, bb = 0.0;
  for (int i = threadIdx.x + 1; i <= L.nx; i += blockDim.x) {
    const int o = j * L.pitch + i;
    rr = fma(L.r[o], L.r[o], rr);
    bb = fma(L.b[o], L.b[o], bb);
  }
  for (int off = 16; off > 0; off >>= 1) {
    rr += __shfl_xor_sync(0xffffffffu, rr, off);
    bb += __shfl_xor_sync(0xffffffffu, bb, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = rr;
    red[1][threadIdx.x >> 5] = bb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int w = 0; w < kDN / 32; ++w) {
      a += red[0][w];
      c += red[1][w];
    }
    rows[2 * blockIdx.x] = a;
    rows[2 * blockIdx.x + 1] = c;
  }
}

// The row sums in row order (a fixed order: the result is deterministic).
__global__ void k_dd_sum_rows(const double* rows, int ny, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0.0, c = 0.0;
  for (int j = 0; j < ny; ++j) {
    a += rows[2 * j];
    c += rows[2 * j + 1];
  }
  out[0] = a;
  out[1] = c;
}

}  // namespace

struct DDPart {
  int nlev = 0;
  std::vector<LevelV<double>> lv;
  std::vector<int> nine;
  char* arena = nullptr;
  double* rows = nullptr;      // 2 doubles per row of the largest block
  double* sums = nullptr;      // 2 doubles
};

namespace {

struct DDCarver {
  char* base = nullptr;
  size_t off = 0;
  double* plane(const Geom& g) {
    off = (off + 255) & ~size_t(255);
    double* p = base ? reinterpret_cast<double*>(base + off) + base_shift<double>() : nullptr;
    off += g.elems * sizeof(double);
    return p;
  }
  double* raw(size_t n) {
    off = (off + 255) & ~size_t(255);
    double* p = base ? reinterpret_cast<double*>(base + off) : nullptr;
    off += n * sizeof(double);
    return p;
  }
};

void carve(DDPart* d, DDCarver& cv, const int* nx, const int* ny) {
  int maxrows = 1;
  for (int k = 0; k < d->nlev; ++k) {
    const Geom g = make_geom<double>(nx[k], ny[k]);
    LevelV<double>& L = d->lv[k];
    L = LevelV<double>{};
    L.nx = nx[k];
    L.ny = ny[k];
    L.pitch = g.pitch;
    L.x = cv.plane(g);
    L.b = cv.plane(g);
    if (k >= 1) {
      L.C = cv.plane(g);
      L.iC = cv.plane(g);
      L.W = cv.plane(g);
      L.S = cv.plane(g);
      L.SW = d->nine[k] ? cv.plane(g) : nullptr;
      L.NW = d->nine[k] ? cv.plane(g) : nullptr;
      L.r = cv.plane(g);
      const Geom gc = make_geom<double>(nx[k - 1], ny[k - 1]);
      for (int q = 0; q < NPW; ++q) L.P[q] = cv.plane(gc);
      L.cpitch = gc.pitch;
    }
    maxrows = std::max(maxrows, ny[k]);
  }
  d->rows = cv.raw(2 * size_t(maxrows));
  d->sums = cv.raw(2);
}

// Host (rows, cols) = (ny + 2, nx + 2) array, ring included, into a plane.
cudaError_t upload(double* plane, int pitch, const double* host, int nx, int ny, cudaStream_t s) {
  return cudaMemcpy2DAsync(plane, size_t(pitch) * sizeof(double), host, size_t(nx + 2) * sizeof(double),
                           size_t(nx + 2) * sizeof(double), size_t(ny + 2), cudaMemcpyHostToDevice, s);
}

DDPart* P(bmg_dd_part* p) { return reinterpret_cast<DDPart*>(p); }

int check(bmg_dd_part* p, int k, int min_level) {
  if (!p) return BMG_EINVAL;
  if (k < min_level || k >= P(p)->nlev) {
    set_last_error("dd: part level %d out of range [%d, %d)", k, min_level, P(p)->nlev);
    return BMG_EINVAL;
  }
  return BMG_OK;
}

int launched() { return cudaGetLastError() == cudaSuccess ? BMG_OK : BMG_ECUDA; }

double* vec_of(const LevelV<double>& L, int vec) {
  return vec == BMG_DD_X ? L.x : vec == BMG_DD_B ? L.b : vec == BMG_DD_R ? L.r : nullptr;
}

}  // namespace

}  // namespace bmg

using bmg::DDPart;

extern "C" {

int bmg_dd_part_create(int nlev, const int* nx, const int* ny, const int* nine,
                       const double* const* stencil_host, const double* const* interp_host,
                       bmg_stream_t stream, bmg_dd_part** out) {
  if (!out) return BMG_EINVAL;
  *out = nullptr;
  if (nlev < 2 || !nx || !ny || !nine || !stencil_host || !interp_host) return BMG_EINVAL;
  for (int k = 0; k < nlev; ++k) {
    if (nx[k] < 1 || ny[k] < 1 || (k >= 1 && (!stencil_host[k] || !interp_host[k]))) {
      bmg::set_last_error("dd: level %d: empty block or missing planes", k);
      return BMG_EINVAL;
    }
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  DDPart* d = new (std::nothrow) DDPart();
  if (!d) return BMG_ENOMEM;
  d->nlev = nlev;
  d->lv.resize(nlev);
  d->nine.assign(nine, nine + nlev);
  bmg::DDCarver cv;
  bmg::carve(d, cv, nx, ny);
  const size_t bytes = cv.off;
  if (cudaMalloc(&d->arena, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete d;
    return BMG_ENOMEM;
  }
  cv.base = d->arena;
  cv.off = 0;
  bmg::carve(d, cv, nx, ny);
  int rc = cudaMemsetAsync(d->arena, 0, bytes, s) == cudaSuccess ? BMG_OK : BMG_ECUDA;
  for (int k = 1; k < nlev && rc == BMG_OK; ++k) {
    const auto& L = d->lv[k];
    const size_t plane = size_t(nx[k] + 2) * (ny[k] + 2);
    double* dst[5] = {L.C, L.W, L.S, L.SW, L.NW};
    for (int q = 0; q < 5 && rc == BMG_OK; ++q)
      if (dst[q] && bmg::upload(dst[q], L.pitch, stencil_host[k] + q * plane, nx[k], ny[k], s) != cudaSuccess)
        rc = BMG_ECUDA;
    const size_t cplane = size_t(nx[k - 1] + 2) * (ny[k - 1] + 2);
    for (int q = 0; q < bmg::NPW && rc == BMG_OK; ++q)
      if (bmg::upload(L.P[q], L.cpitch, interp_host[k] + q * cplane, nx[k - 1], ny[k - 1], s) != cudaSuccess)
        rc = BMG_ECUDA;
    if (rc == BMG_OK) {
      bmg::k_dd_inverse<<<dim3(bmg::cdiv(L.nx, bmg::kDT), L.ny), bmg::kDT, 0, s>>>(L);
      bmg::count_launch();
    }
  }
  if (rc == BMG_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = BMG_ECUDA;
  if (rc != BMG_OK) {
    bmg::set_last_error("dd: part setup: %s", cudaGetErrorString(cudaGetLastError()));
    cudaFree(d->arena);
    delete d;
    return rc;
  }
  *out = reinterpret_cast<bmg_dd_part*>(d);
  return BMG_OK;
}

void bmg_dd_part_destroy(bmg_dd_part* p) {
  if (!p) return;
  DDPart* d = bmg::P(p);
  cudaFree(d->arena);
  delete d;
}

int bmg_dd_relax_colour(bmg_dd_part* p, int k, int colour, bmg_stream_t stream) {
  if (int rc = bmg::check(p, k, 1)) return rc;
  DDPart* d = bmg::P(p);
  const bool nine = d->nine[k] != 0;
  if (colour < 0 || colour >= (nine ? 4 : 2)) return BMG_EINVAL;
  const auto& L = d->lv[k];
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const dim3 grid(bmg::cdiv(L.nx, bmg::kDT), L.ny);
  if (nine)
    bmg::k_dd_colour<double, true><<<grid, bmg::kDT, 0, s>>>(L, bmg::four_mask(colour));
  else
    bmg::k_dd_colour<double, false><<<grid, bmg::kDT, 0, s>>>(L, bmg::rb_mask(colour));
  bmg::count_launch();
  return bmg::launched();
}

int bmg_dd_residual(bmg_dd_part* p, int k, bmg_stream_t stream) {
  if (int rc = bmg::check(p, k, 1)) return rc;
  DDPart* d = bmg::P(p);
  const auto& L = d->lv[k];
  bmg::launch_residual<double>(L, d->nine[k] != 0, L.x, L.b, L.r, reinterpret_cast<cudaStream_t>(stream));
  return bmg::launched();
}

int bmg_dd_restrict(bmg_dd_part* p, int k, bmg_stream_t stream) {
  if (int rc = bmg::check(p, k, 1)) return rc;
  DDPart* d = bmg::P(p);
  bmg::launch_restrict<double>(d->lv[k], d->lv[k].r, d->lv[k - 1], true, reinterpret_cast<cudaStream_t>(stream));
  return bmg::launched();
}

int bmg_dd_interp(bmg_dd_part* p, int k, bmg_stream_t stream) {
  if (int rc = bmg::check(p, k, 1)) return rc;
  DDPart* d = bmg::P(p);
  bmg::launch_interp<double>(d->lv[k], d->lv[k - 1].x, false, reinterpret_cast<cudaStream_t>(stream));
  return bmg::launched();
}

int bmg_dd_norms(bmg_dd_part* p, int k, double* out2_host, bmg_stream_t stream) {
  if (int rc = bmg::check(p, k, 1)) return rc;
  if (!out2_host) return BMG_EINVAL;
  DDPart* d = bmg::P(p);
  const auto& L = d->lv[k];
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  bmg::k_dd_row_norms<<<L.ny, bmg::kDN, 0, s>>>(L, d->rows);
  bmg::k_dd_sum_rows<<<1, 32, 0, s>>>(d->rows, L.ny, d->sums);
  bmg::count_launch(2);
  if (cudaMemcpyAsync(out2_host, d->sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return BMG_ECUDA;
  return BMG_OK;
}

int bmg_dd_copy(bmg_dd_part* p, int k, int vec, int side, int dir, double* buf_dev, bmg_stream_t stream) {
  if (int rc = bmg::check(p, k, 0)) return rc;
  DDPart* d = bmg::P(p);
  const auto& L = d->lv[k];
  double* v = bmg::vec_of(L, vec);
  if (!v || !buf_dev || side < BMG_DD_WEST || side > BMG_DD_NORTH || (dir != 0 && dir != 1)) return BMG_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t w = sizeof(double), pitch = size_t(L.pitch) * w;
  cudaError_t e;
  if (side == BMG_DD_WEST || side == BMG_DD_EAST) {
    // column strip, rows 1..ny: get the owned edge column, put the ring column
    const int col = side == BMG_DD_WEST ? (dir == 0 ? 1 : 0) : (dir == 0 ? L.nx : L.nx + 1);
    double* at = v + L.pitch + col;
    e = dir == 0 ? cudaMemcpy2DAsync(buf_dev, w, at, pitch, w, L.ny, cudaMemcpyDeviceToDevice, s)
                 : cudaMemcpy2DAsync(at, pitch, buf_dev, w, w, L.ny, cudaMemcpyDeviceToDevice, s);
  } else {
    // row strip, columns 0..nx+1 (the ring columns carry the corners)
    const int row = side == BMG_DD_SOUTH ? (dir == 0 ? 1 : 0) : (dir == 0 ? L.ny : L.ny + 1);
    double* at = v + size_t(row) * L.pitch;
    e = dir == 0 ? cudaMemcpyAsync(buf_dev, at, (L.nx + 2) * w, cudaMemcpyDeviceToDevice, s)
                 : cudaMemcpyAsync(at, buf_dev, (L.nx + 2) * w, cudaMemcpyDeviceToDevice, s);
  }
  return e == cudaSuccess ? BMG_OK : BMG_ECUDA;
}

int bmg_dd_block(bmg_dd_part* p, int k, int vec, int dir, int ring, double* dense_dev,
                 bmg_stream_t stream) {
  if (int rc = bmg::check(p, k, 0)) return rc;
  DDPart* d = bmg::P(p);
  const auto& L = d->lv[k];
  double* v = bmg::vec_of(L, vec);
  if (!v || !dense_dev || (dir != 0 && dir != 1)) return BMG_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t w = sizeof(double), pitch = size_t(L.pitch) * w;
  const int cols = ring ? L.nx + 2 : L.nx, rows = ring ? L.ny + 2 : L.ny;
  double* at = ring ? v : v + L.pitch + 1;
  const cudaError_t e =
      dir == 0 ? cudaMemcpy2DAsync(dense_dev, cols * w, at, pitch, cols * w, rows, cudaMemcpyDeviceToDevice, s)
               : cudaMemcpy2DAsync(at, pitch, dense_dev, cols * w, cols * w, rows, cudaMemcpyDeviceToDevice, s);
  return e == cudaSuccess ? BMG_OK : BMG_ECUDA;
}

}  // extern "C"
