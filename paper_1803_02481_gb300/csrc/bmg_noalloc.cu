// Allocation-free residual norm: ||b - A(k) x||_2 and ||b||_2 for the 5-point
// finite-volume operator, assembled from k on the fly, with the reduction
// scratch in a file-scope device array instead of memory from cudaMalloc.
//
// Who needs this: programs that do not let third-party code allocate device
// memory (a framework that reserves the GPU's memory up front and hands out
// every buffer from its own pool), and latency-critical loops where a
// cudaMalloc/cudaFree pair, which can synchronise the whole device, is not
// acceptable.  Such callers cannot create a bmg_hierarchy (bmg_setup
// allocates), but they can still check a solution with this call.
#include "bmg_internal.h"

#include <mutex>

namespace bmg {

namespace {

// One partial sum pair (residual^2, b^2) per grid row.  Every GPU that loads
// the library holds this array until the process exits.
constexpr int kNoAllocMaxRows = 16384;
static __device__ __align__(256) double g_noalloc_rows[2 * kNoAllocMaxRows];

constexpr int kRowThreads = 256;

__device__ __forceinline__ double face(double k1, double k2) { return 2.0 * k1 * k2 / (k1 + k2); }

__device__ __forceinline__ double warp_block_sum(double v, double* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = v;
  __syncthreads();
  v = lane < kRowThreads / 32 ? red[lane] : 0.0;
  if (w == 0) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  }
  __syncthreads();
  return v;
}

// One block per row j: writes that row's sum of r^2 and of b^2 into the
// scratch (every row's slots are overwritten, so nothing needs clearing).
__global__ void __launch_bounds__(kRowThreads) k_resid_rows_static(
    const double* __restrict__ k, const double* __restrict__ x, const double* __restrict__ b,
    int nx, int ny, double* rows) {
  __shared__ double red[kRowThreads / 32];
  const int j = blockIdx.x;
  double rr = 0.0, bb = 0.0;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const size_t q = size_t(j) * nx + i;
    const double kc = k[q], xc = x[q];
    double c = 0.0, ax = 0.0;
    if (i > 0) { const double a = face(k[q - 1], kc); c += a; ax += a * x[q - 1]; } else { c += 2.0 * kc; }
    if (i < nx - 1) { const double a = face(kc, k[q + 1]); c += a; ax += a * x[q + 1]; } else { c += 2.0 * kc; }
    if (j > 0) { const double a = face(k[q - nx], kc); c += a; ax += a * x[q - nx]; } else { c += 2.0 * kc; }
    if (j < ny - 1) { const double a = face(kc, k[q + nx]); c += a; ax += a * x[q + nx]; } else { c += 2.0 * kc; }
    const double r = b[q] - (c * xc - ax);
    rr = fma(r, r, rr);
    bb = fma(b[q], b[q], bb);
  }
  rr = warp_block_sum(rr, red);
  bb = warp_block_sum(bb, red);
  if (threadIdx.x == 0) {
    rows[2 * j] = rr;
    rows[2 * j + 1] = bb;
  }
}

// Sums the row partials in a fixed order and writes the two norms.
__global__ void __launch_bounds__(kRowThreads) k_resid_rows_final(const double* rows, int ny,
                                                                  double* out) {
  __shared__ double red[kRowThreads / 32];
  double rr = 0.0, bb = 0.0;
  for (int j = threadIdx.x; j < ny; j += blockDim.x) {
    rr += rows[2 * j];
    bb += rows[2 * j + 1];
  }
  rr = warp_block_sum(rr, red);
  bb = warp_block_sum(bb, red);
  if (threadIdx.x == 0) {
    out[0] = sqrt(rr);
    out[1] = sqrt(bb);
  }
}

// Device address of the scratch array, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {};

int noalloc_scratch(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BMG_ECUDA;
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_rows) != cudaSuccess || !p) {
      cudaGetLastError();
      return BMG_ECUDA;
    }
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return BMG_OK;
}

}  // namespace

}  // namespace bmg

extern "C" int bmg_residual_norm_noalloc(const double* k_dev, const double* x_dev,
                                         const double* b_dev, int nx, int ny, double* norms_dev,
                                         bmg_stream_t stream) {
  if (!k_dev || !x_dev || !b_dev || !norms_dev || nx < 1 || ny < 1) {
    bmg::set_last_error("residual_norm_noalloc: null pointer or empty grid");
    return BMG_EINVAL;
  }
  if (ny > bmg::kNoAllocMaxRows) {
    bmg::set_last_error("residual_norm_noalloc: ny = %d exceeds the maximum of %d rows", ny,
                        bmg::kNoAllocMaxRows);
    return BMG_EINVAL;
  }
  double* rows = nullptr;
  if (int rc = bmg::noalloc_scratch(&rows)) {
    bmg::set_last_error("residual_norm_noalloc: cudaGetSymbolAddress failed");
    return rc;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  bmg::k_resid_rows_static<<<ny, bmg::kRowThreads, 0, s>>>(k_dev, x_dev, b_dev, nx, ny, rows);
  bmg::k_resid_rows_final<<<1, bmg::kRowThreads, 0, s>>>(rows, ny, norms_dev);
  bmg::count_launch(2);
  if (cudaGetLastError() != cudaSuccess) {
    bmg::set_last_error("residual_norm_noalloc: kernel launch failed");
    return BMG_ECUDA;
  }
  return BMG_OK;
}
