// One multicolour Gauss-Seidel sweep per kernel launch (smoothing of
// Algorithm 1; red-black on 5-point levels, four colours on 9-point levels,
// Section 5).  The tile body is in bmg_sweep_tile.cuh.
#include <cstdlib>

#include "bmg_sweep_stream.cuh"
#include "bmg_sweep_tile.cuh"

namespace bmg {

namespace {

inline int cdiv(long a, long b) { return int((a + b - 1) / b); }

template <typename T, bool NINE, int TX, int TY, int NT, int U = (NINE ? 3 : 1)>
__global__ void __launch_bounds__(NT) k_sweep(LevelV<T> L, const T* __restrict__ xin,
                                              T* __restrict__ xout, unsigned order) {
  sweep_tile<T, NINE, TX, TY, NT, U>(L, xin, xout, order, blockIdx.x, blockIdx.y);
}

}  // namespace

// Streaming kernel shape: 64 threads own a 126-column strip, 32 rows per
// block (36 KB of shared memory in FP64: six blocks per SM).
constexpr int kStreamNT = 64, kStreamR = 32;

// Kernel for large 5-point levels: 0 = streaming strips, 1 = tiled (one
// point per thread step, the default: measured fastest), 2 = tiled with two
// points' loads issued together.  BMG_RB_KERNEL overrides the default, for
// measurements.
static int rb_kernel_choice() {
  static const int v = [] {
    const char* e = std::getenv("BMG_RB_KERNEL");
    return e ? std::atoi(e) : 1;
  }();
  return v;
}
static bool stream_rb_enabled() { return rb_kernel_choice() == 0; }

template <typename T>
void launch_sweep(const LevelV<T>& L, bool nine, bool reverse, const T* xin, T* xout,
                  cudaStream_t s) {
  // Large tiles keep the redundant halo work small (4% red-black, 12% four
  // colours); levels narrower than 1024 use small tiles so that they still
  // spread over all SMs.
  const bool small = L.nx < 1024;
  if (nine) {
    if (small) {
      constexpr int TX = 32, TY = 16;
      k_sweep<T, true, TX, TY, 128><<<dim3(cdiv(L.nx, TX), cdiv(L.ny, TY)), 128, 0, s>>>(
          L, xin, xout, four_order(reverse));
    } else {
      constexpr int TX = 128, TY = 32;
      k_sweep<T, true, TX, TY, 256><<<dim3(cdiv(L.nx, TX), cdiv(L.ny, TY)), 256, 0, s>>>(
          L, xin, xout, four_order(reverse));
    }
  } else {
    if (small) {
      constexpr int TX = 32, TY = 16;
      k_sweep<T, false, TX, TY, 128><<<dim3(cdiv(L.nx, TX), cdiv(L.ny, TY)), 128, 0, s>>>(
          L, xin, xout, rb_order(reverse));
    } else if (stream_rb_enabled()) {
      constexpr int NT = kStreamNT, R = kStreamR;
      using S = StreamRB<T, NT, R>;
      const size_t smem = sizeof(typename S::Row) * S::NSLOT;
      k_sweep_rb_stream<T, NT, R><<<dim3(cdiv(L.nx, S::OWN), cdiv(L.ny, R)), NT, smem, s>>>(
          L, xin, xout, reverse ? 1 : 0);
    } else if (rb_kernel_choice() == 2) {
      constexpr int TX = 128, TY = 32;
      k_sweep<T, false, TX, TY, 256, 2><<<dim3(cdiv(L.nx, TX), cdiv(L.ny, TY)), 256, 0, s>>>(
          L, xin, xout, rb_order(reverse));
    } else {
      constexpr int TX = 128, TY = 32;
      k_sweep<T, false, TX, TY, 256><<<dim3(cdiv(L.nx, TX), cdiv(L.ny, TY)), 256, 0, s>>>(
          L, xin, xout, rb_order(reverse));
    }
  }
  count_launch();
}

// Opt the streaming kernels into more than 48 KB of dynamic shared memory
// (once per process, before any launch or graph capture).
void prepare_sweep_kernels() {
  static const bool done = [] {
    using S64 = StreamRB<double, kStreamNT, kStreamR>;
    using S32 = StreamRB<float, kStreamNT, kStreamR>;
    cudaFuncSetAttribute(k_sweep_rb_stream<double, kStreamNT, kStreamR>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         int(sizeof(S64::Row) * S64::NSLOT));
    cudaFuncSetAttribute(k_sweep_rb_stream<float, kStreamNT, kStreamR>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         int(sizeof(S32::Row) * S32::NSLOT));
    return true;
  }();
  (void)done;
}

template void launch_sweep<double>(const LevelV<double>&, bool, bool, const double*, double*,
                                   cudaStream_t);
template void launch_sweep<float>(const LevelV<float>&, bool, bool, const float*, float*,
                                  cudaStream_t);

}  // namespace bmg
