// One multicolour Gauss-Seidel sweep per kernel launch (smoothing of
// Algorithm 1; red-black on 5-point levels, four colours on 9-point levels,
// Section 5).  The tile body is in bmg_sweep_tile.cuh.
#include "bmg_sweep_tile.cuh"

namespace bmg {

namespace {

inline int cdiv(long a, long b) { return int((a + b - 1) / b); }

template <typename T, bool NINE, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT) k_sweep(LevelV<T> L, const T* __restrict__ xin,
                                              T* __restrict__ xout, unsigned order) {
  sweep_tile<T, NINE, TX, TY, NT>(L, xin, xout, order, blockIdx.x, blockIdx.y);
}

}  // namespace

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
    } else {
      constexpr int TX = 128, TY = 32;
      k_sweep<T, false, TX, TY, 256><<<dim3(cdiv(L.nx, TX), cdiv(L.ny, TY)), 256, 0, s>>>(
          L, xin, xout, rb_order(reverse));
    }
  }
  count_launch();
}

template void launch_sweep<double>(const LevelV<double>&, bool, bool, const double*, double*,
                                   cudaStream_t);
template void launch_sweep<float>(const LevelV<float>&, bool, bool, const float*, float*,
                                  cudaStream_t);

}  // namespace bmg
