// One multicolour Gauss-Seidel sweep per kernel launch (smoothing of
// Algorithm 1; red-black on 5-point levels, four colours on 9-point levels,
// Section 5).  The tile body is in bmg_sweep_tile.cuh.
#include <cstdlib>
#include <cstring>

#include "bmg_sweep_stream.cuh"
#include "bmg_sweep_tile.cuh"
#include "bmg_sweep_tma.cuh"

namespace bmg {

namespace {

inline int cdiv(long a, long b) { return int((a + b - 1) / b); }

template <typename T, bool NINE, int TX, int TY, int NT, int U = (NINE ? 3 : 1)>
__global__ void __launch_bounds__(NT) k_sweep(LevelV<T> L, const T* __restrict__ xin,
                                              T* __restrict__ xout, unsigned order) {
  griddep_wait();
  sweep_tile<T, NINE, TX, TY, NT, U>(L, xin, xout, order, blockIdx.x, blockIdx.y);
}

// The small-level red-black sweep carrying the stop test (sweep_tile's NRM):
// pre-smoothing order, one partial of the squared residual per block.
template <int TX, int TY, int NT>
__global__ void __launch_bounds__(NT) k_sweep_nrm(LevelV<double> L, const double* __restrict__ xin,
                                                  double* __restrict__ xout, double* __restrict__ nrm) {
  griddep_wait();
  sweep_tile<double, false, TX, TY, NT, 1, true>(L, xin, xout, rb_order(false), blockIdx.x,
                                                 blockIdx.y, nrm);
}

}  // namespace

// Streaming kernel shape: 64 threads own a 126-column strip, 32 rows per
// block (36 KB of shared memory in FP64: six blocks per SM).
constexpr int kStreamNT = 64, kStreamR = 32;

// TMA-staged kernel shapes: tile TX x TY, NT threads, MINB blocks per SM,
// NSTAGE shared-memory stages per block.  Entry 0 of each table is the
// default, the fastest measured on the GB300:
//  * 5-point levels (the finest level): FP64 64 x 16 tiles, 608 threads, two
//    blocks per SM, two stages (FP64 is ALU-bound: more warps hide the FP64
//    latency, and 608 threads give every thread one point in each colour
//    phase, 594 red points on the grown tile); FP32 128 x 16 tiles, 256
//    threads, two blocks per SM, two stages (memory-bound: four stages per
//    SM in flight).
//  * 9-point levels (2047^2 and 4095^2 levels): one stage per block and four
//    blocks per SM (FP64 40 x 16 tiles, FP32 64 x 16): with four colour
//    phases per tile, more resident warps beat a second stage.  40 x 16 is
//    the widest FP64 tile of which four blocks fit an SM; wider tiles cut the
//    redundant halo work but lose the fourth block.
// BMG_TMA_CFG (5-point) and BMG_TMA9_CFG (9-point) select other entries, for
// measurements.
struct TmaCfg {
  int tx, ty, nt, minb, nstage;
};
constexpr TmaCfg kRb64[] = {{64, 16, 608, 2, 2}, {64, 16, 512, 2, 2}, {64, 16, 512, 4, 1}};
constexpr TmaCfg kRb32[] = {{128, 16, 256, 2, 2}, {64, 16, 256, 3, 2}, {128, 16, 256, 4, 1}};
constexpr int kNumRbCfg = 3;
constexpr TmaCfg kNine64[] = {{40, 16, 256, 4, 1}, {32, 16, 256, 4, 1}, {36, 16, 256, 4, 1},
                              {36, 16, 192, 4, 1}, {28, 20, 192, 4, 1}, {40, 16, 192, 4, 1}};
constexpr TmaCfg kNine32[] = {{64, 16, 256, 4, 1}, {64, 16, 256, 5, 1}, {80, 16, 256, 4, 1},
                              {128, 8, 256, 4, 1}, {64, 32, 256, 2, 1}, {32, 32, 256, 4, 1}};
constexpr int kNumNineCfg = 6;

static int env_int(const char* name, int dflt) {
  const char* e = std::getenv(name);
  return e && e[0] ? std::atoi(e) : dflt;
}
static int nine_cfg_index() {
  static const int v = [] {
    const int k = env_int("BMG_TMA9_CFG", 0);
    return k >= 0 && k < kNumNineCfg ? k : 0;
  }();
  return v;
}
// 9-point levels narrower than this use the tiled kernel (BMG_TMA9_MIN).
static int nine_tma_min_side() {
  static const int v = env_int("BMG_TMA9_MIN", 0);
  return v;
}
static int rb_cfg_index() {
  static const int v = [] {
    const int k = env_int("BMG_TMA_CFG", 0);
    return k >= 0 && k < kNumRbCfg ? k : 0;
  }();
  return v;
}
template <typename T>
static TmaCfg tma_cfg(bool nine) {
  if (!nine) return sizeof(T) == 8 ? kRb64[rb_cfg_index()] : kRb32[rb_cfg_index()];
  return sizeof(T) == 8 ? kNine64[nine_cfg_index()] : kNine32[nine_cfg_index()];
}

// Kernel for large 5-point levels: 0 = streaming strips, 1 = tiled (one
// point per thread step), 2 = tiled with two points' loads issued together,
// 3 = persistent TMA-staged tiles (the default).  BMG_RB_KERNEL overrides the
// default, for measurements.
static int rb_kernel_choice() {
  static const int v = env_int("BMG_RB_KERNEL", 3);
  return v;
}
static bool stream_rb_enabled() { return rb_kernel_choice() == 0; }

static int sm_count() {
  static const int n = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  return n;
}

// cuTensorMapEncodeTiled, from the driver through the runtime (no link
// against libcuda).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                        &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    cudaGetLastError();
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  return fn;
}

// Descriptor of one plane (base = element (0, 0)) as a 2-D tensor of
// (ny + 2) rows of `pitch` elements, starting base_shift elements before the
// plane base (the 128-byte aligned start of its allocation), staged in boxes
// of bw x bh elements.
template <typename T>
static bool encode_plane(CUtensorMap* m, const T* base, int pitch, int ny, int bw, int bh) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn || !base) return false;
  void* start = const_cast<T*>(base - base_shift<T>());
  const cuuint64_t dims[2] = {cuuint64_t(pitch), cuuint64_t(ny + 2)};
  const cuuint64_t strides[1] = {cuuint64_t(pitch) * sizeof(T)};
  const cuuint32_t box[2] = {cuuint32_t(bw), cuuint32_t(bh)};
  const cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt =
      sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  return fn(m, dt, 2, start, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Descriptors of the planes of L for boxes of a c.tx x c.ty tile and nph
// colour phases.
template <typename T>
static bool encode_level(const LevelV<T>& L, const TmaCfg& c, int nph, int* err,
                         SweepMaps<T>* m) {
  const bool nine = L.SW != nullptr;
  std::memset(static_cast<void*>(m), 0, sizeof(*m));
  const int align = int(16 / sizeof(T));
  const int ha = nph > align ? nph : align;
  const int bw = c.tx + 2 * ha, bh = c.ty + 2 * kTmaHaloRows;
  auto enc = [&](CUtensorMap* mm, const T* base) {
    return encode_plane<T>(mm, base, L.pitch, L.ny, bw, bh);
  };
  bool ok = enc(&m->x, L.x) && enc(&m->x2, L.x2) && enc(&m->ic, L.iC) && enc(&m->w, L.W) &&
            enc(&m->s, L.S) && enc(&m->b, L.b);
  if (nine) ok = ok && enc(&m->sw, L.SW) && enc(&m->nw, L.NW);
  m->xp = L.x;
  m->x2p = L.x2;
  m->err = err;
  m->nine = nine;
  return ok;
}

// Prescaled finest level: the TMA red-black sweep stages b/C and the four
// couplings divided by C in place of 1/C, W, S, b and takes four fused
// multiply-adds per point instead of four and a product (environment
// BMG_RB_PRESCALE=0 turns it off).  Only levels the TMA sweep handles.
// Tile sides of the prescaled shapes (BMG_TMA_PRE_DISPATCH order).
constexpr int kPreTile[6][2] = {{32, 16}, {64, 16}, {64, 12}, {32, 16}, {32, 8}, {32, 16}};

static int pre_cfg_index() {
  static const int v = [] {
    const int k = env_int("BMG_TMA_PRE_CFG", 0);
    return k >= 0 && k < 6 ? k : 0;
  }();
  return v;
}

bool prescale_enabled(int nx) {
  static const bool on = env_int("BMG_RB_PRESCALE", 1) != 0;
  return on && rb_kernel_choice() == 3 && nx >= 1024;
}

template <typename T>
__global__ void k_prescale_coeffs(LevelV<T> L) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1, j = blockIdx.y + 1;
  if (i > L.nx) return;
  const int o = j * L.pitch + i;
  const T ic = L.iC[o];
  L.PR[PR_W][o] = L.W[o] * ic;
  L.PR[PR_E][o] = L.W[o + 1] * ic;
  L.PR[PR_S][o] = L.S[o] * ic;
  L.PR[PR_N][o] = L.S[o + L.pitch] * ic;
}

template <typename T>
__global__ void k_prescale_b(LevelV<T> L) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1, j = blockIdx.y + 1;
  if (i > L.nx) return;
  const int o = j * L.pitch + i;
  L.PR[PR_B][o] = L.b[o] * L.iC[o];
}

template <typename T>
void launch_prescale_coeffs(const LevelV<T>& L, cudaStream_t s) {
  k_prescale_coeffs<T><<<dim3(cdiv(L.nx, 256), L.ny), 256, 0, s>>>(L);
  count_launch();
}

template <typename T>
void launch_prescale_b(const LevelV<T>& L, cudaStream_t s) {
  k_prescale_b<T><<<dim3(cdiv(L.nx, 256), L.ny), 256, 0, s>>>(L);
  count_launch();
}

template <typename T>
bool make_sweep_maps(const LevelV<T>& L, int* err, SweepMaps<T>* m) {
  const bool nine = L.SW != nullptr;
  if (!nine && (rb_kernel_choice() != 3 || L.nx < 1024)) return false;
  if (nine && L.nx < nine_tma_min_side()) return false;
  if (!encode_level<T>(L, tma_cfg<T>(nine), nine ? 4 : 2, err, m)) return false;
  if (!nine && L.PR[PR_B]) {
    // the prescaled shapes stage boxes of (TX + 4) x (TY + 4)
    const int bw = kPreTile[pre_cfg_index()][0] + 4, bh = kPreTile[pre_cfg_index()][1] + 4;
    auto enc = [&](CUtensorMap* mm, const T* base) {
      return encode_plane<T>(mm, base, L.pitch, L.ny, bw, bh);
    };
    if (!(enc(&m->x, L.x) && enc(&m->x2, L.x2) && enc(&m->pb, L.PR[PR_B]) &&
          enc(&m->pw, L.PR[PR_W]) && enc(&m->pe, L.PR[PR_E]) && enc(&m->ps, L.PR[PR_S]) &&
          enc(&m->pn, L.PR[PR_N])))
      return false;
    m->pre = true;
  }
  return true;
}


// Blocks of a TMA sweep shape resident per SM (at most MINB), measured once;
// first called from prepare_sweep_kernels, after the shared-memory opt-in and
// before any graph capture.
template <typename T, bool NINE, int TX, int TY, int NT, int MINB, int NSTAGE, bool PRE = false,
          bool NRM = false, bool ZERO = false>
static int tma_resident() {
  static const int r = [] {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &n, k_sweep_tma<T, NINE, TX, TY, NT, MINB, NSTAGE, PRE, NRM, ZERO>, NT,
            TmaTile<T, NINE, TX, TY, NSTAGE, PRE>::SMEM) != cudaSuccess ||
        n < 1)
      n = 1;
    cudaGetLastError();
    return n < MINB ? n : MINB;
  }();
  return r;
}

// `order`: 4 bits per colour phase (sub-lattice masks, see rb_order).
// ZERO: a forward sweep of a zero iterate (order must be the forward one).
template <typename T, bool NINE, int TX, int TY, int NT, int MINB, int NSTAGE, bool ZERO = false>
static void launch_tma_shape(const LevelV<T>& L, const SweepMaps<T>& m, const CUtensorMap& mx,
                             unsigned order, T* xout, cudaStream_t s) {
  using G = TmaTile<T, NINE, TX, TY, NSTAGE>;
  const int ntiles = ((L.nx + TX - 1) / TX) * ((L.ny + TY - 1) / TY);
  // persistent blocks: no more than fit on the GPU at once
  const int cap = sm_count() * tma_resident<T, NINE, TX, TY, NT, MINB, NSTAGE, false, false, ZERO>();
  // 5-point levels have no SW/NW planes: their maps are passed unused
  const CUtensorMap& msw = NINE ? m.sw : m.b;
  const CUtensorMap& mnw = NINE ? m.nw : m.b;
  launch_pdl(k_sweep_tma<T, NINE, TX, TY, NT, MINB, NSTAGE, false, false, ZERO>,
             dim3(ntiles < cap ? ntiles : cap), dim3(NT), G::SMEM, s, mx, m.ic, m.w, m.s, m.b, msw,
             mnw, L, xout, order, m.err, (const T*)nullptr, (double*)nullptr);
}

template <typename T, bool NINE, int TX, int TY, int NT, int MINB, int NSTAGE, bool PRE = false,
          bool NRM = false, bool ZERO = false>
static void allow_tma_smem() {
  cudaFuncSetAttribute(k_sweep_tma<T, NINE, TX, TY, NT, MINB, NSTAGE, PRE, NRM, ZERO>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                       int(TmaTile<T, NINE, TX, TY, NSTAGE, PRE>::SMEM));
  tma_resident<T, NINE, TX, TY, NT, MINB, NSTAGE, PRE, NRM, ZERO>();
}

// The prescaled red-black sweep (FP64, 5-point): x, b/C, W/C, S/C, E/C, N/C.
// ZERO: a forward sweep of a zero iterate.
template <int TX, int TY, int NT, int MINB, int NSTAGE, bool ZERO = false>
static void launch_tma_pre(const LevelV<double>& L, const SweepMaps<double>& m,
                           const CUtensorMap& mx, unsigned order, double* xout, cudaStream_t s) {
  using G = TmaTile<double, false, TX, TY, NSTAGE, true>;
  const int ntiles = ((L.nx + TX - 1) / TX) * ((L.ny + TY - 1) / TY);
  const int cap =
      sm_count() * tma_resident<double, false, TX, TY, NT, MINB, NSTAGE, true, false, ZERO>();
  launch_pdl(k_sweep_tma<double, false, TX, TY, NT, MINB, NSTAGE, true, false, ZERO>,
             dim3(ntiles < cap ? ntiles : cap), dim3(NT), G::SMEM, s, mx, m.pb, m.pw, m.ps, m.pe,
             m.pn, m.pn, L, xout, order, m.err, (const double*)nullptr, (double*)nullptr);
}

// The same sweep in the pre-smoothing colour order with the fused residual
// (NRM); returns its grid, the number of partials written.
template <int TX, int TY, int NT, int MINB, int NSTAGE>
static int launch_tma_pre_norm(const LevelV<double>& L, const SweepMaps<double>& m,
                               const CUtensorMap& mx, double* xout, double* partials, int nmax,
                               cudaStream_t s) {
  using G = TmaTile<double, false, TX, TY, NSTAGE, true>;
  const int ntiles = ((L.nx + TX - 1) / TX) * ((L.ny + TY - 1) / TY);
  const int cap = sm_count() * tma_resident<double, false, TX, TY, NT, MINB, NSTAGE, true, true>();
  const int grid = std::min(std::min(ntiles, cap), nmax);
  launch_pdl(k_sweep_tma<double, false, TX, TY, NT, MINB, NSTAGE, true, true>, dim3(grid), dim3(NT),
             G::SMEM, s, mx, m.pb, m.pw, m.ps, m.pe, m.pn, m.pn, L, xout, rb_order(false), m.err,
             (const double*)L.C, partials);
  return grid;
}

#define BMG_TMA_PRE_DISPATCH(K, BODY)      \
  do {                                     \
    switch (K) {                           \
      case 1: BODY(64, 16, 512, 3, 1); break; \
      case 2: BODY(64, 12, 512, 2, 2); break; \
      case 3: BODY(32, 16, 384, 3, 2); break; \
      case 4: BODY(32, 8, 128, 5, 2); break;  \
      case 5: BODY(32, 16, 128, 3, 2); break; \
      default: BODY(32, 16, 256, 3, 2); break; \
    }                                      \
  } while (0)

// Instantiates BODY(T, NINE, TX, TY, NT, MINB, NSTAGE) for entry K of T's
// 5-point or 9-point table (the shapes of kRb64/kRb32, kNine64/kNine32).
#define BMG_TMA_DISPATCH(T, NINE, K, BODY)                             \
  do {                                                                 \
    if constexpr (!(NINE) && sizeof(T) == 8) {                         \
      switch (K) {                                                     \
        case 1: BODY(T, false, 64, 16, 512, 2, 2); break;              \
        case 2: BODY(T, false, 64, 16, 512, 4, 1); break;              \
        default: BODY(T, false, 64, 16, 608, 2, 2); break;             \
      }                                                                \
    } else if constexpr (!(NINE)) {                                    \
      switch (K) {                                                     \
        case 1: BODY(T, false, 64, 16, 256, 3, 2); break;              \
        case 2: BODY(T, false, 128, 16, 256, 4, 1); break;             \
        default: BODY(T, false, 128, 16, 256, 2, 2); break;            \
      }                                                                \
    } else if constexpr (sizeof(T) == 8) {                             \
      switch (K) {                                                     \
        case 1: BODY(T, true, 32, 16, 256, 4, 1); break;               \
        case 2: BODY(T, true, 36, 16, 256, 4, 1); break;               \
        case 3: BODY(T, true, 36, 16, 192, 4, 1); break;               \
        case 4: BODY(T, true, 28, 20, 192, 4, 1); break;               \
        case 5: BODY(T, true, 40, 16, 192, 4, 1); break;               \
        default: BODY(T, true, 40, 16, 256, 4, 1); break;              \
      }                                                                \
    } else {                                                           \
      switch (K) {                                                     \
        case 1: BODY(T, true, 64, 16, 256, 5, 1); break;               \
        case 2: BODY(T, true, 80, 16, 256, 4, 1); break;               \
        case 3: BODY(T, true, 128, 8, 256, 4, 1); break;               \
        case 4: BODY(T, true, 64, 32, 256, 2, 1); break;               \
        case 5: BODY(T, true, 32, 32, 256, 4, 1); break;               \
        default: BODY(T, true, 64, 16, 256, 4, 1); break;              \
      }                                                                \
    }                                                                  \
  } while (0)

template <typename T>
static void launch_sweep_tma(const LevelV<T>& L, const SweepMaps<T>& m, bool reverse,
                             const T* xin, T* xout, cudaStream_t s, bool zero) {
  const CUtensorMap& mx = xin == m.xp ? m.x : m.x2;
  const unsigned order = m.nine ? four_order(reverse) : rb_order(reverse);
  if constexpr (sizeof(T) == 8) {
    if (zero && !reverse && m.pre) {
#define BMG_TMA_PRE_LAUNCH_Z(TX, TY, NT, MB, NS) \
  launch_tma_pre<TX, TY, NT, MB, NS, true>(L, m, mx, order, xout, s)
      BMG_TMA_PRE_DISPATCH(pre_cfg_index(), BMG_TMA_PRE_LAUNCH_Z);
#undef BMG_TMA_PRE_LAUNCH_Z
      return;
    }
  }
  if (zero && !reverse && !m.pre) {
#define BMG_TMA_LAUNCH_Z(TT, NN, TX, TY, NT, MB, NS) \
  launch_tma_shape<TT, NN, TX, TY, NT, MB, NS, true>(L, m, mx, order, xout, s)
    if (m.nine)
      BMG_TMA_DISPATCH(T, true, nine_cfg_index(), BMG_TMA_LAUNCH_Z);
    else
      BMG_TMA_DISPATCH(T, false, rb_cfg_index(), BMG_TMA_LAUNCH_Z);
#undef BMG_TMA_LAUNCH_Z
    return;
  }
  if constexpr (sizeof(T) == 8) {
    if (m.pre) {
#define BMG_TMA_PRE_LAUNCH(TX, TY, NT, MB, NS) launch_tma_pre<TX, TY, NT, MB, NS>(L, m, mx, order, xout, s)
      BMG_TMA_PRE_DISPATCH(pre_cfg_index(), BMG_TMA_PRE_LAUNCH);
#undef BMG_TMA_PRE_LAUNCH
      return;
    }
  }
#define BMG_TMA_LAUNCH(TT, NN, TX, TY, NT, MB, NS) \
  launch_tma_shape<TT, NN, TX, TY, NT, MB, NS>(L, m, mx, order, xout, s)
  if (m.nine)
    BMG_TMA_DISPATCH(T, true, nine_cfg_index(), BMG_TMA_LAUNCH);
  else
    BMG_TMA_DISPATCH(T, false, rb_cfg_index(), BMG_TMA_LAUNCH);
#undef BMG_TMA_LAUNCH
}


// Tiles of the small-level red-black sweep (launch_sweep's `small` shape).
constexpr int kSmallTX = 32, kSmallTY = 16;

int sweep_norm_partials(const LevelV<double>& L, const SweepMaps<double>* maps, int nmax) {
  if (maps && maps->pre) return std::min(nmax, 4 * sm_count());
  if (L.SW != nullptr || L.nx >= 1024) return 0;
  const int tiles = cdiv(L.nx, kSmallTX) * cdiv(L.ny, kSmallTY);
  return tiles <= nmax ? tiles : 0;
}

int launch_sweep_pre_norm(const LevelV<double>& L, const SweepMaps<double>* maps,
                          const double* xin, double* xout, double* partials, int nmax,
                          cudaStream_t s) {
  if (!(maps && maps->pre)) {
    // a level swept by the small tiled kernel: one partial per tile
    const int tiles = sweep_norm_partials(L, maps, nmax);
    if (tiles < 1) return 0;
    launch_pdl(k_sweep_nrm<kSmallTX, kSmallTY, 128>, dim3(cdiv(L.nx, kSmallTX), cdiv(L.ny, kSmallTY)),
               dim3(128), 0, s, L, xin, xout, partials);
    count_launch();
    return tiles;
  }
  if (nmax < 1 || (xin != maps->xp && xin != maps->x2p)) return 0;
  const CUtensorMap& mx = xin == maps->xp ? maps->x : maps->x2;
  int grid = 0;
#define BMG_TMA_PRE_NORM_LAUNCH(TX, TY, NT, MB, NS) \
  grid = launch_tma_pre_norm<TX, TY, NT, MB, NS>(L, *maps, mx, xout, partials, nmax, s)
  BMG_TMA_PRE_DISPATCH(pre_cfg_index(), BMG_TMA_PRE_NORM_LAUNCH);
#undef BMG_TMA_PRE_NORM_LAUNCH
  count_launch();
  return grid;
}

template <typename T>
void launch_sweep(const LevelV<T>& L, bool nine, bool reverse, const T* xin, T* xout,
                  cudaStream_t s, const SweepMaps<T>* maps, bool zero) {
  // Large tiles keep the redundant halo work small (4% red-black, 12% four
  // colours); levels narrower than 1024 use small tiles so that they still
  // spread over all SMs.
  const bool small = L.nx < 1024;
  const bool tma = maps && maps->nine == nine && (xin == maps->xp || xin == maps->x2p);
  if (tma) {
    launch_sweep_tma<T>(L, *maps, reverse, xin, xout, s, zero);
  } else if (nine) {
    if (small) {
      constexpr int TX = 32, TY = 16;
      launch_pdl(k_sweep<T, true, TX, TY, 128>, dim3(cdiv(L.nx, TX), cdiv(L.ny, TY)), dim3(128), 0, s, L, xin, xout,
                 four_order(reverse));
    } else {
      constexpr int TX = 128, TY = 32;
      launch_pdl(k_sweep<T, true, TX, TY, 256>, dim3(cdiv(L.nx, TX), cdiv(L.ny, TY)), dim3(256), 0, s, L, xin, xout,
                 four_order(reverse));
    }
  } else {
    if (small) {
      constexpr int TX = kSmallTX, TY = kSmallTY;
      launch_pdl(k_sweep<T, false, TX, TY, 128>, dim3(cdiv(L.nx, TX), cdiv(L.ny, TY)), dim3(128), 0, s, L, xin, xout,
                 rb_order(reverse));
    } else if (stream_rb_enabled()) {
      constexpr int NT = kStreamNT, R = kStreamR;
      using S = StreamRB<T, NT, R>;
      const size_t smem = sizeof(typename S::Row) * S::NSLOT;
      k_sweep_rb_stream<T, NT, R><<<dim3(cdiv(L.nx, S::OWN), cdiv(L.ny, R)), NT, smem, s>>>(
          L, xin, xout, reverse ? 1 : 0);
    } else if (rb_kernel_choice() == 2) {
      constexpr int TX = 128, TY = 32;
      launch_pdl(k_sweep<T, false, TX, TY, 256, 2>, dim3(cdiv(L.nx, TX), cdiv(L.ny, TY)), dim3(256), 0, s, L, xin, xout,
                 rb_order(reverse));
    } else {
      constexpr int TX = 128, TY = 32;
      launch_pdl(k_sweep<T, false, TX, TY, 256>, dim3(cdiv(L.nx, TX), cdiv(L.ny, TY)), dim3(256), 0, s, L, xin, xout,
                 rb_order(reverse));
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
#define BMG_TMA_ALLOW(TT, NN, TX, TY, NT, MB, NS) allow_tma_smem<TT, NN, TX, TY, NT, MB, NS>()
#define BMG_TMA_ALLOW_Z(TT, NN, TX, TY, NT, MB, NS) \
  allow_tma_smem<TT, NN, TX, TY, NT, MB, NS, false, false, true>()
    BMG_TMA_DISPATCH(double, false, rb_cfg_index(), BMG_TMA_ALLOW);
    BMG_TMA_DISPATCH(float, false, rb_cfg_index(), BMG_TMA_ALLOW);
    BMG_TMA_DISPATCH(double, true, nine_cfg_index(), BMG_TMA_ALLOW);
    BMG_TMA_DISPATCH(float, true, nine_cfg_index(), BMG_TMA_ALLOW);
    BMG_TMA_DISPATCH(double, false, rb_cfg_index(), BMG_TMA_ALLOW_Z);
    BMG_TMA_DISPATCH(float, false, rb_cfg_index(), BMG_TMA_ALLOW_Z);
    BMG_TMA_DISPATCH(double, true, nine_cfg_index(), BMG_TMA_ALLOW_Z);
    BMG_TMA_DISPATCH(float, true, nine_cfg_index(), BMG_TMA_ALLOW_Z);
#undef BMG_TMA_ALLOW_Z
#undef BMG_TMA_ALLOW
#define BMG_TMA_PRE_ALLOW(TX, TY, NT, MB, NS) allow_tma_smem<double, false, TX, TY, NT, MB, NS, true>()
    BMG_TMA_PRE_DISPATCH(pre_cfg_index(), BMG_TMA_PRE_ALLOW);
#undef BMG_TMA_PRE_ALLOW
#define BMG_TMA_PRE_NORM_ALLOW(TX, TY, NT, MB, NS) \
  allow_tma_smem<double, false, TX, TY, NT, MB, NS, true, true>()
    BMG_TMA_PRE_DISPATCH(pre_cfg_index(), BMG_TMA_PRE_NORM_ALLOW);
#undef BMG_TMA_PRE_NORM_ALLOW
#define BMG_TMA_PRE_ZERO_ALLOW(TX, TY, NT, MB, NS) \
  allow_tma_smem<double, false, TX, TY, NT, MB, NS, true, false, true>()
    BMG_TMA_PRE_DISPATCH(pre_cfg_index(), BMG_TMA_PRE_ZERO_ALLOW);
#undef BMG_TMA_PRE_ZERO_ALLOW
    sm_count();
    encode_tiled();
    return true;
  }();
  (void)done;
}

// Failure-detection self-test: one thread waits, with the bounded wait of
// the TMA sweeps, on an mbarrier phase that expects 16 bytes no copy ever
// delivers, and records DEV_TIMEOUT when the wait gives up.
__global__ void k_selftest_wait(int* __restrict__ err) {
  using namespace tma_detail;
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_mbar_init();
  mbar_expect_tx(&bar, 16);
  if (!mbar_wait_bounded(&bar, 0)) atomicOr(err, DEV_TIMEOUT);
}

int selftest_bounded_wait(cudaStream_t s) {
  int* d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return BMG_ENOMEM;
  int h = 0, rc = BMG_ECUDA;
  if (cudaMemsetAsync(d, 0, sizeof(int), s) == cudaSuccess) {
    k_selftest_wait<<<1, 32, 0, s>>>(d);
    count_launch();
    if (cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
        cudaStreamSynchronize(s) == cudaSuccess)
      rc = (h & DEV_TIMEOUT) ? BMG_ETIMEOUT : BMG_OK;
  }
  cudaFree(d);
  return rc;
}

template void launch_sweep<double>(const LevelV<double>&, bool, bool, const double*, double*,
                                   cudaStream_t, const SweepMaps<double>*, bool);
template void launch_sweep<float>(const LevelV<float>&, bool, bool, const float*, float*,
                                  cudaStream_t, const SweepMaps<float>*, bool);
template bool make_sweep_maps<double>(const LevelV<double>&, int*, SweepMaps<double>*);
template void launch_prescale_coeffs<double>(const LevelV<double>&, cudaStream_t);
template void launch_prescale_b<double>(const LevelV<double>&, cudaStream_t);
template bool make_sweep_maps<float>(const LevelV<float>&, int*, SweepMaps<float>*);

}  // namespace bmg
