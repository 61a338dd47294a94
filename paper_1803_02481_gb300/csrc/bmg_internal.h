// Internal declarations of the GB300 BoxMG library: device data layout, the
// per-point stencil arithmetic shared by every kernel, and the host-side
// launch interface.
//
// Data layout in HBM
// ------------------
// Every grid quantity of a level lives in a "plane": (ny + 2) rows of `pitch`
// elements, with a one-cell ghost ring that holds zeros (the Dirichlet
// condition of Eq. (diffusion_bc) and the zero coarse values outside the
// domain).  Element (i, j), 0 <= i <= nx + 1, 0 <= j <= ny + 1, 1-based in
// the interior, is at base[j * pitch + i].  `base` is offset inside the
// allocation so that every interior row starts (i = 1) on a 128-byte
// boundary; pitch is a multiple of 128 bytes.
//
// Operator of a level (symmetric; the five stored planes give all nine
// entries, as in BoxMG):
//   C(i,j)  = A[(i,j),(i,j)]              iC = 1 / C (so no divide in sweeps)
//   W(i,j)  = -A[(i,j),(i-1,j)]           E(i,j)  = W(i+1,j)
//   S(i,j)  = -A[(i,j),(i,j-1)]           N(i,j)  = S(i,j+1)
//   SW(i,j) = -A[(i,j),(i-1,j-1)]         NE(i,j) = SW(i+1,j+1)
//   NW(i,j) = -A[(i,j),(i-1,j+1)]         SE(i,j) = NW(i+1,j-1)
// The assembled finest level is 5-point (no SW/NW planes).
//
// Interpolation P_l (level l-1 -> l) is stored as eight planes on the coarse
// grid of level l-1 (index (I, J), 0..nc), one weight per (fine point,
// coarse neighbour) pair, 1-based fine indices:
//   XW, XE           x-edge point (2I+1, 2J)   -> coarse (I,J), (I+1,J)
//   YS, YN           y-edge point (2I, 2J+1)   -> coarse (I,J), (I,J+1)
//   CSW, CSE, CNW, CNE  centre (2I+1, 2J+1)    -> (I,J),(I+1,J),(I,J+1),(I+1,J+1)
// Coarse point (I, J) is fine point (2I, 2J) with weight 1.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/boxmg.h"

namespace bmg {

enum PIdx { XW = 0, XE, YS, YN, CSW, CSE, CNW, CNE, NPW };

// Grid geometry of one plane.
struct Geom {
  int nx, ny, pitch;   // pitch in elements
  size_t elems;        // elements reserved per plane (incl. alignment slack)
};

template <typename T>
inline Geom make_geom(int nx, int ny) {
  const int per128 = int(128 / sizeof(T));
  Geom g;
  g.nx = nx;
  g.ny = ny;
  // pitch >= nx + 1 + 128 / sizeof(T): counted from the 128-byte aligned
  // start of a row's storage (i = 1 - base_shift), the row's pitch elements
  // reach the east ghost column i = nx + 1 (the extent a plane's TMA
  // descriptor gives a row)
  g.pitch = ((nx + 1 + per128 + per128 - 1) / per128) * per128;
  g.elems = size_t(ny + 2) * g.pitch + per128;
  return g;
}

// Offset of the plane base inside its allocation: interior i = 1 lands on a
// 128-byte boundary.
template <typename T>
constexpr int base_shift() { return int(128 / sizeof(T)) - 1; }

// Line smoothing (bmg_line.cuh): points per block of a line (kLineM - 1
// interior points and one separator), and the planes of precomputed factors
// per line direction: block LU forward multiplier, reciprocal pivot and
// back-substitution coefficient (at separators: those of the Schur system),
// and the two spikes.
constexpr int kLineM = 16;
enum { LF_MU = 0, LF_IU, LF_CA, LF_V, LF_W, NLF };
// Per-separator arrays of a line direction, compact: separator t (0-based)
// of line q at q * spp + t.  Setup: the Schur system's forward multiplier,
// reciprocal pivot, back-substitution coefficient, the coupling a_{s+1} to
// the point after the separator, and the products of the multipliers from
// the start of t's group to t (P) and of the coefficients from t to the end
// of its group (Q; groups of sgl separators, see bmg_line.cuh).  Per sweep:
// d_s + a_s g_{s-1} (then the substitutions' partial values) and g_{s+1},
// written by the block solves.
enum { SP_MU = 0, SP_IU, SP_CA, SP_AN, SP_P, SP_Q, SP_RL, SP_GF, NSP };

// Device view of one level.  Pointers are plane bases (element (0,0) is the
// lower-left ghost).  SW/NW are null on a 5-point level.  P holds the
// interpolation INTO this level from the next coarser one (null on level 0).
// LF[d] holds the line factors of direction d (0: x-lines, 1: y-lines), null
// unless the smoother uses that direction.
template <typename T>
struct LevelV {
  int nx, ny, pitch;
  T *C, *iC, *W, *S, *SW, *NW;
  T *x, *b, *r;
  T *x2;               // second iterate buffer (sweeps write out of place)
  T *PR[5];            // prescaled 5-point finest level (else null): b/C, W/C, E/C,
                       // S/C, N/C, E and N the couplings to i + 1 and j + 1
  T *LF[2][NLF];       // x-lines: plane layout; y-lines: colour-compacted
  T *SP[2][NSP];
  int spp[2];          // separators per line, rounded up (0: no separators)
  int sgl[2];          // separators per group of the Schur substitutions
  T *ys;               // y-line scratch, colour-compacted
  int ycp, yhalf;      // colour-compacted layout: column c + 2 j + 1 of
                       // colour c at c * yhalf + row * ycp + j
  T *P[NPW];
  int cpitch;          // pitch of the coarse grid the P planes live on
};

// Programmatic dependent launch.  A kernel launched with launch_pdl may be
// scheduled while the kernel before it in the stream (or graph) is still
// finishing; its first statement is griddep_wait(), which returns once that
// kernel has completed and its memory operations are visible, so nothing it
// reads or writes can race with it -- only the launch itself overlaps.  No
// kernel triggers its dependents early (they launch as its blocks exit):
// triggering right after the wait let waiting blocks of the next kernel hold
// SM resources and cost the 4095^2 solve 10 % (measured), while the overlap
// at exit gains 3 % on the launch-bound 255^2 cycle.  (griddepcontrol.wait is
// a no-op in a kernel launched without the attribute.)  Environment
// BMG_PDL=0 launches without it.
__device__ __forceinline__ void griddep_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
bool pdl_enabled();
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// ---------------------------------------------------------------------------
// Per-point arithmetic.  Every kernel (full-grid or persistent) uses these,
// so a level gives bit-identical results whichever kernel processes it.
// ---------------------------------------------------------------------------

// Gauss-Seidel update of one point: x = (b + sum_X a_X x_X) * (1/C), the
// neighbour terms accumulated in the order W, E, S, N, SW, SE, NW, NE.
// The coefficients of the point are loaded first (GsCoef), then applied to
// the iterate through an accessor `xa(dx, dy)`; the same arithmetic serves
// iterates in global memory and in shared-memory tiles, so every kernel
// produces the same bits.
template <typename T, bool NINE>
struct GsCoef {
  T b, ic, w, e, s, n, sw, se, nw, ne;
};

template <typename T, bool NINE>
__device__ __forceinline__ GsCoef<T, NINE> gs_load(const LevelV<T>& L, int o, T bval) {
  const int p = L.pitch;
  GsCoef<T, NINE> c;
  c.b = bval;
  c.ic = __ldg(L.iC + o);
  c.w = __ldg(L.W + o);
  c.e = __ldg(L.W + o + 1);
  c.s = __ldg(L.S + o);
  c.n = __ldg(L.S + o + p);
  if (NINE) {
    c.sw = __ldg(L.SW + o);
    c.se = __ldg(L.NW + o + 1 - p);
    c.nw = __ldg(L.NW + o);
    c.ne = __ldg(L.SW + o + 1 + p);
  }
  return c;
}

// gs_apply with only the neighbour terms whose bit is set in `mask` (bits in
// the order W, E, S, N, SW, SE, NW, NE): the caller knows the others' x to
// be zero, and fma(a, 0, acc) = acc, so the value is gs_apply's (a zero
// result may differ in sign).  `mask` is a compile-time constant at every
// call after unrolling, so the skipped terms cost nothing.
template <typename T, bool NINE, class XA>
__device__ __forceinline__ T gs_apply_masked(const GsCoef<T, NINE>& c, XA xa, unsigned mask) {
  T acc = c.b;
  if (mask & 0x01u) acc = fma(c.w, xa(-1, 0), acc);
  if (mask & 0x02u) acc = fma(c.e, xa(1, 0), acc);
  if (mask & 0x04u) acc = fma(c.s, xa(0, -1), acc);
  if (mask & 0x08u) acc = fma(c.n, xa(0, 1), acc);
  if (NINE) {
    if (mask & 0x10u) acc = fma(c.sw, xa(-1, -1), acc);
    if (mask & 0x20u) acc = fma(c.se, xa(1, -1), acc);
    if (mask & 0x40u) acc = fma(c.nw, xa(-1, 1), acc);
    if (mask & 0x80u) acc = fma(c.ne, xa(1, 1), acc);
  }
  return acc * c.ic;
}

template <typename T, bool NINE, class XA>
__device__ __forceinline__ T gs_apply(const GsCoef<T, NINE>& c, XA xa) {
  T acc = c.b;
  acc = fma(c.w, xa(-1, 0), acc);
  acc = fma(c.e, xa(1, 0), acc);
  acc = fma(c.s, xa(0, -1), acc);
  acc = fma(c.n, xa(0, 1), acc);
  if (NINE) {
    acc = fma(c.sw, xa(-1, -1), acc);
    acc = fma(c.se, xa(1, -1), acc);
    acc = fma(c.nw, xa(-1, 1), acc);
    acc = fma(c.ne, xa(1, 1), acc);
  }
  return acc * c.ic;
}

// Gauss-Seidel update of a point of a prescaled level: the same neighbour
// order with every coefficient already divided by C, so no final product:
// x = b/C + (W/C) x_W + (E/C) x_E + (S/C) x_S + (N/C) x_N.
enum { PR_B = 0, PR_W, PR_E, PR_S, PR_N };

template <typename T, class XA>
__device__ __forceinline__ T gs_pre_apply(T pb, T pw, T pe, T ps, T pn, XA xa) {
  T acc = pb;
  acc = fma(pw, xa(-1, 0), acc);
  acc = fma(pe, xa(1, 0), acc);
  acc = fma(ps, xa(0, -1), acc);
  acc = fma(pn, xa(0, 1), acc);
  return acc;
}

template <typename T>
__device__ __forceinline__ T gs_pre_value(const LevelV<T>& L, const T* __restrict__ x, int o) {
  const int p = L.pitch;
  return gs_pre_apply<T>(L.PR[PR_B][o], L.PR[PR_W][o], L.PR[PR_E][o], L.PR[PR_S][o],
                         L.PR[PR_N][o], [&](int dx, int dy) { return x[o + dx + dy * p]; });
}

template <typename T, bool NINE, class XA>
__device__ __forceinline__ T gs_update(const LevelV<T>& L, XA xa, T bval, int o) {
  return gs_apply<T, NINE>(gs_load<T, NINE>(L, o, bval), xa);
}

template <typename T, bool NINE>
__device__ __forceinline__ T gs_value(const LevelV<T>& L, const T* __restrict__ x,
                                      T bval, int o) {
  const int p = L.pitch;
  return gs_update<T, NINE>(L, [&](int dx, int dy) { return x[o + dx + dy * p]; }, bval, o);
}

// Residual of one point: r = b - (C x - sum_X a_X x_X), accumulated as
// b - C x first, then + a_X x_X (one FMA per stencil entry).
template <typename T, bool NINE>
__device__ __forceinline__ T resid_value(const LevelV<T>& L, const T* __restrict__ x,
                                         T bval, int o) {
  const int p = L.pitch;
  T r = fma(-L.C[o], x[o], bval);
  r = fma(L.W[o], x[o - 1], r);
  r = fma(L.W[o + 1], x[o + 1], r);
  r = fma(L.S[o], x[o - p], r);
  r = fma(L.S[o + p], x[o + p], r);
  if (NINE) {
    r = fma(L.SW[o], x[o - p - 1], r);
    r = fma(L.NW[o + 1 - p], x[o + 1 - p], r);
    r = fma(L.NW[o], x[o + p - 1], r);
    r = fma(L.SW[o + 1 + p], x[o + 1 + p], r);
  }
  return r;
}

// Weight of fine point (2I + rx, 2J + ry) towards coarse point (I, J),
// rx, ry in {-1, 0, 1}; c = J * cpitch + I.
template <typename T>
__device__ __forceinline__ T pweight(T* const* P, int cp, int rx, int ry, int c) {
  if (rx == 0 && ry == 0) return T(1);
  if (ry == 0) return rx > 0 ? P[XW][c] : P[XE][c - 1];
  if (rx == 0) return ry > 0 ? P[YS][c] : P[YN][c - cp];
  if (rx > 0 && ry > 0) return P[CSW][c];
  if (rx < 0 && ry > 0) return P[CSE][c - 1];
  if (rx > 0 && ry < 0) return P[CNW][c - cp];
  return P[CNE][c - cp - 1];
}

// Restriction at coarse point (I, J): b_c = sum over the 3x3 fine block of
// P(p, I) r(p) (R = P^T, Algorithm 1).  f = fine offset of (2I, 2J).
template <typename T>
__device__ __forceinline__ T restrict_value(T* const* P, int cp, const T* __restrict__ r,
                                            int fp, int c, int f) {
  T acc = r[f];
  acc = fma(P[XE][c - 1], r[f - 1], acc);
  acc = fma(P[XW][c], r[f + 1], acc);
  acc = fma(P[YN][c - cp], r[f - fp], acc);
  acc = fma(P[YS][c], r[f + fp], acc);
  acc = fma(P[CNE][c - cp - 1], r[f - fp - 1], acc);
  acc = fma(P[CNW][c - cp], r[f - fp + 1], acc);
  acc = fma(P[CSE][c - 1], r[f + fp - 1], acc);
  acc = fma(P[CSW][c], r[f + fp + 1], acc);
  return acc;
}

// Interpolated correction (P x_c)(i, j) at fine point (i, j), 1-based.
template <typename T>
__device__ __forceinline__ T interp_value(T* const* P, int cp, const T* __restrict__ xc,
                                          int i, int j) {
  const int I = i >> 1, J = j >> 1;
  const int c = J * cp + I;
  if (!(i & 1)) {
    if (!(j & 1)) return xc[c];
    return fma(P[YS][c], xc[c], P[YN][c] * xc[c + cp]);
  }
  if (!(j & 1)) return fma(P[XW][c], xc[c], P[XE][c] * xc[c + 1]);
  T v = P[CSW][c] * xc[c];
  v = fma(P[CSE][c], xc[c + 1], v);
  v = fma(P[CNW][c], xc[c + cp], v);
  v = fma(P[CNE][c], xc[c + cp + 1], v);
  return v;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

// Error word written by device code (0 = fine).
// Bits 8.. of the error word name the levels whose interpolation met a
// non-positive denominator (bit 8 + l for P_l).
enum DevErr { DEV_OK = 0, DEV_BADK = 1, DEV_NOTSPD = 2, DEV_BADDEN = 4, DEV_NAN = 8,
              DEV_TIMEOUT = 16, DEV_BADLINE = 32 };

// Thread-local detail message of the last failure (bmg_last_error).
void set_last_error(const char* fmt, ...);

struct Scalars {            // device-resident solve state
  double bnorm2;            // ||b||^2
  double rnorm2;            // ||r||^2 of the latest residual
  double scale2;            // FP32_REFINE: ||r||^2 of the previous residual,
                            // the square of the scale the latest residual was
                            // divided by before the cast to FP32
  double rel;               // sqrt(rnorm2 / bnorm2)
  double tol;               // stop test
  double scale;             // sqrt(scale2), set with scale2 (one thread)
  double inv;               // 1 / sqrt(rnorm2) (0 when rnorm2 == 0), set with rnorm2
  double rnorm;             // sqrt(rnorm2), set with rnorm2
  double rz;                // BMG_SOLVER_PCG: r.z of the current iteration
  double alpha, beta;       // BMG_SOLVER_PCG: step and direction coefficients
  int cycles;               // cycles / refinement steps run
  int max_cycles;
  int go;                   // 1 while the loop should continue
  int err;                  // DevErr bits
};

// 2-D TMA descriptors of the planes the TMA-staged sweep reads, for one
// level (built at setup; see make_sweep_maps).
template <typename T>
struct SweepMaps {
  CUtensorMap x, x2, ic, w, s, b, sw, nw;   // sw, nw: 9-point levels only
  CUtensorMap pb, pw, pe, ps, pn;           // prescaled planes (pre)
  bool pre;         // prescaled 5-point level: the sweep stages x and PR
  const T* xp;      // plane the map `x` describes
  const T* x2p;     // plane the map `x2` describes
  int* err;         // device error word (DEV_TIMEOUT)
  bool nine;        // 9-point level (four colours, seven staged planes)
};

struct Timing;

struct Hierarchy {
  int nx = 0, ny = 0, L = 0;
  bmg_options opt{};
  int threshold = 1;                 // levels l < threshold: persistent kernel
  int coarse_ctas = 1;               // its thread blocks (1: one block; more: a cluster)
  std::vector<LevelV<double>> d;     // FP64 levels (all for FP64; finest only
                                     // for FP32_REFINE)
  std::vector<LevelV<float>> f;      // FP32 levels (FP32_REFINE)
  std::vector<Geom> geo64, geo32;
  double* kcopy = nullptr;           // dense (ny, nx) copy of k
  double* chol = nullptr;            // N0 x N0 lower factor (row-major)
  double* chol_idiag = nullptr;      // 1 / L[i][i]
  int n0 = 0;
  double* partials = nullptr;        // reduction scratch
  double* hist = nullptr;            // relative residual per cycle (BMG_MAX_HISTORY)
  int npartials = 0;
  Scalars* sc = nullptr;             // device scalars
  Scalars* sc_host = nullptr;        // pinned mirror
  LevelV<double>* dlev64 = nullptr;  // device copies of the level views (for
  LevelV<float>* dlev32 = nullptr;   // the persistent coarse kernel)
  double predicted_us[16] = {};      // cost model: V-cycle time per threshold
  // The solve loop as one CUDA graph: [first residual + stop test] then
  // WHILE(go) { V-cycle; (refinement update;) residual + stop test }.
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaGraphConditionalHandle cond = 0;
  int graph_state = 0;               // 0 not built, 1 ready, -1 unavailable
  bool fused_norm_allowed = true;    // stop test inside the next fine sweep
                                     // where it applies (BMG_FUSED_NORM at setup)
  void* arena = nullptr;
  size_t arena_bytes = 0;
  double setup_ms = 0.0;
  // TMA descriptors per level of d / f (null where a level is swept by the
  // tiled kernel)
  std::vector<SweepMaps<double>*> maps64;
  std::vector<SweepMaps<float>*> maps32;
  // BMG_SOLVER_PCG planes on the finest level (FP64): iterate, right-hand
  // side, search direction and A p.  The fine level's b plane holds the
  // residual r (the V-cycle's right-hand side) and its x plane z.
  double *pcg_x = nullptr, *pcg_b = nullptr, *pcg_p = nullptr, *pcg_q = nullptr;

};

// Observability: launch counter and optional event bracketing of one kernel
// class (bmg_profile.cu).
void count_launch(int n = 1);
bool prof_active();
// Host-side NVTX range named after a V-cycle operation, with the level as
// its payload, for profilers that record NVTX (ncu --nvtx, Nsight Systems).
// On the stream-launched path it brackets the operation's launches; while a
// graph is being captured it brackets the recording.
struct NvtxRange {
  NvtxRange(const char* op, int level);
  ~NvtxRange();
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

void prof_begin(int which, cudaStream_t s);
void prof_end(int which, cudaStream_t s);

// Hierarchy lifetime (bmg_api.cu).
int setup_impl(const double* k, int nx, int ny, const bmg_options* opt, cudaStream_t s,
               Hierarchy** out);
void free_hierarchy(Hierarchy* h);

// Kernel launch wrappers (defined in the .cu files).
template <typename T>
int launch_assemble(const double* k, int nx, int ny, LevelV<T> L, double* kcopy,
                    int* derr, bool log_k, double r, double aspect, const double* bc_beta,
                    cudaStream_t s);
template <typename T>
int launch_interp_weights(const LevelV<T>& fine, bool nine, int* derr, int level, cudaStream_t s);
template <typename T>
int launch_rap(const LevelV<T>& fine, bool nine, LevelV<T> coarse, cudaStream_t s);
int launch_coarse_factor(Hierarchy* h, const LevelV<double>* l0d, const LevelV<float>* l0f,
                         cudaStream_t s);
int launch_downcast_fine(const LevelV<double>& d, LevelV<float> f, cudaStream_t s);

template <typename T>
void launch_pack(const double* src, T* dst, int nx, int ny, int pitch, cudaStream_t s);
template <typename T>
void launch_unpack(const T* src, double* dst, int nx, int ny, int pitch, cudaStream_t s);

template <typename T>
void launch_residual(const LevelV<T>& L, bool nine, const T* x, const T* b, T* r,
                     cudaStream_t s);
template <typename T>
void launch_restrict(const LevelV<T>& fine, const T* r, LevelV<T> coarse, bool zero_x,
                     cudaStream_t s);
// Residual and restriction of `fine` into `coarse` in one pass (coarse x set
// to zero); rr_fused says whether the V-cycle uses it for a level.
template <typename T>
void launch_resid_restrict(const LevelV<T>& fine, bool nine, LevelV<T> coarse, cudaStream_t s);
bool rr_fused(bool nine, bool fp64);
// Threads of the one-block persistent coarse kernel.
int coarse_block_threads();
template <typename T>
void launch_interp(const LevelV<T>& fine, const T* xc, bool add_r_over_c, cudaStream_t s,
                   T* out = nullptr);
void prepare_sweep_kernels();

// Threads per block of the cluster coarse kernel, and the largest cluster
// (blocks, a power of two <= 16) the device can run it with; 1 when thread-
// block clusters are unavailable.
constexpr int kCoarseClusterThreads = 512;
int max_cluster_ctas(bool fp32);
// Runs the TMA sweeps' bounded mbarrier wait on a phase nothing completes
// (bmg_selftest_bounded_wait).
int selftest_bounded_wait(cudaStream_t s);
// TMA descriptors of a level for the TMA-staged sweep; false (and no
// descriptors) when the level is swept by the tiled kernel instead.
template <typename T>
bool make_sweep_maps(const LevelV<T>& L, int* err, SweepMaps<T>* m);

// One multicolour Gauss-Seidel sweep of a level as a single kernel: reads
// the iterate from xin and writes the swept iterate to xout (xin != xout).
// `maps` (the level's descriptors, may be null) selects the TMA-staged
// kernel.  `zero`: xin is known to be zero (a forward sweep may then use the
// zero-start form: the same values, less work).
template <typename T>
void launch_sweep(const LevelV<T>& L, bool nine, bool reverse, const T* xin, T* xout,
                  cudaStream_t s, const SweepMaps<T>* maps = nullptr, bool zero = false);
// The prescaled level's red-black sweep in the pre-smoothing colour order
// that also sums the stop test's squared residual of its input iterate into
// partials[0 .. grid) (grid <= nmax, returned).  Valid only when the sweep
// before it on this level was a post-smoothing sweep (reverse colour order)
// and nothing changed the iterate since; returns 0 and launches nothing when
// the level cannot take it (see sweep_norm_partials).
int launch_sweep_pre_norm(const LevelV<double>& L, const SweepMaps<double>* maps,
                          const double* xin, double* xout, double* partials, int nmax,
                          cudaStream_t s);
// Partials that sweep writes on this level (at most nmax), 0 where it cannot
// run: prescaled TMA levels, and 5-point levels narrower than 1024 (swept by
// the small tiled kernel) with at most nmax tiles.
int sweep_norm_partials(const LevelV<double>& L, const SweepMaps<double>* maps, int nmax);
template <typename T>
void launch_coarse_cycle(Hierarchy* h, const LevelV<T>* levels, int threshold,
                         cudaStream_t s);

// Prescaled finest level (bmg_sweep.cu): whether the finest FP64 level of a
// hierarchy is prescaled; the coefficient planes W/C, E/C, S/C, N/C (setup)
// and b/C (whenever the level's b changes).
bool prescale_enabled(int nx);
template <typename T>
void launch_prescale_coeffs(const LevelV<T>& L, cudaStream_t s);
template <typename T>
void launch_prescale_b(const LevelV<T>& L, cudaStream_t s);

// Line smoothing (bmg_line.cu).  factor: the block LU factors, spikes and
// Schur factors of every line of the directions `smoother` uses (setup; a
// non-positive pivot sets DEV_BADLINE).  sweep: one line Gauss-Seidel sweep
// (every step of line_steps), reading the iterate from xin and leaving the
// swept iterate in xout (xin == xout allowed); uses L.r as scratch.
template <typename T>
int launch_line_factor(const LevelV<T>& L, int smoother, int* derr, cudaStream_t s);
template <typename T>
void launch_line_sweep(const LevelV<T>& L, bool nine, int smoother, bool reverse, const T* xin,
                       T* xout, cudaStream_t s);

// ||b - A x||^2 (or ||b||^2 when x == nullptr) of the finest FP64 level into
// sc->rnorm2 / sc->bnorm2; then updates rel/go.  `what`: 0 = b norm, 1 =
// residual norm + convergence flag.
void launch_fine_norm(Hierarchy* h, const double* x, const double* b, int what,
                      double tol, cudaStream_t s, bool in_graph = false);
// FP32_REFINE: r = b - A x in FP64 on the finest level, cast r/scale to FP32
// into the FP32 fine RHS; zero the FP32 fine x.
void launch_refine_residual(Hierarchy* h, double tol, cudaStream_t s, bool in_graph = false);
void launch_refine_update(Hierarchy* h, cudaStream_t s);
// Sums h->partials (the first n, else npartials, squared-residual partials) into the stop test:
// rnorm2, rel, history, go, cycles; in a graph it also sets the WHILE
// condition.
void launch_norm_final(Hierarchy* h, cudaStream_t s, bool in_graph, int n = 0);

// Preconditioned conjugate gradients (bmg_pcg.cu).  init: r = b - A x, z = 0,
// ||r||^2 and the stop test; ap: q = A p, p.q, alpha; xr: x += alpha p,
// r -= alpha q, z = 0, ||r||^2 and the stop test; rz: r.z and beta (first:
// beta = 0); p: p = z + beta p.
void launch_pcg_init(Hierarchy* h, cudaStream_t s, bool in_graph);
void launch_pcg_ap(Hierarchy* h, cudaStream_t s);
void launch_pcg_xr(Hierarchy* h, cudaStream_t s, bool in_graph);
void launch_pcg_rz(Hierarchy* h, bool first, cudaStream_t s);
void launch_pcg_p(Hierarchy* h, cudaStream_t s);
// z = M^{-1} r for PCG: one V-cycle on the residual in the finest level's b
// plane (FP64 levels; BMG_FP32_REFINE: r / ||r|| cast to the FP32 finest
// level, the FP32 cycle, z = ||r|| e cast back).
void launch_pcg_precond(Hierarchy* h, cudaStream_t s);

// One V-cycle of the FP64 (d) or FP32 (f) hierarchy (bmg_api.cu);
// skip_first: the top level's first pre-smoothing sweep was already issued;
// top_zero: the top level's iterate is zero on entry (as every coarser
// level's is after its restriction).
template <typename T>
void enqueue_vcycle(Hierarchy* h, std::vector<LevelV<T>>& lv, const LevelV<T>* dlev, int thr,
                    cudaStream_t s, int top = -1, bool skip_first = false, bool top_zero = false);

void launch_assemble_backward(const double* k, const double* u, const double* lam,
                              double* g, int nx, int ny, cudaStream_t s);

}  // namespace bmg
