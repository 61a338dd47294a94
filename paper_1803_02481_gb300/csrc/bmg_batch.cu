// Batched solves: many independent diffusion problems of uneven size, each
// solved with FP32 V-cycles (Algorithm 1) inside FP64 iterative refinement,
// all advanced together.
//
// Organisation.  Every problem is set up as a hierarchy of its own.  The
// solve groups, for every grid side n, the levels of that side across all
// problems (5-point finest levels and 9-point coarse levels separately) and
// runs each operation of the V-cycle as ONE launch over all of them: the
// problem index is blockIdx.z, and a problem that has converged leaves at
// once.  Levels at or below `coarse_side` run in the persistent coarse
// kernel, one thread block per problem.  Per-problem FP64 residual norms and
// stop tests decide which problems stay active; the whole refinement loop is
// one CUDA graph whose WHILE node repeats while any problem is active.  Tile
// shapes of the batched sweeps are chosen per level side by timing the
// candidates on the batch (autotuner, cached per process and optionally in
// the file named by BMG_TUNE_CACHE).
#include "bmg_coarse.cuh"
#include "bmg_sweep_tile.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

namespace bmg {

namespace {

constexpr int kPB = 64;           // FP64 partial sums per problem
constexpr int kNT = 256;          // threads of the norm kernels
constexpr int kCoarseSide = 31;   // levels with side <= this: persistent kernel

inline int cdiv(long a, long b) { return int((a + b - 1) / b); }

__device__ __forceinline__ double bsum(double v) {
  __shared__ double red[kNT / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = v;
  __syncthreads();
  v = lane < kNT / 32 ? red[lane] : 0.0;
  if (w == 0) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  }
  return v;
}

// ---------------------------------------------------------------------------
// Batched V-cycle kernels (FP32).  z = blockIdx.z indexes the class members.
// ---------------------------------------------------------------------------

template <bool NINE, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT) k_bsweep(const LevelV<float>* __restrict__ views,
                                               const int* __restrict__ pids,
                                               const Scalars* __restrict__ sc, unsigned order) {
  const int z = blockIdx.z;
  if (!sc[pids[z]].go) return;
  const LevelV<float> L = views[z];
  sweep_tile<float, NINE, TX, TY, NT>(L, L.x, L.x2, order, blockIdx.x, blockIdx.y);
}

template <bool NINE>
__global__ void k_bresid(const LevelV<float>* __restrict__ views, const int* __restrict__ pids,
                         const Scalars* __restrict__ sc) {
  const int z = blockIdx.z;
  if (!sc[pids[z]].go) return;
  const LevelV<float> L = views[z];
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int j = blockIdx.y + 1;
  if (i > L.nx) return;
  const int o = j * L.pitch + i;
  L.r[o] = resid_value<float, NINE>(L, L.x, L.b[o], o);
}

__global__ void k_brestrict(const LevelV<float>* __restrict__ fine,
                            const LevelV<float>* __restrict__ coarse, const int* __restrict__ pids,
                            const Scalars* __restrict__ sc) {
  const int z = blockIdx.z;
  if (!sc[pids[z]].go) return;
  const LevelV<float> F = fine[z];
  const LevelV<float> Cc = coarse[z];
  const int I = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int J = blockIdx.y + 1;
  if (I > Cc.nx) return;
  const int c = J * Cc.pitch + I;
  Cc.b[c] = restrict_value<float>(F.P, Cc.pitch, F.r, F.pitch, c, 2 * J * F.pitch + 2 * I);
  Cc.x[c] = 0.0f;
}

__global__ void k_binterp(const LevelV<float>* __restrict__ fine,
                          const LevelV<float>* __restrict__ coarse, const int* __restrict__ pids,
                          const Scalars* __restrict__ sc, int out_of_place) {
  const int z = blockIdx.z;
  if (!sc[pids[z]].go) return;
  const LevelV<float> F = fine[z];
  const float* xc = coarse[z].x;
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int j = blockIdx.y + 1;
  if (i > F.nx) return;
  const int o = j * F.pitch + i;
  const float v = F.x[o] + interp_value<float>(F.P, F.cpitch, xc, i, j);
  (out_of_place ? F.x2 : F.x)[o] = v;
}

struct BCoarse {                  // per problem, for the persistent kernel
  const LevelV<float>* lev;
  const double* chol;
  const double* idiag;
  int thr, n0, top_nine;
};

__global__ void __launch_bounds__(1024) k_bcoarse(const BCoarse* __restrict__ pc,
                                                  const Scalars* __restrict__ sc, int nu1,
                                                  int nu2) {
  const int p = blockIdx.x;
  if (!sc[p].go) return;
  const BCoarse q = pc[p];
  CoarseArgs<float> a;
  a.lev = q.lev;
  a.thr = q.thr;
  a.nu1 = nu1;
  a.nu2 = nu2;
  a.add_rc = 0;
  a.smoother = BMG_SMOOTH_POINT;
  a.top_nine = q.top_nine;
  a.chol = q.chol;
  a.idiag = q.idiag;
  a.n0 = q.n0;
  coarse_cycle_body<float>(a);
}

// ---------------------------------------------------------------------------
// Batched refinement kernels (FP64 on each problem's finest level).
// ---------------------------------------------------------------------------

// what == 0: partial sums of b^2.  what == 1 (active problems only): r = b -
// A x in FP64, partial sums of r^2, FP32 right-hand side r / ||r_prev||, FP32
// iterate reset to zero.  One problem per blockIdx.y, kPB blocks each.
__global__ void __launch_bounds__(kNT) k_brefine_resid(const LevelV<double>* __restrict__ f64,
                                                       const LevelV<float>* __restrict__ f32,
                                                       const int* __restrict__ pids,
                                                       const Scalars* __restrict__ sc,
                                                       double* __restrict__ partials, int what) {
  const int z = blockIdx.y;
  const int p = pids[z];
  if (what == 1 && !sc[p].go) return;
  const LevelV<double> L = f64[z];
  const LevelV<float> F = f32[z];
  const double inv = what ? sc[p].inv : 0.0;
  // FP32 scaling of the right-hand side, as in the single-problem kernel
  const bool fp32_scale = inv > 1e-28 && inv < 1e28;
  const float inv32 = float(inv);
  double acc = 0.0;
  for (int j = blockIdx.x + 1; j <= L.ny; j += gridDim.x) {
    for (int i = threadIdx.x + 1; i <= L.nx; i += blockDim.x) {
      const int o = j * L.pitch + i;
      if (what == 0) {
        const double bv = L.b[o];
        acc = fma(bv, bv, acc);
      } else {
        const double r = resid_value<double, false>(L, L.x, L.b[o], o);
        acc = fma(r, r, acc);
        const int of = j * F.pitch + i;
        F.b[of] = fp32_scale ? float(r) * inv32 : float(r * inv);
        F.x[of] = 0.0f;
      }
    }
  }
  acc = bsum(acc);
  if (threadIdx.x == 0) partials[size_t(p) * kPB + blockIdx.x] = acc;
}

// One block per problem: sums its partials and applies the stop test.
__global__ void __launch_bounds__(kNT) k_bnorm_final(const double* __restrict__ partials,
                                                     Scalars* __restrict__ sc, int what) {
  const int p = blockIdx.x;
  Scalars* s = sc + p;
  if (what == 1 && !s->go) return;
  double acc = threadIdx.x < kPB ? partials[size_t(p) * kPB + threadIdx.x] : 0.0;
  acc = bsum(acc);
  if (threadIdx.x != 0) return;
  if (what == 0) {
    s->bnorm2 = acc;
    s->rnorm2 = acc;
    s->rnorm = sqrt(acc);
    s->inv = acc > 0.0 ? 1.0 / s->rnorm : 0.0;
    s->go = acc > 0.0 ? 1 : 0;     // a zero right-hand side needs no cycle
    s->rel = 0.0;
    return;
  }
  s->scale2 = s->rnorm2;
  s->scale = sqrt(s->scale2);
  s->rnorm2 = acc;
  s->rnorm = sqrt(acc);
  s->inv = acc > 0.0 ? 1.0 / s->rnorm : 0.0;
  const double rel = sqrt(acc / s->bnorm2);
  s->rel = rel;
  const bool finite = isfinite(rel);
  if (!finite) s->err |= DEV_NAN;
  const int go = (finite && rel > s->tol && s->cycles < s->max_cycles && s->err == 0) ? 1 : 0;
  s->go = go;
  s->cycles += go;
}

// Is any problem still active?  Drives the graph's WHILE node.
__global__ void __launch_bounds__(kNT) k_bany(const Scalars* __restrict__ sc, int nprob,
                                              cudaGraphConditionalHandle handle, int use_handle,
                                              int* any_out) {
  int any = 0;
  for (int p = threadIdx.x; p < nprob; p += blockDim.x) any |= sc[p].go;
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    *any_out = any;
    if (use_handle) cudaGraphSetConditional(handle, any ? 1u : 0u);
  }
}

__global__ void k_bupdate(const LevelV<double>* __restrict__ f64,
                          const LevelV<float>* __restrict__ f32, const int* __restrict__ pids,
                          const Scalars* __restrict__ sc) {
  const int z = blockIdx.z;
  const int p = pids[z];
  if (!sc[p].go) return;
  const LevelV<double> L = f64[z];
  const float* e = f32[z].x;
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int j = blockIdx.y + 1;
  if (i > L.nx) return;
  const double s = sc[p].scale;
  const int o = j * L.pitch + i;
  L.x[o] = fma(s, double(e[j * f32[z].pitch + i]), L.x[o]);
}

// ---------------------------------------------------------------------------
// Batched conjugate gradients (BMG_SOLVER_PCG): per problem, CG on its finest
// operator in FP64, preconditioned by one symmetric FP32 V(nu, nu) cycle of
// the batched V-cycle (r / ||r|| cast to the FP32 finest level, z = ||r|| e
// cast back), in the single-problem solver's order.  The FP64 finest level's
// b plane holds r and its x plane z; X, B, P, Q are the problem's CG planes.
// ---------------------------------------------------------------------------

struct BPcg {
  double *x, *b, *p, *q;
};

enum { BPCG_INIT = 0, BPCG_AP = 1, BPCG_XR = 2, BPCG_RZ = 3, BPCG_P = 4 };

// One problem per blockIdx.y, kPB blocks each, active problems only:
// INIT r = B - A X, z = 0, partials of r.r; AP Q = A P, partials of P.Q;
// XR X += alpha P, r -= alpha Q, z = 0, partials of r.r; RZ partials of r.z;
// P P = z + beta P.
__global__ void __launch_bounds__(kNT) k_bpcg(const LevelV<double>* __restrict__ f64,
                                              const BPcg* __restrict__ vec,
                                              const int* __restrict__ pids,
                                              const Scalars* __restrict__ sc,
                                              double* __restrict__ partials, int what) {
  const int z = blockIdx.y;
  const int pr = pids[z];
  if (!sc[pr].go) return;
  const LevelV<double> L = f64[z];
  const BPcg v = vec[z];
  const double alpha = sc[pr].alpha, beta = sc[pr].beta;
  double acc = 0.0;
  for (int j = blockIdx.x + 1; j <= L.ny; j += gridDim.x) {
    for (int i = threadIdx.x + 1; i <= L.nx; i += blockDim.x) {
      const int o = j * L.pitch + i;
      if (what == BPCG_INIT) {
        const double r = resid_value<double, false>(L, v.x, v.b[o], o);
        L.b[o] = r;
        L.x[o] = 0.0;
        acc = fma(r, r, acc);
      } else if (what == BPCG_AP) {
        const double q = -resid_value<double, false>(L, v.p, 0.0, o);
        v.q[o] = q;
        acc = fma(v.p[o], q, acc);
      } else if (what == BPCG_XR) {
        v.x[o] = fma(alpha, v.p[o], v.x[o]);
        const double r = fma(-alpha, v.q[o], L.b[o]);
        L.b[o] = r;
        L.x[o] = 0.0;
        acc = fma(r, r, acc);
      } else if (what == BPCG_RZ) {
        acc = fma(L.b[o], L.x[o], acc);
      } else {
        v.p[o] = fma(beta, v.p[o], L.x[o]);
      }
    }
  }
  if (what == BPCG_P) return;
  acc = bsum(acc);
  if (threadIdx.x == 0) partials[size_t(pr) * kPB + blockIdx.x] = acc;
}

// One block per problem: AP alpha = rz / sum (0 for a zero denominator); RZ
// beta = sum / rz (0 while rz is 0: the first direction is z), rz = sum.
__global__ void __launch_bounds__(kNT) k_bpcg_scalar(const double* __restrict__ partials,
                                                     Scalars* __restrict__ sc, int what) {
  const int pr = blockIdx.x;
  Scalars* s = sc + pr;
  if (!s->go) return;
  double acc = threadIdx.x < kPB ? partials[size_t(pr) * kPB + threadIdx.x] : 0.0;
  acc = bsum(acc);
  if (threadIdx.x != 0) return;
  if (what == BPCG_AP) {
    s->alpha = acc != 0.0 ? s->rz / acc : 0.0;
  } else {
    s->beta = s->rz != 0.0 ? acc / s->rz : 0.0;
    s->rz = acc;
  }
}

// The preconditioner's casts: dir 0, FP32 finest b = r / ||r|| and x = 0;
// dir 1, z = ||r|| e (||r|| of the latest residual, set once per problem by
// k_bnorm_final).
__global__ void k_bpcg_cast(const LevelV<double>* __restrict__ f64,
                            const LevelV<float>* __restrict__ f32, const int* __restrict__ pids,
                            const Scalars* __restrict__ sc, int dir) {
  const int z = blockIdx.z;
  const int pr = pids[z];
  if (!sc[pr].go) return;
  const LevelV<double> L = f64[z];
  const LevelV<float> F = f32[z];
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int j = blockIdx.y + 1;
  if (i > L.nx) return;
  const int o = j * L.pitch + i, of = j * F.pitch + i;
  if (dir == 0) {
    F.b[of] = float(L.b[o] * sc[pr].inv);
    F.x[of] = 0.0f;
  } else {
    L.x[o] = sc[pr].rnorm * double(F.x[of]);
  }
}

// Dense user arrays <-> FP64 finest planes, batched over one finest side.
// which: 0 the finest b plane, 1 its x plane, 2 the CG right-hand side B,
// 3 the CG iterate X.
__global__ void k_bpack(const LevelV<double>* __restrict__ f64, double* const* __restrict__ src,
                        int which, const BPcg* __restrict__ vec) {
  const int z = blockIdx.z;
  const LevelV<double> L = f64[z];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= L.nx) return;
  const double v = src[z][size_t(j) * L.nx + i];
  double* dst = which == 0 ? L.b : which == 1 ? L.x : which == 2 ? vec[z].b : vec[z].x;
  dst[(j + 1) * L.pitch + i + 1] = v;
}

// x = 0 for problems whose right-hand side is zero (they run no cycle).
// The iterate (the finest x plane, or the CG iterate X when vec is given).
__global__ void k_bzero_x(const LevelV<double>* __restrict__ f64, const int* __restrict__ pids,
                          const Scalars* __restrict__ sc, const BPcg* __restrict__ vec) {
  const int z = blockIdx.z;
  if (sc[pids[z]].bnorm2 != 0.0) return;
  const LevelV<double> L = f64[z];
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int j = blockIdx.y + 1;
  if (i > L.nx) return;
  (vec ? vec[z].x : L.x)[j * L.pitch + i] = 0.0;
}

__global__ void k_bunpack(const LevelV<double>* __restrict__ f64, double* const* __restrict__ dst,
                          const BPcg* __restrict__ vec) {
  const int z = blockIdx.z;
  const LevelV<double> L = f64[z];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= L.nx) return;
  dst[z][size_t(j) * L.nx + i] = (vec ? vec[z].x : L.x)[(j + 1) * L.pitch + i + 1];
}

// ---------------------------------------------------------------------------
// Tile variants of the batched sweep and their autotuner.
// ---------------------------------------------------------------------------

constexpr int kTileVariants = 3;   // 32x16/128 threads, 64x16/256, 128x32/256

void launch_bsweep(int variant, bool nine, int n, int count, const LevelV<float>* views,
                   const int* pids, const Scalars* sc, unsigned order, cudaStream_t s) {
#define BMG_BSWEEP(TX, TY, NT)                                                          \
  do {                                                                                  \
    const dim3 grid(cdiv(n, TX), cdiv(n, TY), count);                                   \
    if (nine)                                                                           \
      k_bsweep<true, TX, TY, NT><<<grid, NT, 0, s>>>(views, pids, sc, order);           \
    else                                                                                \
      k_bsweep<false, TX, TY, NT><<<grid, NT, 0, s>>>(views, pids, sc, order);          \
  } while (0)
  switch (variant) {
    case 0: BMG_BSWEEP(32, 16, 128); break;
    case 1: BMG_BSWEEP(64, 16, 256); break;
    default: BMG_BSWEEP(128, 32, 256); break;
  }
#undef BMG_BSWEEP
  count_launch();
}

std::mutex g_tune_mu;
std::map<std::string, int> g_tune;   // "device/n/kind/count" -> variant
bool g_tune_loaded = false;

std::string tune_key(int n, bool nine, int count) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, dev);
  char buf[256];
  std::snprintf(buf, sizeof(buf), "%s/%d/%d/%d", prop.name, n, nine ? 9 : 5, count);
  std::string k(buf);
  for (char& c : k)
    if (c == ' ') c = '_';
  return k;
}

void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("BMG_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char key[256];
  int v;
  while (std::fscanf(f, "%255s %d", key, &v) == 2) g_tune[key] = v;
  std::fclose(f);
}

void tune_store(const std::string& key, int v) {
  g_tune[key] = v;
  const char* path = std::getenv("BMG_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d\n", key.c_str(), v);
  std::fclose(f);
}

}  // namespace

// ---------------------------------------------------------------------------
// Batch object
// ---------------------------------------------------------------------------

struct BClass {                  // levels of one side and one kind across problems
  int n = 0;
  bool nine = false;
  int count = 0;
  int tile = 1;
  int* pids = nullptr;                       // device
  LevelV<float>* view[2] = {nullptr, nullptr};   // parity 0: (x, x2); 1: swapped
  LevelV<float>* coarse = nullptr;           // next coarser level of the same problems
  int parity_after_pre = 0;
};

struct BFine {                   // FP64 finest levels of the problems of one side
  int n = 0;
  int count = 0;
  int* pids = nullptr;
  LevelV<double>* f64 = nullptr;
  LevelV<float>* f32 = nullptr;
  double** user = nullptr;       // device array of user pointers (b, x)
  BPcg* pcg = nullptr;           // the problems' CG planes (BMG_SOLVER_PCG), else null
};

struct Batch {
  int nprob = 0;
  bmg_options opt{};
  std::vector<Hierarchy*> hs;
  std::vector<int> side;
  std::vector<BClass> cls;       // descending side; per side 5-point first
  std::vector<BFine> fines;
  Scalars* sc = nullptr;
  Scalars* sc_host = nullptr;
  double* partials = nullptr;
  BCoarse* pc = nullptr;
  int* any = nullptr;
  void* arena = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle handle = 0;
  double setup_ms = 0.0;
};

namespace {

template <typename T>
T* carve(char*& p, size_t n) {
  T* r = reinterpret_cast<T*>(p);
  p += ((n * sizeof(T) + 255) / 256) * 256;
  return r;
}

void destroy_batch(Batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (Hierarchy* h : b->hs) free_hierarchy(h);
  if (b->arena) cudaFree(b->arena);
  if (b->sc_host) cudaFreeHost(b->sc_host);
  delete b;
}

// Downward half of the batched V-cycle, coarse kernel, upward half.
void enqueue_bvcycle(Batch* b, cudaStream_t s) {
  const int nu1 = b->opt.nu1, nu2 = b->opt.nu2;
  const bool oop = ((nu1 + nu2) & 1) != 0;
  for (BClass& c : b->cls) {
    int par = 0;
    for (int k = 0; k < nu1; ++k) {
      launch_bsweep(c.tile, c.nine, c.n, c.count, c.view[par], c.pids, b->sc,
                    c.nine ? four_order(false) : rb_order(false), s);
      par ^= 1;
    }
    const dim3 g(cdiv(c.n, 128), c.n, c.count);
    if (c.nine)
      k_bresid<true><<<g, 128, 0, s>>>(c.view[par], c.pids, b->sc);
    else
      k_bresid<false><<<g, 128, 0, s>>>(c.view[par], c.pids, b->sc);
    const int nc = (c.n - 1) / 2;
    k_brestrict<<<dim3(cdiv(nc, 128), nc, c.count), 128, 0, s>>>(c.view[par], c.coarse, c.pids,
                                                                  b->sc);
    count_launch(2);
    c.parity_after_pre = par;
  }
  k_bcoarse<<<b->nprob, 1024, 0, s>>>(b->pc, b->sc, nu1, nu2);
  count_launch();
  for (auto it = b->cls.rbegin(); it != b->cls.rend(); ++it) {
    BClass& c = *it;
    int par = c.parity_after_pre;
    k_binterp<<<dim3(cdiv(c.n, 128), c.n, c.count), 128, 0, s>>>(c.view[par], c.coarse, c.pids,
                                                                  b->sc, oop ? 1 : 0);
    count_launch();
    if (oop) par ^= 1;
    for (int k = 0; k < nu2; ++k) {
      launch_bsweep(c.tile, c.nine, c.n, c.count, c.view[par], c.pids, b->sc,
                    c.nine ? four_order(true) : rb_order(true), s);
      par ^= 1;
    }
  }
}

void enqueue_residuals(Batch* b, int what, bool use_handle, cudaStream_t s) {
  for (BFine& f : b->fines) {
    k_brefine_resid<<<dim3(kPB, f.count), kNT, 0, s>>>(f.f64, f.f32, f.pids, b->sc, b->partials,
                                                      what);
  }
  k_bnorm_final<<<b->nprob, kNT, 0, s>>>(b->partials, b->sc, what);
  k_bany<<<1, kNT, 0, s>>>(b->sc, b->nprob, b->handle, use_handle ? 1 : 0, b->any);
  count_launch(int(b->fines.size()) + 2);
}

void enqueue_update(Batch* b, cudaStream_t s) {
  for (BFine& f : b->fines) {
    k_bupdate<<<dim3(cdiv(f.n, 128), f.n, f.count), 128, 0, s>>>(f.f64, f.f32, f.pids, b->sc);
  }
  count_launch(int(b->fines.size()));
}

void enqueue_pcg_vec(Batch* b, int what, cudaStream_t s) {
  for (BFine& f : b->fines)
    k_bpcg<<<dim3(kPB, f.count), kNT, 0, s>>>(f.f64, f.pcg, f.pids, b->sc, b->partials, what);
  count_launch(int(b->fines.size()));
}

void enqueue_pcg_cast(Batch* b, int dir, cudaStream_t s) {
  for (BFine& f : b->fines)
    k_bpcg_cast<<<dim3(cdiv(f.n, 128), f.n, f.count), 128, 0, s>>>(f.f64, f.f32, f.pids, b->sc, dir);
  count_launch(int(b->fines.size()));
}

// The first residual of PCG (r = B - A X, z = 0) and its stop test.
void enqueue_pcg_init(Batch* b, cudaStream_t s) {
  enqueue_pcg_vec(b, BPCG_INIT, s);
  k_bnorm_final<<<b->nprob, kNT, 0, s>>>(b->partials, b->sc, 1);
  k_bany<<<1, kNT, 0, s>>>(b->sc, b->nprob, b->handle, 0, b->any);
  count_launch(2);
}

// One batched PCG iteration of the active problems: z = M^{-1} r (the FP32
// batched V-cycle between the casts), r.z and beta, p = z + beta p,
// q = A p and alpha, x += alpha p and r -= alpha q, the stop test, any.
void enqueue_pcg_iter(Batch* b, bool use_handle, cudaStream_t s) {
  enqueue_pcg_cast(b, 0, s);
  enqueue_bvcycle(b, s);
  enqueue_pcg_cast(b, 1, s);
  enqueue_pcg_vec(b, BPCG_RZ, s);
  k_bpcg_scalar<<<b->nprob, kNT, 0, s>>>(b->partials, b->sc, BPCG_RZ);
  enqueue_pcg_vec(b, BPCG_P, s);
  enqueue_pcg_vec(b, BPCG_AP, s);
  k_bpcg_scalar<<<b->nprob, kNT, 0, s>>>(b->partials, b->sc, BPCG_AP);
  enqueue_pcg_vec(b, BPCG_XR, s);
  k_bnorm_final<<<b->nprob, kNT, 0, s>>>(b->partials, b->sc, 1);
  k_bany<<<1, kNT, 0, s>>>(b->sc, b->nprob, b->handle, use_handle ? 1 : 0, b->any);
  count_launch(4);
}

// Pick the fastest tile variant of every class by timing sweeps on the batch
// (x = 0 and b = 0 after setup, so the timing sweeps change nothing).
int autotune(Batch* b, cudaStream_t s) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  tune_load();
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return BMG_ECUDA;
  // every problem must count as active while timing
  for (int p = 0; p < b->nprob; ++p) b->sc_host[p] = Scalars{};
  std::vector<Scalars> act(b->nprob);
  for (auto& a : act) a.go = 1;
  cudaMemcpyAsync(b->sc, act.data(), sizeof(Scalars) * b->nprob, cudaMemcpyHostToDevice, s);
  for (BClass& c : b->cls) {
    const std::string key = tune_key(c.n, c.nine, c.count);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      c.tile = it->second;
      continue;
    }
    float best = 1e30f;
    int bv = 1;
    for (int v = 0; v < kTileVariants; ++v) {
      const unsigned order = c.nine ? four_order(false) : rb_order(false);
      launch_bsweep(v, c.nine, c.n, c.count, c.view[0], c.pids, b->sc, order, s);
      cudaEventRecord(e0, s);
      for (int r = 0; r < 3; ++r)
        launch_bsweep(v, c.nine, c.n, c.count, c.view[0], c.pids, b->sc, order, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        bv = v;
      }
    }
    c.tile = bv;
    tune_store(key, bv);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return cudaGetLastError() == cudaSuccess ? BMG_OK : BMG_ECUDA;
}

int build_graph_on(Batch* b, cudaStream_t s);

// The refinement loop as one graph: WHILE(any active) { V-cycle; update;
// residuals + stop tests + any }, or (BMG_SOLVER_PCG) WHILE(any active) {
// one PCG iteration }.  Recorded on a private stream (the
// caller's stream may be the legacy default stream, which cannot capture);
// recording executes nothing.
int build_graph(Batch* b) {
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return BMG_ECUDA;
  const int rc = build_graph_on(b, s);
  cudaStreamDestroy(s);
  return rc;
}

int build_graph_on(Batch* b, cudaStream_t s) {
  if (cudaGraphCreate(&b->graph, 0) != cudaSuccess) return BMG_ECUDA;
  if (cudaGraphConditionalHandleCreate(&b->handle, b->graph, 1, cudaGraphCondAssignDefault) !=
      cudaSuccess)
    return BMG_ECUDA;
  // zeroed storage: the struct's unions have no default constructor
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  std::memset(raw, 0, sizeof(raw));
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(raw);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = b->handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, b->graph, nullptr, nullptr, 0, &cp) != cudaSuccess) return BMG_ECUDA;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if (cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
      cudaSuccess)
    return BMG_ECUDA;
  if (b->opt.solver == BMG_SOLVER_PCG) {
    enqueue_pcg_iter(b, true, s);
  } else {
    enqueue_bvcycle(b, s);
    enqueue_update(b, s);
    enqueue_residuals(b, 1, true, s);
  }
  cudaGraph_t out = nullptr;
  if (cudaStreamEndCapture(s, &out) != cudaSuccess) return BMG_ECUDA;
  if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) return BMG_ECUDA;
  return BMG_OK;
}

double now_ms() {
  return std::chrono::duration<double, std::milli>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

}  // namespace

}  // namespace bmg

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

using bmg::Batch;

extern "C" int bmg_batch_setup(int nprob, const double* const* k_dev, const int* n,
                               const bmg_options* opt_in, bmg_stream_t stream, bmg_batch** out) {
  using namespace bmg;
  if (!out) return BMG_EINVAL;
  *out = nullptr;
  if (nprob < 1 || !k_dev || !n) return BMG_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const double t0 = now_ms();
  bmg_options opt;
  bmg_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (opt.smoother != BMG_SMOOTH_POINT) {
    set_last_error("batch setup: only the point smoother is batched");
    return BMG_EINVAL;
  }
  if (opt.solver == BMG_SOLVER_PCG && (opt.nu1 != opt.nu2 || opt.interp_residual_term)) {
    set_last_error("batch setup: BMG_SOLVER_PCG needs nu1 == nu2 and interp_residual_term == 0");
    return BMG_EINVAL;
  }
  if (opt.solver != BMG_SOLVER_VCYCLE && opt.solver != BMG_SOLVER_PCG) return BMG_EINVAL;
  opt.precision = BMG_FP32_REFINE;
  Batch* b = new Batch();
  b->nprob = nprob;
  b->opt = opt;
  auto fail = [&](int code) {
    destroy_batch(b);
    return code;
  };
  // individual hierarchies (threshold: levels of side <= 31 in the coarse kernel)
  for (int p = 0; p < nprob; ++p) {
    // batched problems: square, sides 2^m - 1 (the level classes below rely on it)
    if (!k_dev[p] || n[p] < 3 || ((n[p] + 1) & n[p]) != 0) return fail(BMG_EINVAL);
    int levels_small = 0;
    for (int m = n[p]; m >= 3; m = (m - 1) / 2)
      if (m <= kCoarseSide) ++levels_small;
    bmg_options o = opt;
    o.coarse_threshold = std::max(1, levels_small);
    o.coarse_ctas = 1;         // the batched coarse kernel runs one block per problem
    Hierarchy* h = nullptr;
    const int rc = setup_impl(k_dev[p], n[p], n[p], &o, s, &h);
    if (rc) {
      set_last_error("batch setup: problem %d: %s", p, bmg_last_error());
      return fail(rc);
    }
    b->hs.push_back(h);
    b->side.push_back(n[p]);
  }
  // classes: for each side > kCoarseSide, the 5-point finest levels and the
  // 9-point levels of larger problems
  std::vector<int> sides;
  for (int v : b->side)
    for (int m = v; m > kCoarseSide; m = (m - 1) / 2) sides.push_back(m);
  std::sort(sides.begin(), sides.end(), std::greater<int>());
  sides.erase(std::unique(sides.begin(), sides.end()), sides.end());
  struct HostClass {
    BClass c;
    std::vector<int> pids;
    std::vector<LevelV<float>> v0, v1, vc;
  };
  std::vector<HostClass> hc;
  for (int m : sides) {
    for (int kind = 0; kind < 2; ++kind) {
      HostClass x;
      x.c.n = m;
      x.c.nine = kind == 1;
      for (int p = 0; p < nprob; ++p) {
        const Hierarchy* h = b->hs[p];
        const bool finest = b->side[p] == m;
        if (b->side[p] < m || finest == x.c.nine) continue;
        int l = h->L - 1;
        while (h->f[l].nx != m) --l;
        LevelV<float> a = h->f[l], bb = h->f[l];
        std::swap(bb.x, bb.x2);
        x.pids.push_back(p);
        x.v0.push_back(a);
        x.v1.push_back(bb);
        x.vc.push_back(h->f[l - 1]);
      }
      x.c.count = int(x.pids.size());
      if (x.c.count) hc.push_back(std::move(x));
    }
  }
  std::map<int, std::vector<int>> by_side;
  for (int p = 0; p < nprob; ++p) by_side[b->side[p]].push_back(p);
  // device arena for the descriptors
  size_t bytes = 0;
  auto al = [](size_t v) { return ((v + 255) / 256) * 256; };
  for (auto& x : hc) bytes += al(sizeof(int) * x.c.count) + 3 * al(sizeof(LevelV<float>) * x.c.count);
  for (auto& kv : by_side)
    bytes += al(sizeof(int) * kv.second.size()) + al(sizeof(LevelV<double>) * kv.second.size()) +
             al(sizeof(LevelV<float>) * kv.second.size()) + al(sizeof(double*) * kv.second.size()) +
             al(sizeof(BPcg) * kv.second.size());
  bytes += al(sizeof(Scalars) * nprob) + al(sizeof(double) * kPB * nprob) +
           al(sizeof(BCoarse) * nprob) + al(sizeof(int));
  if (cudaMalloc(&b->arena, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(BMG_ENOMEM);
  }
  if (cudaMallocHost(&b->sc_host, sizeof(Scalars) * nprob) != cudaSuccess) return fail(BMG_ENOMEM);
  char* cur = static_cast<char*>(b->arena);
  for (auto& x : hc) {
    BClass c = x.c;
    c.pids = carve<int>(cur, c.count);
    c.view[0] = carve<LevelV<float>>(cur, c.count);
    c.view[1] = carve<LevelV<float>>(cur, c.count);
    c.coarse = carve<LevelV<float>>(cur, c.count);
    cudaMemcpyAsync(c.pids, x.pids.data(), sizeof(int) * c.count, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(c.view[0], x.v0.data(), sizeof(LevelV<float>) * c.count, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(c.view[1], x.v1.data(), sizeof(LevelV<float>) * c.count, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(c.coarse, x.vc.data(), sizeof(LevelV<float>) * c.count, cudaMemcpyHostToDevice, s);
    b->cls.push_back(c);
  }
  for (auto& kv : by_side) {
    BFine f;
    f.n = kv.first;
    f.count = int(kv.second.size());
    std::vector<LevelV<double>> v64;
    std::vector<LevelV<float>> v32;
    std::vector<BPcg> vp;
    for (int p : kv.second) {
      const Hierarchy* h = b->hs[p];
      v64.push_back(h->d.back());
      v32.push_back(h->f.back());
      vp.push_back(BPcg{h->pcg_x, h->pcg_b, h->pcg_p, h->pcg_q});
    }
    f.pids = carve<int>(cur, f.count);
    f.f64 = carve<LevelV<double>>(cur, f.count);
    f.f32 = carve<LevelV<float>>(cur, f.count);
    f.user = carve<double*>(cur, f.count);
    BPcg* pcg_dev = carve<BPcg>(cur, f.count);
    if (opt.solver == BMG_SOLVER_PCG) {
      f.pcg = pcg_dev;
      cudaMemcpyAsync(f.pcg, vp.data(), sizeof(BPcg) * f.count, cudaMemcpyHostToDevice, s);
    }
    cudaMemcpyAsync(f.pids, kv.second.data(), sizeof(int) * f.count, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(f.f64, v64.data(), sizeof(LevelV<double>) * f.count, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(f.f32, v32.data(), sizeof(LevelV<float>) * f.count, cudaMemcpyHostToDevice, s);
    b->fines.push_back(f);
  }
  b->sc = carve<Scalars>(cur, nprob);
  b->partials = carve<double>(cur, size_t(kPB) * nprob);
  b->pc = carve<BCoarse>(cur, nprob);
  b->any = carve<int>(cur, 1);
  std::vector<BCoarse> pcs(nprob);
  for (int p = 0; p < nprob; ++p) {
    const Hierarchy* h = b->hs[p];
    pcs[p] = BCoarse{h->dlev32, h->chol, h->chol_idiag, h->threshold, h->n0,
                     h->threshold < h->L ? 1 : 0};
  }
  cudaMemcpyAsync(b->pc, pcs.data(), sizeof(BCoarse) * nprob, cudaMemcpyHostToDevice, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(BMG_ECUDA);
  int rc = autotune(b, s);
  if (rc) return fail(rc);
  if ((rc = build_graph(b))) {
    set_last_error("batch setup: building the CUDA graph failed (%s)",
                   cudaGetErrorString(cudaGetLastError()));
    return fail(rc);
  }
  b->setup_ms = now_ms() - t0;
  *out = reinterpret_cast<bmg_batch*>(b);
  return BMG_OK;
}

extern "C" int bmg_batch_solve(bmg_batch* bp, const double* const* b_dev, double* const* x_dev,
                               double tol, bmg_info* per_prob, bmg_stream_t stream) {
  using namespace bmg;
  Batch* b = reinterpret_cast<Batch*>(bp);
  if (!b || !b_dev || !x_dev || !(tol > 0.0)) return BMG_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const double t0 = now_ms();
  // pack b and x (batched per finest side)
  std::map<int, std::vector<int>> by_side;
  for (int p = 0; p < b->nprob; ++p) by_side[b->side[p]].push_back(p);
  const bool pcg = b->opt.solver == BMG_SOLVER_PCG;
  for (int pass = 0; pass < 2; ++pass) {
    for (BFine& f : b->fines) {
      std::vector<double*> ptr;
      for (int p : by_side[f.n]) ptr.push_back(pass == 0 ? const_cast<double*>(b_dev[p]) : x_dev[p]);
      cudaMemcpyAsync(f.user, ptr.data(), sizeof(double*) * ptr.size(), cudaMemcpyHostToDevice, s);
      const dim3 g(cdiv(f.n, 128), f.n, f.count);
      // V-cycles: b and x into the finest planes; PCG: b also into B, x into X
      if (pass == 0 || !pcg) k_bpack<<<g, 128, 0, s>>>(f.f64, f.user, pass, f.pcg);
      if (pcg) k_bpack<<<g, 128, 0, s>>>(f.f64, f.user, pass == 0 ? 2 : 3, f.pcg);
      count_launch(pcg && pass == 0 ? 2 : 1);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return BMG_ECUDA;
  }
  for (int p = 0; p < b->nprob; ++p) {
    Scalars z{};
    z.tol = tol;
    z.max_cycles = b->opt.max_cycles;
    b->sc_host[p] = z;
  }
  cudaMemcpyAsync(b->sc, b->sc_host, sizeof(Scalars) * b->nprob, cudaMemcpyHostToDevice, s);
  enqueue_residuals(b, 0, false, s);       // ||b||, go = (b != 0)
  if (pcg)
    enqueue_pcg_init(b, s);                // r = B - A X and the stop test
  else
    enqueue_residuals(b, 1, false, s);     // first residual and stop test
  if (cudaGraphLaunch(b->exec, s) != cudaSuccess) return BMG_ECUDA;
  for (BFine& f : b->fines) {
    k_bzero_x<<<dim3(cdiv(f.n, 128), f.n, f.count), 128, 0, s>>>(f.f64, f.pids, b->sc, f.pcg);
    count_launch();
    std::vector<double*> ptr;
    for (int p : by_side[f.n]) ptr.push_back(x_dev[p]);
    cudaMemcpyAsync(f.user, ptr.data(), sizeof(double*) * ptr.size(), cudaMemcpyHostToDevice, s);
    k_bunpack<<<dim3(cdiv(f.n, 128), f.n, f.count), 128, 0, s>>>(f.f64, f.user, f.pcg);
    count_launch();
    if (cudaStreamSynchronize(s) != cudaSuccess) return BMG_ECUDA;
  }
  if (cudaMemcpyAsync(b->sc_host, b->sc, sizeof(Scalars) * b->nprob, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return BMG_ECUDA;
  const double ms = now_ms() - t0;
  int rc = BMG_OK;
  for (int p = 0; p < b->nprob; ++p) {
    const Scalars& r = b->sc_host[p];
    if (per_prob) per_prob[p] = bmg_info{r.cycles, b->hs[p]->threshold, r.rel, b->setup_ms, ms, 1};
    if (r.err & DEV_NAN) rc = BMG_ENAN;
    else if (!(r.rel <= tol) && r.bnorm2 > 0.0 && rc == BMG_OK) rc = BMG_ENOCONV;
  }
  return rc;
}

extern "C" void bmg_batch_destroy(bmg_batch* bp) { bmg::destroy_batch(reinterpret_cast<Batch*>(bp)); }

extern "C" int bmg_batch_size(const bmg_batch* bp, int* nprob) {
  const Batch* b = reinterpret_cast<const Batch*>(bp);
  if (!b || !nprob) return BMG_EINVAL;
  *nprob = b->nprob;
  return BMG_OK;
}
