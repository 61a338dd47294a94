// Host side of the GB300 BoxMG library: the hierarchy (one device arena per
// setup), the setup sequence of Section 2, the V-cycle launch schedule of
// Algorithm 1 with the coarse levels below the threshold run by one
// persistent kernel (the single-GPU reading of Algorithm 2), the solve loops
// (plain FP64, and FP32 V-cycles inside FP64 iterative refinement), and the
// extern "C" entry points declared in include/boxmg.h.
#include "bmg_internal.h"
#include "bmg_schedule.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <tuple>
#include <utility>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <type_traits>

namespace bmg {

static thread_local char g_last_error[256] = "";

void set_last_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
}

namespace {

#define BMG_CUDA(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return BMG_ECUDA;            \
  } while (0)

// Grid sides: any n >= 2 (a side of n points coarsens to floor(n / 2)).
bool valid_side(int n) { return n >= 2; }

double now_ms() {
  using clk = std::chrono::steady_clock;
  return std::chrono::duration<double, std::milli>(clk::now().time_since_epoch()).count();
}

// Carves planes out of one allocation.  First pass (base == nullptr) only
// counts bytes.
struct Carver {
  char* base = nullptr;
  size_t off = 0;
  template <typename T>
  T* plane(const Geom& g) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) + base_shift<T>() : nullptr;
    off += g.elems * sizeof(T);
    return p;
  }
  template <typename T>
  T* raw(size_t n) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += n * sizeof(T);
    return p;
  }
};

template <typename T>
void carve_levels(Carver& cv, const std::vector<Geom>& geo, int first, std::vector<LevelV<T>>& lv,
                  int finest_index, int smoother, bool prescale = false) {
  const bool xl = smoother == BMG_SMOOTH_XLINE || smoother == BMG_SMOOTH_ALTLINE;
  const bool yl = smoother == BMG_SMOOTH_YLINE || smoother == BMG_SMOOTH_ALTLINE;
  // lv[i] corresponds to hierarchy level first + i.
  const int n = int(geo.size());
  lv.assign(n, LevelV<T>{});
  for (int i = 0; i < n; ++i) {
    const int l = first + i;
    const Geom& g = geo[i];
    LevelV<T>& L = lv[i];
    L.nx = g.nx;
    L.ny = g.ny;
    L.pitch = g.pitch;
    L.C = cv.plane<T>(g);
    L.iC = cv.plane<T>(g);
    L.W = cv.plane<T>(g);
    L.S = cv.plane<T>(g);
    const bool nine = l != finest_index;
    L.SW = nine ? cv.plane<T>(g) : nullptr;
    L.NW = nine ? cv.plane<T>(g) : nullptr;
    L.x = cv.plane<T>(g);
    L.x2 = cv.plane<T>(g);
    L.b = cv.plane<T>(g);
    L.r = cv.plane<T>(g);
    for (int k = 0; k < 5; ++k) L.PR[k] = prescale && l == finest_index ? cv.plane<T>(g) : nullptr;
    // colour-compacted planes of the y-lines: (ny + 2) rows of ycp columns
    // per colour, ycp >= the columns of a colour, a multiple of 32
    L.ycp = ((g.nx + 1) / 2 + 31) / 32 * 32;
    L.yhalf = (g.ny + 2) * L.ycp;
    L.ys = yl ? cv.raw<T>(2 * size_t(L.yhalf)) : nullptr;
    for (int d = 0; d < 2; ++d) {
      const bool use = d == 0 ? xl : yl;
      for (int k = 0; k < NLF; ++k)
        L.LF[d][k] = !use ? nullptr : d == 0 ? cv.plane<T>(g) : cv.raw<T>(2 * size_t(L.yhalf));
      const int n = d == 0 ? g.nx : g.ny, nl = d == 0 ? g.ny : g.nx;
      const int nsep = n / kLineM;
      L.spp[d] = use && nsep > 0 ? (nsep + 3) / 4 * 4 : 0;
      L.sgl[d] = std::max(16, (nsep + 255) / 256);   // at most 256 groups per line
      // (16 = the separator kernel's register group: lines up to 65551 points)
      for (int k = 0; k < NSP; ++k)
        L.SP[d][k] = L.spp[d] ? cv.raw<T>(size_t(nl + 1) * L.spp[d]) : nullptr;
    }
    if (l >= 1 && i >= 1) {
      const Geom& gc = geo[i - 1];
      for (int k = 0; k < NPW; ++k) L.P[k] = cv.plane<T>(gc);
      L.cpitch = gc.pitch;
    } else {
      for (int k = 0; k < NPW; ++k) L.P[k] = nullptr;
      L.cpitch = 0;
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Setup
// ---------------------------------------------------------------------------

static int check_derr(Hierarchy* h, cudaStream_t s) {
  if (cudaMemcpyAsync(h->sc_host, h->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    set_last_error("setup: %s", cudaGetErrorString(cudaGetLastError()));
    return BMG_ECUDA;
  }
  const int e = h->sc_host->err;
  if (e & DEV_BADK) {
    set_last_error("setup: a coefficient k is not finite and positive");
    return BMG_EINVAL;
  }
  if (e & DEV_BADDEN) {
    char lv[96] = "";
    for (int l = 0; l < 20; ++l)
      if (e & (1 << (8 + l))) std::snprintf(lv + std::strlen(lv), sizeof(lv) - std::strlen(lv), " %d", l);
    set_last_error("setup: interpolation denominator <= 0 building P on level(s)%s", lv);
    return BMG_EINVAL;
  }
  if (e & DEV_NOTSPD) {
    set_last_error("setup: coarsest operator is not positive definite");
    return BMG_EINVAL;
  }
  if (e & DEV_BADLINE) {
    set_last_error("setup: a line system of the line smoother has a non-positive pivot");
    return BMG_EINVAL;
  }
  return BMG_OK;
}

template <typename T>
static int build_coarse(Hierarchy* h, std::vector<LevelV<T>>& lv, cudaStream_t s) {
  int* derr = &h->sc->err;
  const int L = h->L;
  for (int l = L - 1; l >= 1; --l) {
    const bool nine = l != L - 1;
    if (launch_interp_weights<T>(lv[l], nine, derr, l, s)) return BMG_ECUDA;
    if (launch_rap<T>(lv[l], nine, lv[l - 1], s)) return BMG_ECUDA;
  }
  // line factors of every level the smoother visits (all but the coarsest)
  if (h->opt.smoother != BMG_SMOOTH_POINT)
    for (int l = L - 1; l >= 1; --l)
      if (launch_line_factor<T>(lv[l], h->opt.smoother, derr, s)) return BMG_ECUDA;
  return BMG_OK;
}

void free_hierarchy(Hierarchy* h) {
  if (!h) return;
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  if (h->arena) cudaFree(h->arena);
  if (h->sc_host) cudaFreeHost(h->sc_host);
  for (auto* m : h->maps64) delete m;
  for (auto* m : h->maps32) delete m;
  delete h;
}

int setup_impl(const double* k, int nx, int ny, const bmg_options* opt_in, cudaStream_t s,
               Hierarchy** out) {
  *out = nullptr;
  g_last_error[0] = 0;
  if (!k || !valid_side(nx) || !valid_side(ny)) return BMG_EINVAL;
  bmg_options opt;
  bmg_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (opt.nu1 < 0 || opt.nu2 < 0 || opt.nu1 + opt.nu2 < 1 || opt.max_cycles < 0) return BMG_EINVAL;
  if (opt.precision != BMG_FP64 && opt.precision != BMG_FP32_REFINE) return BMG_EINVAL;
  if (opt.solver != BMG_SOLVER_VCYCLE && opt.solver != BMG_SOLVER_PCG) return BMG_EINVAL;
  if (opt.smoother < BMG_SMOOTH_POINT || opt.smoother > BMG_SMOOTH_ALTLINE) {
    set_last_error("smoother must be one of BMG_SMOOTH_*");
    return BMG_EINVAL;
  }
  if (!(opt.aniso_r > 0.0 && opt.aniso_r < INFINITY && opt.cell_aspect > 0.0 &&
        opt.cell_aspect < INFINITY)) {
    set_last_error("aniso_r and cell_aspect must be finite and positive");
    return BMG_EINVAL;
  }
  {
    int neumann = 0;
    for (double b : opt.bc_beta) {
      if (!(b < INFINITY) || b != b) {
        set_last_error("bc_beta entries must be finite");
        return BMG_EINVAL;
      }
      neumann += b == 0.0;
    }
    if (neumann == 4) {
      set_last_error("Neumann on every wall: the operator is singular");
      return BMG_EINVAL;
    }
  }
  if (opt.solver == BMG_SOLVER_PCG && (opt.nu1 != opt.nu2 || opt.interp_residual_term)) {
    set_last_error("BMG_SOLVER_PCG needs nu1 == nu2 and interp_residual_term == 0 "
                   "(a symmetric V-cycle)");
    return BMG_EINVAL;
  }
  const double t0 = now_ms();
  prepare_sweep_kernels();

  Hierarchy* h = new (std::nothrow) Hierarchy();
  if (!h) return BMG_ENOMEM;
  if (const char* e = std::getenv("BMG_FUSED_NORM")) h->fused_norm_allowed = e[0] != '0';
  h->nx = nx;
  h->ny = ny;
  h->opt = opt;
  // level sizes, finest last
  std::vector<std::pair<int, int>> sz;
  {
    int a = nx, b = ny;
    sz.push_back({a, b});
    while (std::min(a, b) > 3) {
      a = a / 2;   // coarse point I is fine point 2I
      b = b / 2;
      sz.push_back({a, b});
    }
  }
  h->L = int(sz.size());
  const int L = h->L;
  h->n0 = sz.back().first * sz.back().second;
  if (h->n0 > BMG_MAX_COARSEST) {
    delete h;
    return BMG_EINVAL;
  }
  if (opt.coarse_threshold != -1 && (opt.coarse_threshold < 1 || opt.coarse_threshold > L)) {
    delete h;
    return BMG_EINVAL;
  }
  if (opt.coarse_ctas != -1 &&
      (opt.coarse_ctas < 1 || opt.coarse_ctas > 16 ||
       (opt.coarse_ctas > 1 && (opt.smoother != BMG_SMOOTH_POINT ||
                                opt.coarse_ctas > max_cluster_ctas(opt.precision == BMG_FP32_REFINE))))) {
    set_last_error("coarse_ctas must be -1 or 1..%d, and 1 with a line smoother",
                   max_cluster_ctas(opt.precision == BMG_FP32_REFINE));
    delete h;
    return BMG_EINVAL;
  }
  const bool fp32 = opt.precision == BMG_FP32_REFINE;
  for (int l = 0; l < L; ++l) {
    const auto& q = sz[L - 1 - l];
    h->geo64.push_back(make_geom<double>(q.first, q.second));
    h->geo32.push_back(make_geom<float>(q.first, q.second));
  }
  h->npartials = 4 * 152;

  // Two passes: size, then carve.
  std::vector<Geom> g64 = fp32 ? std::vector<Geom>{h->geo64.back()} : h->geo64;
  Carver cv;
  for (int pass = 0; pass < 2; ++pass) {
    cv.off = 0;
    carve_levels<double>(cv, g64, fp32 ? L - 1 : 0, h->d, L - 1,
                         fp32 ? BMG_SMOOTH_POINT : opt.smoother,
                         !fp32 && opt.smoother == BMG_SMOOTH_POINT && prescale_enabled(nx));
    if (fp32) carve_levels<float>(cv, h->geo32, 0, h->f, L - 1, opt.smoother);
    h->kcopy = cv.raw<double>(size_t(nx) * ny);
    h->chol = cv.raw<double>(size_t(h->n0) * h->n0);
    h->chol_idiag = cv.raw<double>(h->n0);
    h->partials = cv.raw<double>(h->npartials);
    h->hist = cv.raw<double>(BMG_MAX_HISTORY);
    h->sc = cv.raw<Scalars>(1);
    h->dlev64 = cv.raw<LevelV<double>>(L);
    h->dlev32 = cv.raw<LevelV<float>>(L);
    if (opt.solver == BMG_SOLVER_PCG) {
      const Geom& gf = h->geo64.back();
      h->pcg_x = cv.plane<double>(gf);
      h->pcg_b = cv.plane<double>(gf);
      h->pcg_p = cv.plane<double>(gf);
      h->pcg_q = cv.plane<double>(gf);
    }
    if (pass == 0) {
      h->arena_bytes = cv.off;
      if (cudaMalloc(&h->arena, h->arena_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return BMG_ENOMEM;
      }
      cv.base = static_cast<char*>(h->arena);
    }
  }
  if (cudaMallocHost(&h->sc_host, sizeof(Scalars)) != cudaSuccess) {
    free_hierarchy(h);
    return BMG_ENOMEM;
  }
  int rc = BMG_OK;
  auto fail = [&](int code) {
    free_hierarchy(h);
    return code;
  };
  if (cudaMemsetAsync(h->arena, 0, h->arena_bytes, s) != cudaSuccess) return fail(BMG_ECUDA);

  // Assembly (Section 5), then P and RAP level by level (Section 2).
  int* derr = &h->sc->err;
  LevelV<double>& fine64 = h->d.back();
  if (launch_assemble<double>(k, nx, ny, fine64, h->kcopy, derr, opt.log_coefficients != 0,
                              opt.aniso_r, opt.cell_aspect, opt.bc_beta, s))
    return fail(BMG_ECUDA);
  if (fine64.PR[PR_B]) launch_prescale_coeffs<double>(fine64, s);
  if (!fp32) {
    if ((rc = build_coarse<double>(h, h->d, s))) return fail(rc);
    if (launch_coarse_factor(h, &h->d[0], nullptr, s)) return fail(BMG_ECUDA);
  } else {
    if (launch_downcast_fine(fine64, h->f.back(), s)) return fail(BMG_ECUDA);
    if ((rc = build_coarse<float>(h, h->f, s))) return fail(rc);
    if (launch_coarse_factor(h, nullptr, &h->f[0], s)) return fail(BMG_ECUDA);
  }
  // level views for the persistent kernel
  if (!fp32) {
    if (cudaMemcpyAsync(h->dlev64, h->d.data(), sizeof(LevelV<double>) * L,
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
      return fail(BMG_ECUDA);
  } else {
    if (cudaMemcpyAsync(h->dlev32, h->f.data(), sizeof(LevelV<float>) * L,
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
      return fail(BMG_ECUDA);
  }
  if ((rc = check_derr(h, s))) return fail(rc);

  // TMA descriptors of every level swept by the TMA-staged kernel
  auto make_maps = [&](auto& lv, auto& maps) {
    using M = std::remove_pointer_t<typename std::remove_reference_t<decltype(maps)>::value_type>;
    maps.assign(lv.size(), nullptr);
    for (size_t l = 0; l < lv.size(); ++l) {
      M* m = new M;
      if (make_sweep_maps(lv[l], derr, m))
        maps[l] = m;
      else
        delete m;
    }
  };
  if (!fp32) {
    make_maps(h->d, h->maps64);
  } else {
    make_maps(h->f, h->maps32);
  }

  // Level schedule: which levels leave the full-grid launches, and how many
  // blocks run them.
  choose_schedule(h);
  h->setup_ms = now_ms() - t0;
  *out = h;
  return BMG_OK;
}

// ---------------------------------------------------------------------------
// V-cycle schedule (Algorithm 1)
// ---------------------------------------------------------------------------

// TMA descriptors of level l of the FP64 (d) or FP32 (f) hierarchy, or null.
template <typename T>
const SweepMaps<T>* level_maps(const Hierarchy* h, int l);
template <>
const SweepMaps<double>* level_maps<double>(const Hierarchy* h, int l) {
  return l >= 0 && l < int(h->maps64.size()) ? h->maps64[l] : nullptr;
}
template <>
const SweepMaps<float>* level_maps<float>(const Hierarchy* h, int l) {
  return l >= 0 && l < int(h->maps32.size()) ? h->maps32[l] : nullptr;
}

template <typename T>
void enqueue_vcycle(Hierarchy* h, std::vector<LevelV<T>>& lv, const LevelV<T>* dlev, int thr,
                    cudaStream_t s, int top, bool skip_first, bool top_zero) {
  const int L = h->L;
  // a cycle from level `top` down (the finest unless given): the levels
  // below the schedule's threshold still run in the persistent kernel
  if (top < 0 || top > L - 1) top = L - 1;
  thr = std::min(thr, top + 1);
  const int nu1 = h->opt.nu1, nu2 = h->opt.nu2;
  const bool rc = h->opt.interp_residual_term != 0;
  // Sweeps write the other iterate buffer; with nu1 + nu2 odd the
  // interpolation also writes out of place, so every level's iterate is back
  // in lv[l].x when the cycle ends and every cycle issues the same launches.
  const bool interp_oop = ((nu1 + nu2) & 1) != 0;
  // zero: the level's iterate is zero (its first pre-sweep: every level below
  // the top was zeroed by its restriction); the sweep may then take the
  // zero-start form (environment BMG_ZERO_START=0 turns it off)
  static const bool zero_start = [] {
    const char* e = std::getenv("BMG_ZERO_START");
    return !(e && e[0] == '0');
  }();
  auto sweep = [&](int l, bool reverse, bool zero) {
    zero = zero && zero_start;
    LevelV<T>& V = lv[l];
    const bool nine = l != L - 1;
    if (!nine) prof_begin(BMG_PROF_FINE_SMOOTH, s);
    if (h->opt.smoother != BMG_SMOOTH_POINT)
      launch_line_sweep<T>(V, nine, h->opt.smoother, reverse, V.x, V.x2, s);
    else
      launch_sweep<T>(V, nine, reverse, V.x, V.x2, s, level_maps<T>(h, l), zero);
    if (!nine) prof_end(BMG_PROF_FINE_SMOOTH, s);
    std::swap(V.x, V.x2);
  };
  prof_begin(BMG_PROF_CYCLE, s);
  NvtxRange cycle_range("vcycle", top);
  for (int l = top; l >= thr; --l) {
    NvtxRange r("restrict_leg", l);
    const bool nine = l != L - 1;
    if (nine) prof_begin(BMG_PROF_LEVELS, s);
    for (int k = skip_first && l == top ? 1 : 0; k < nu1; ++k)
      sweep(l, false, k == 0 && (l < top || top_zero));
    if (!rc && rr_fused(nine, sizeof(T) == 8)) {
      launch_resid_restrict<T>(lv[l], nine, lv[l - 1], s);
    } else {
      launch_residual<T>(lv[l], nine, lv[l].x, lv[l].b, lv[l].r, s);
      launch_restrict<T>(lv[l], lv[l].r, lv[l - 1], true, s);
    }
    if (nine) prof_end(BMG_PROF_LEVELS, s);
  }
  {
    NvtxRange r("coarse_cycle", thr - 1);
    launch_coarse_cycle<T>(h, dlev, thr, s);
  }
  for (int l = thr; l <= top; ++l) {
    NvtxRange r("interp_leg", l);
    const bool nine = l != L - 1;
    if (nine) prof_begin(BMG_PROF_LEVELS, s);
    if (interp_oop) {
      launch_interp<T>(lv[l], lv[l - 1].x, rc, s, lv[l].x2);
      std::swap(lv[l].x, lv[l].x2);
    } else {
      launch_interp<T>(lv[l], lv[l - 1].x, rc, s);
    }
    for (int k = 0; k < nu2; ++k) sweep(l, true, false);
    if (nine) prof_end(BMG_PROF_LEVELS, s);
  }
  prof_end(BMG_PROF_CYCLE, s);
}

template void enqueue_vcycle<double>(Hierarchy*, std::vector<LevelV<double>>&,
                                     const LevelV<double>*, int, cudaStream_t, int, bool, bool);
template void enqueue_vcycle<float>(Hierarchy*, std::vector<LevelV<float>>&, const LevelV<float>*,
                                    int, cudaStream_t, int, bool, bool);

// Stop test inside the next cycle's first fine sweep.  The V(nu1, nu2)
// cycle's last fine sweep is a post-smoothing sweep (reverse colour order),
// and the next cycle starts with a pre-smoothing sweep of the same level, so
// that sweep can sum the residual of the iterate it reads
// (launch_sweep_pre_norm).  The solve loop then runs as: stop test of x0
// (separate norm pass), first pre-sweep; WHILE(go) { rest of the cycle, the
// next cycle's first pre-sweep with the residual of the cycle's result, stop
// test }.  On exit the result is the iterate that sweep read; its output is
// dropped.  Applies to FP64 V-cycles with point smoothing whose finest level
// is swept outside the persistent coarse kernel by the prescaled TMA kernel
// or the small tiled one, with nu1 and nu2 >= 1 (environment
// BMG_FUSED_NORM=0 at setup turns it off).
static bool fused_norm_on(const Hierarchy* h) {
  const int L = h->L;
  const SweepMaps<double>* m = level_maps<double>(h, L - 1);
  return h->fused_norm_allowed && h->opt.solver == BMG_SOLVER_VCYCLE && h->opt.precision == BMG_FP64 &&
         h->opt.smoother == BMG_SMOOTH_POINT && h->opt.nu1 >= 1 && h->opt.nu2 >= 1 &&
         h->threshold < L && sweep_norm_partials(h->d.back(), m, h->npartials) > 0;
}

// The finest level's first pre-smoothing sweep of a cycle: plain, or with
// the stop test (the sweep summing the residual, then the stop test on its
// partials; timed as the norm class, not as a fine sweep).
static void fine_presweep(Hierarchy* h, cudaStream_t s, bool with_norm, bool in_graph) {
  LevelV<double>& F = h->d.back();
  const SweepMaps<double>* m = level_maps<double>(h, h->L - 1);
  const bool fusable = sweep_norm_partials(F, m, h->npartials) > 0 &&
                       (!(m && m->pre) || F.x == m->xp || F.x == m->x2p);
  if (with_norm && !fusable) {
    // (not reached while fused_norm_on holds) the same result in two passes
    launch_fine_norm(h, F.x, F.b, 1, 0.0, s, in_graph);
    with_norm = false;
  }
  if (with_norm) {
    prof_begin(BMG_PROF_NORM, s);
    const int n = launch_sweep_pre_norm(F, m, F.x, F.x2, h->partials, h->npartials, s);
    launch_norm_final(h, s, in_graph, n);
    prof_end(BMG_PROF_NORM, s);
  } else {
    prof_begin(BMG_PROF_FINE_SMOOTH, s);
    launch_sweep<double>(F, false, false, F.x, F.x2, s, m);
    prof_end(BMG_PROF_FINE_SMOOTH, s);
  }
  std::swap(F.x, F.x2);
}

static int read_scalars(Hierarchy* h, cudaStream_t s) {
  BMG_CUDA(cudaMemcpyAsync(h->sc_host, h->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
  BMG_CUDA(cudaStreamSynchronize(s));
  return BMG_OK;
}

// Record the solve loop of h as one graph (see Hierarchy::graph).  Recording
// runs on a private stream (the caller's may be the legacy default stream,
// which cannot capture) and executes nothing.
static int build_solve_graph(Hierarchy* h) {
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return BMG_ECUDA;
  const bool fp32 = h->opt.precision == BMG_FP32_REFINE;
  const bool pcg = h->opt.solver == BMG_SOLVER_PCG;
  const bool fused = !pcg && !fp32 && fused_norm_on(h);
  LevelV<double>& F = h->d.back();
  // recording swaps the levels' iterate buffers as the launches would; the
  // roles are put back afterwards (with the fused stop test the solve's
  // result is in the buffer its input was packed into)
  std::vector<std::pair<double*, double*>> roles64;
  std::vector<std::pair<float*, float*>> roles32;
  for (auto& V : h->d) roles64.emplace_back(V.x, V.x2);
  for (auto& V : h->f) roles32.emplace_back(V.x, V.x2);
  // [prologue: first residual and stop test] WHILE(go) { body }
  auto prologue = [&] {
    if (pcg) {
      launch_pcg_init(h, s, true);
      launch_pcg_precond(h, s);
      launch_pcg_rz(h, true, s);
      launch_pcg_p(h, s);
    } else if (fp32) {
      launch_refine_residual(h, 0.0, s, true);
    } else {
      launch_fine_norm(h, F.x, F.b, 1, 0.0, s, true);
      if (fused) fine_presweep(h, s, false, true);
    }
  };
  auto body = [&] {
    if (pcg) {
      // after the stop test the rest of the body only prepares the next
      // direction (x no longer changes), so a last pass is harmless
      launch_pcg_ap(h, s);
      launch_pcg_xr(h, s, true);
      launch_pcg_precond(h, s);
      launch_pcg_rz(h, false, s);
      launch_pcg_p(h, s);
    } else if (fp32) {
      // the refinement residual zeroed the FP32 fine iterate
      enqueue_vcycle<float>(h, h->f, h->dlev32, h->threshold, s, -1, false, true);
      launch_refine_update(h, s);
      launch_refine_residual(h, 0.0, s, true);
    } else if (fused) {
      enqueue_vcycle<double>(h, h->d, h->dlev64, h->threshold, s, -1, true);
      fine_presweep(h, s, true, true);
    } else {
      enqueue_vcycle<double>(h, h->d, h->dlev64, h->threshold, s);
      launch_fine_norm(h, F.x, F.b, 1, 0.0, s, true);
    }
  };
  int rc = BMG_ECUDA;
  do {
    if (cudaGraphCreate(&h->graph, 0) != cudaSuccess) break;
    if (cudaGraphConditionalHandleCreate(&h->cond, h->graph, 0, cudaGraphCondAssignDefault) !=
        cudaSuccess)
      break;
    if (cudaStreamBeginCaptureToGraph(s, h->graph, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed) != cudaSuccess)
      break;
    prologue();
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    if (cudaStreamGetCaptureInfo(s, &st, nullptr, nullptr, &deps, nullptr, &ndeps) != cudaSuccess)
      break;
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
    std::memset(raw, 0, sizeof(raw));
    cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h->cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, h->graph, deps, nullptr, ndeps, &cp) != cudaSuccess) break;
    if (cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                            cudaStreamSetCaptureDependencies) != cudaSuccess)
      break;
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture(s, &g) != cudaSuccess) break;
    cudaGraph_t gbody = cp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(s, gbody, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed) != cudaSuccess)
      break;
    body();
    if (cudaStreamEndCapture(s, &g) != cudaSuccess) break;
    if (cudaGraphInstantiate(&h->gexec, h->graph, 0) != cudaSuccess) break;
    rc = BMG_OK;
  } while (0);
  for (size_t l = 0; l < h->d.size(); ++l) std::tie(h->d[l].x, h->d[l].x2) = roles64[l];
  for (size_t l = 0; l < h->f.size(); ++l) std::tie(h->f[l].x, h->f[l].x2) = roles32[l];
  cudaStreamDestroy(s);
  if (rc != BMG_OK) {
    cudaGetLastError();
    if (h->graph) cudaGraphDestroy(h->graph);
    h->graph = nullptr;
  }
  return rc;
}

static bool graphs_disabled() {
  static const bool off = [] {
    const char* e = std::getenv("BMG_NO_GRAPH");
    return e && e[0] && e[0] != '0';
  }();
  return off;
}

static int solve_impl(Hierarchy* h, const double* b, double* x, double tol, bmg_info* info,
                      cudaStream_t s) {
  if (!h || !b || !x || !(tol > 0.0)) return BMG_EINVAL;
  const double t0 = now_ms();
  const int L = h->L;
  LevelV<double>& F = h->d.back();
  const bool pcg = h->opt.solver == BMG_SOLVER_PCG;
  // the iterate and right-hand side: the fine level's x and b planes, or the
  // conjugate-gradient planes (whose b and x planes then hold r and z)
  double* xk = pcg ? h->pcg_x : F.x;
  double* bk = pcg ? h->pcg_b : F.b;
  launch_pack<double>(b, bk, h->nx, h->ny, F.pitch, s);
  // the V-cycle solver's fine right-hand side is fixed for the whole solve
  if (!pcg && F.PR[PR_B] && h->opt.precision == BMG_FP64) launch_prescale_b<double>(F, s);
  launch_pack<double>(x, xk, h->nx, h->ny, F.pitch, s);
  if (pcg)
    BMG_CUDA(cudaMemsetAsync(h->pcg_p, 0, sizeof(double) * size_t(h->ny + 2) * F.pitch, s));
  Scalars init{};
  init.tol = tol;
  init.max_cycles = h->opt.max_cycles;
  *h->sc_host = init;
  BMG_CUDA(cudaMemcpyAsync(h->sc, h->sc_host, sizeof(Scalars), cudaMemcpyHostToDevice, s));
  launch_fine_norm(h, nullptr, bk, 0, tol, s);
  const bool fp32 = h->opt.precision == BMG_FP32_REFINE;
  int rc = BMG_OK;
  // Graph path: the whole loop in one launch (not while kernel classes are
  // being timed with events, which need the stream path).
  if (!prof_active() && !graphs_disabled()) {
    if (h->graph_state == 0) h->graph_state = build_solve_graph(h) == BMG_OK ? 1 : -1;
    if (h->graph_state == 1) {
      BMG_CUDA(cudaGraphLaunch(h->gexec, s));
      launch_unpack<double>(xk, x, h->nx, h->ny, F.pitch, s);
      if ((rc = read_scalars(h, s))) return rc;
      const Scalars& r = *h->sc_host;
      if (r.bnorm2 == 0.0) {
        BMG_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * size_t(h->nx) * h->ny, s));
        BMG_CUDA(cudaStreamSynchronize(s));
        if (info) *info = bmg_info{0, h->threshold, 0.0, h->setup_ms, now_ms() - t0, h->coarse_ctas};
        return BMG_OK;
      }
      if (info) *info = bmg_info{r.cycles, h->threshold, r.rel, h->setup_ms, now_ms() - t0, h->coarse_ctas};
      if (r.err & DEV_NAN) return BMG_ENAN;
      if (r.err & DEV_TIMEOUT) return BMG_ETIMEOUT;
      if (!(r.rel <= tol)) return BMG_ENOCONV;
      return BMG_OK;
    }
  }
  if (pcg) {
    launch_pcg_init(h, s, false);
    if ((rc = read_scalars(h, s))) return rc;
    if (h->sc_host->bnorm2 == 0.0) {
      BMG_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * size_t(h->nx) * h->ny, s));
      BMG_CUDA(cudaStreamSynchronize(s));
      if (info) *info = bmg_info{0, h->threshold, 0.0, h->setup_ms, now_ms() - t0, h->coarse_ctas};
      return BMG_OK;
    }
    if (h->sc_host->go) {
      launch_pcg_precond(h, s);
      launch_pcg_rz(h, true, s);
      launch_pcg_p(h, s);
      for (;;) {
        launch_pcg_ap(h, s);
        launch_pcg_xr(h, s, false);
        if ((rc = read_scalars(h, s))) return rc;
        if (!h->sc_host->go) break;
        launch_pcg_precond(h, s);
        launch_pcg_rz(h, false, s);
        launch_pcg_p(h, s);
      }
    }
  } else if (!fp32) {
    launch_fine_norm(h, F.x, F.b, 1, tol, s);
    if ((rc = read_scalars(h, s))) return rc;
    if (h->sc_host->bnorm2 == 0.0) {
      BMG_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * size_t(h->nx) * h->ny, s));
      BMG_CUDA(cudaStreamSynchronize(s));
      if (info) *info = bmg_info{0, h->threshold, 0.0, h->setup_ms, now_ms() - t0, h->coarse_ctas};
      return BMG_OK;
    }
    if (fused_norm_on(h)) {
      // the loop of build_solve_graph, step by step
      if (h->sc_host->go) {
        fine_presweep(h, s, false, false);
        while (h->sc_host->go) {
          enqueue_vcycle<double>(h, h->d, h->dlev64, h->threshold, s, -1, true);
          fine_presweep(h, s, true, false);
          if ((rc = read_scalars(h, s))) break;
        }
        // the result is the input of the last sweep
        std::swap(F.x, F.x2);
        if (rc) return rc;
      }
    } else {
      while (h->sc_host->go) {
        enqueue_vcycle<double>(h, h->d, h->dlev64, h->threshold, s);
        launch_fine_norm(h, F.x, F.b, 1, tol, s);
        if ((rc = read_scalars(h, s))) return rc;
      }
    }
  } else {
    if ((rc = read_scalars(h, s))) return rc;
    if (h->sc_host->bnorm2 == 0.0) {
      BMG_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * size_t(h->nx) * h->ny, s));
      BMG_CUDA(cudaStreamSynchronize(s));
      if (info) *info = bmg_info{0, h->threshold, 0.0, h->setup_ms, now_ms() - t0, h->coarse_ctas};
      return BMG_OK;
    }
    for (;;) {
      launch_refine_residual(h, tol, s);
      if ((rc = read_scalars(h, s))) return rc;
      if (!h->sc_host->go) break;
      enqueue_vcycle<float>(h, h->f, h->dlev32, h->threshold, s, -1, false, true);
      launch_refine_update(h, s);
    }
  }
  (void)L;
  launch_unpack<double>(xk, x, h->nx, h->ny, F.pitch, s);
  BMG_CUDA(cudaGetLastError());
  BMG_CUDA(cudaStreamSynchronize(s));
  const Scalars& r = *h->sc_host;
  if (info) *info = bmg_info{r.cycles, h->threshold, r.rel, h->setup_ms, now_ms() - t0, h->coarse_ctas};
  if (r.err & DEV_NAN) return BMG_ENAN;
  if (r.err & DEV_TIMEOUT) return BMG_ETIMEOUT;
  if (!(r.rel <= tol)) return BMG_ENOCONV;
  return BMG_OK;
}

}  // namespace bmg

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

using bmg::Hierarchy;

static Hierarchy* H(bmg_hierarchy* p) { return reinterpret_cast<Hierarchy*>(p); }
static const Hierarchy* H(const bmg_hierarchy* p) { return reinterpret_cast<const Hierarchy*>(p); }

extern "C" {

void bmg_default_options(bmg_options* opt) {
  if (!opt) return;
  opt->nu1 = 2;
  opt->nu2 = 1;
  opt->precision = BMG_FP64;
  opt->interp_residual_term = 0;
  opt->coarse_threshold = -1;
  opt->max_cycles = 200;
  opt->smoother = BMG_SMOOTH_POINT;
  opt->coarse_ctas = -1;
  opt->log_coefficients = 0;
  opt->solver = BMG_SOLVER_VCYCLE;
  opt->aniso_r = 1.0;
  opt->cell_aspect = 1.0;
  for (double& b : opt->bc_beta) b = -1.0;
}

const char* bmg_last_error(void) { return bmg::g_last_error; }

const char* bmg_strerror(int code) {
  switch (code) {
    case BMG_OK: return "success";
    case BMG_EINVAL: return "invalid argument (size, coefficient, option or level)";
    case BMG_ENOMEM: return "device allocation failed";
    case BMG_ECUDA: return "CUDA runtime error";
    case BMG_ENOCONV: return "no convergence within max_cycles";
    case BMG_ENAN: return "residual norm is NaN or Inf";
    case BMG_ETIMEOUT: return "bounded device wait timed out";
    default: return "unknown error";
  }
}

int bmg_setup(const double* k_dev, int nx, int ny, const bmg_options* opt, bmg_stream_t stream,
              bmg_hierarchy** out) {
  if (!out) return BMG_EINVAL;
  Hierarchy* h = nullptr;
  const int rc = bmg::setup_impl(k_dev, nx, ny, opt, reinterpret_cast<cudaStream_t>(stream), &h);
  *out = reinterpret_cast<bmg_hierarchy*>(h);
  return rc;
}

int bmg_solve(bmg_hierarchy* h, const double* b_dev, double* x_dev, double tol, bmg_info* info,
              bmg_stream_t stream) {
  return bmg::solve_impl(H(h), b_dev, x_dev, tol, info, reinterpret_cast<cudaStream_t>(stream));
}

void bmg_destroy(bmg_hierarchy* h) { bmg::free_hierarchy(H(h)); }

int bmg_solve_host(const double* k_host, const double* b_host, double* x_host, int nx, int ny,
                   const bmg_options* opt, double tol, bmg_info* info, bmg_stream_t stream) {
  if (!k_host || !b_host || !x_host) return BMG_EINVAL;
  if (!bmg::valid_side(nx) || !bmg::valid_side(ny)) return BMG_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t bytes = sizeof(double) * size_t(nx) * ny;
  double* buf = nullptr;
  if (cudaMalloc(&buf, 3 * bytes) != cudaSuccess) {
    cudaGetLastError();
    return BMG_ENOMEM;
  }
  double *k = buf, *b = buf + size_t(nx) * ny, *x = buf + 2 * size_t(nx) * ny;
  int rc = BMG_OK;
  bmg_hierarchy* h = nullptr;
  if (cudaMemcpyAsync(k, k_host, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(b, b_host, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(x, x_host, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) {
    rc = BMG_ECUDA;
  }
  if (rc == BMG_OK) rc = bmg_setup(k, nx, ny, opt, stream, &h);
  double setup_ms = 0.0;
  if (rc == BMG_OK) {
    setup_ms = H(h)->setup_ms;
    rc = bmg_solve(h, b, x, tol, info, stream);
    if (rc == BMG_OK || rc == BMG_ENOCONV) {
      if (cudaMemcpyAsync(x_host, x, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        rc = BMG_ECUDA;
    }
  }
  if (info) info->setup_ms = setup_ms;
  bmg_destroy(h);
  cudaFree(buf);
  return rc;
}

int bmg_set_max_cycles(bmg_hierarchy* hp, int max_cycles) {
  Hierarchy* h = H(hp);
  if (!h || max_cycles < 0) return BMG_EINVAL;
  h->opt.max_cycles = max_cycles;
  return BMG_OK;
}

int bmg_residual_history(const bmg_hierarchy* hp, double* host_out, int capacity, int* n) {
  const Hierarchy* h = H(hp);
  if (!h || !n || (capacity > 0 && !host_out)) return BMG_EINVAL;
  if (cudaMemcpy(h->sc_host, h->sc, sizeof(bmg::Scalars), cudaMemcpyDeviceToHost) != cudaSuccess)
    return BMG_ECUDA;
  const int count = std::min(h->sc_host->cycles + 1, BMG_MAX_HISTORY);
  *n = count;
  const int m = std::min(count, capacity);
  if (m > 0 && cudaMemcpy(host_out, h->hist, sizeof(double) * m, cudaMemcpyDeviceToHost) != cudaSuccess)
    return BMG_ECUDA;
  return BMG_OK;
}

int bmg_num_levels(const bmg_hierarchy* h, int* nlevels) {
  if (!h || !nlevels) return BMG_EINVAL;
  *nlevels = H(h)->L;
  return BMG_OK;
}

int bmg_level_prescaled(const bmg_hierarchy* hp, int level, int* out) {
  const Hierarchy* h = H(hp);
  if (!h || !out || level < 0 || level >= h->L) return BMG_EINVAL;
  const int first = h->L - int(h->d.size());      // h->d holds levels first .. L-1
  *out = level >= first && h->d[level - first].PR[bmg::PR_B] != nullptr ? 1 : 0;
  return BMG_OK;
}

int bmg_level_shape(const bmg_hierarchy* h, int level, int* nx, int* ny) {
  if (!h || !nx || !ny || level < 0 || level >= H(h)->L) return BMG_EINVAL;
  *nx = H(h)->geo64[level].nx;
  *ny = H(h)->geo64[level].ny;
  return BMG_OK;
}

}  // extern "C"

namespace bmg {

// Copy the interior of a device plane to a dense host array (as double).
template <typename T>
static int plane_to_host(const T* plane, int nx, int ny, int pitch, double* out) {
  if (!plane) {
    std::memset(out, 0, sizeof(double) * size_t(nx) * ny);
    return BMG_OK;
  }
  std::vector<T> tmp(size_t(ny + 2) * pitch);
  BMG_CUDA(cudaMemcpy(tmp.data(), plane, sizeof(T) * tmp.size(), cudaMemcpyDeviceToHost));
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) out[size_t(j) * nx + i] = double(tmp[size_t(j + 1) * pitch + i + 1]);
  return BMG_OK;
}

template <typename T>
static int plane_block_to_host(const T* plane, int nx1, int ny1, int pitch, double* out) {
  // entries (I, J), 0 <= I < nx1, 0 <= J < ny1 of a coarse-grid plane
  std::vector<T> tmp(size_t(ny1 + 1) * pitch);
  BMG_CUDA(cudaMemcpy(tmp.data(), plane, sizeof(T) * tmp.size(), cudaMemcpyDeviceToHost));
  for (int J = 0; J < ny1; ++J)
    for (int I = 0; I < nx1; ++I) out[size_t(J) * nx1 + I] = double(tmp[size_t(J) * pitch + I]);
  return BMG_OK;
}

template <typename T>
static int stencil_out(const LevelV<T>& L, double* out) {
  const size_t n = size_t(L.nx) * L.ny;
  int rc;
  if ((rc = plane_to_host<T>(L.C, L.nx, L.ny, L.pitch, out))) return rc;
  if ((rc = plane_to_host<T>(L.W, L.nx, L.ny, L.pitch, out + n))) return rc;
  if ((rc = plane_to_host<T>(L.S, L.nx, L.ny, L.pitch, out + 2 * n))) return rc;
  if ((rc = plane_to_host<T>(L.SW, L.nx, L.ny, L.pitch, out + 3 * n))) return rc;
  return plane_to_host<T>(L.NW, L.nx, L.ny, L.pitch, out + 4 * n);
}

template <typename T>
static int interp_out(const LevelV<T>& L, const LevelV<T>& Lc, double* out) {
  const int nx1 = Lc.nx + 1, ny1 = Lc.ny + 1;
  for (int k = 0; k < NPW; ++k) {
    int rc = plane_block_to_host<T>(L.P[k], nx1, ny1, L.cpitch, out + size_t(k) * nx1 * ny1);
    if (rc) return rc;
  }
  return BMG_OK;
}

}  // namespace bmg

extern "C" {

int bmg_level_stencil(const bmg_hierarchy* hp, int level, double* host_out) {
  const Hierarchy* h = H(hp);
  if (!h || !host_out || level < 0 || level >= h->L) return BMG_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return BMG_ECUDA;
  if (h->opt.precision == BMG_FP32_REFINE) return bmg::stencil_out<float>(h->f[level], host_out);
  return bmg::stencil_out<double>(h->d[level], host_out);
}

int bmg_level_interp(const bmg_hierarchy* hp, int level, double* host_out) {
  const Hierarchy* h = H(hp);
  if (!h || !host_out || level < 1 || level >= h->L) return BMG_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return BMG_ECUDA;
  if (h->opt.precision == BMG_FP32_REFINE)
    return bmg::interp_out<float>(h->f[level], h->f[level - 1], host_out);
  return bmg::interp_out<double>(h->d[level], h->d[level - 1], host_out);
}

int bmg_selftest_bounded_wait(bmg_stream_t stream) {
  return bmg::selftest_bounded_wait(reinterpret_cast<cudaStream_t>(stream));
}

int bmg_coarse_factor(const bmg_hierarchy* hp, double* host_out, int n0_capacity) {
  const Hierarchy* h = H(hp);
  if (!h || !host_out || n0_capacity < h->n0) return BMG_EINVAL;
  if (cudaMemcpy(host_out, h->chol, sizeof(double) * size_t(h->n0) * h->n0,
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return BMG_ECUDA;
  return BMG_OK;
}

static int op_check(bmg_hierarchy* hp, int level, int lo) {
  Hierarchy* h = H(hp);
  if (!h || level < lo || level >= h->L) return BMG_EINVAL;
  if (h->opt.precision != BMG_FP64) return BMG_EINVAL;
  return BMG_OK;
}

int bmg_op_relax(bmg_hierarchy* hp, int level, double* x, const double* b, int nu, int reverse,
                 bmg_stream_t stream) {
  int rc = op_check(hp, level, 0);
  if (rc) return rc;
  if (!x || !b || nu < 0) return BMG_EINVAL;
  Hierarchy* h = H(hp);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  auto& L = h->d[level];
  bmg::launch_pack<double>(x, L.x, L.nx, L.ny, L.pitch, s);
  bmg::launch_pack<double>(b, L.b, L.nx, L.ny, L.pitch, s);
  if (L.PR[bmg::PR_B]) bmg::launch_prescale_b<double>(L, s);
  const bool fine = level == h->L - 1;
  for (int k = 0; k < nu; ++k) {
    if (h->opt.smoother != BMG_SMOOTH_POINT)
      bmg::launch_line_sweep<double>(L, !fine, h->opt.smoother, reverse != 0, L.x, L.x2, s);
    else
      bmg::launch_sweep<double>(L, !fine, reverse != 0, L.x, L.x2, s,
                                bmg::level_maps<double>(h, level));
    std::swap(L.x, L.x2);
  }
  bmg::launch_unpack<double>(L.x, x, L.nx, L.ny, L.pitch, s);
  // keep the level's buffer roles as the recorded solve graph expects them
  if (nu & 1) std::swap(L.x, L.x2);
  return cudaGetLastError() == cudaSuccess ? BMG_OK : BMG_ECUDA;
}

int bmg_op_residual(bmg_hierarchy* hp, int level, const double* x, const double* b, double* r,
                    bmg_stream_t stream) {
  int rc = op_check(hp, level, 0);
  if (rc) return rc;
  if (!x || !b || !r) return BMG_EINVAL;
  Hierarchy* h = H(hp);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  auto& L = h->d[level];
  bmg::launch_pack<double>(x, L.x, L.nx, L.ny, L.pitch, s);
  bmg::launch_pack<double>(b, L.b, L.nx, L.ny, L.pitch, s);
  bmg::launch_residual<double>(L, level != h->L - 1, L.x, L.b, L.r, s);
  bmg::launch_unpack<double>(L.r, r, L.nx, L.ny, L.pitch, s);
  return cudaGetLastError() == cudaSuccess ? BMG_OK : BMG_ECUDA;
}

int bmg_op_restrict(bmg_hierarchy* hp, int level, const double* r, double* bc,
                    bmg_stream_t stream) {
  int rc = op_check(hp, level, 1);
  if (rc) return rc;
  if (!r || !bc) return BMG_EINVAL;
  Hierarchy* h = H(hp);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  auto& L = h->d[level];
  auto& Lc = h->d[level - 1];
  bmg::launch_pack<double>(r, L.r, L.nx, L.ny, L.pitch, s);
  bmg::launch_restrict<double>(L, L.r, Lc, false, s);
  bmg::launch_unpack<double>(Lc.b, bc, Lc.nx, Lc.ny, Lc.pitch, s);
  return cudaGetLastError() == cudaSuccess ? BMG_OK : BMG_ECUDA;
}

int bmg_op_interp(bmg_hierarchy* hp, int level, const double* xc, double* x,
                  bmg_stream_t stream) {
  int rc = op_check(hp, level, 1);
  if (rc) return rc;
  if (!xc || !x) return BMG_EINVAL;
  Hierarchy* h = H(hp);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  auto& L = h->d[level];
  auto& Lc = h->d[level - 1];
  bmg::launch_pack<double>(xc, Lc.x, Lc.nx, Lc.ny, Lc.pitch, s);
  bmg::launch_pack<double>(x, L.x, L.nx, L.ny, L.pitch, s);
  bmg::launch_interp<double>(L, Lc.x, false, s);
  bmg::launch_unpack<double>(L.x, x, L.nx, L.ny, L.pitch, s);
  return cudaGetLastError() == cudaSuccess ? BMG_OK : BMG_ECUDA;
}

int bmg_op_vcycle_from(bmg_hierarchy* hp, int level, const double* b, double* x, bmg_stream_t stream) {
  int rc = op_check(hp, level, 0);
  if (rc) return rc;
  if (!b || !x) return BMG_EINVAL;
  Hierarchy* h = H(hp);
  if (h->opt.smoother != BMG_SMOOTH_POINT) {
    bmg::set_last_error("bmg_op_vcycle_from: point smoother hierarchies only");
    return BMG_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  auto& L = h->d[level];
  bmg::launch_pack<double>(b, L.b, L.nx, L.ny, L.pitch, s);
  if (L.PR[bmg::PR_B]) bmg::launch_prescale_b<double>(L, s);
  if (cudaMemsetAsync(L.x - bmg::base_shift<double>(), 0, h->geo64[level].elems * sizeof(double), s) !=
      cudaSuccess)
    return BMG_ECUDA;
  bmg::enqueue_vcycle<double>(h, h->d, h->dlev64, h->threshold, s, level);
  bmg::launch_unpack<double>(L.x, x, L.nx, L.ny, L.pitch, s);
  return cudaGetLastError() == cudaSuccess ? BMG_OK : BMG_ECUDA;
}

int bmg_assemble_backward(bmg_hierarchy* hp, const double* u, const double* lam, double* dtheta,
                          bmg_stream_t stream) {
  Hierarchy* h = H(hp);
  if (!h || !u || !lam || !dtheta) return BMG_EINVAL;
  if (h->opt.aniso_r != 1.0 || h->opt.cell_aspect != 1.0) return BMG_EINVAL;
  for (double b : h->opt.bc_beta)
    if (b >= 0.0) return BMG_EINVAL;
  bmg::launch_assemble_backward(h->kcopy, u, lam, dtheta, h->nx, h->ny,
                                reinterpret_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? BMG_OK : BMG_ECUDA;
}

}  // extern "C"
