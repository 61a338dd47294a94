/*
 * boxmg.h -- C ABI of the GB300 BoxMG library (2D heterogeneous diffusion).
 *
 * Method: Reisner, Olson, Moulton, "Scaling Structured Multigrid to 500K+
 * Cores through Coarse-Grid Redistribution".  The library implements
 *   - the 5-point cell-centred finite-volume operator of Eq. (diffusion) with
 *     the Dirichlet condition of Eq. (diffusion_bc) (Section 5);
 *   - BoxMG setup (Section 2): operator-induced interpolation P_l, the
 *     Galerkin coarse operators A_{l-1} = P_l^T A_l P_l, and the Cholesky
 *     factor of the coarsest operator (Section 3, coarse-solve cost model);
 *   - the V-cycle of Algorithm 1 with multicolour Gauss-Seidel, residual,
 *     restriction R = P^T and interpolate-and-correct;
 *   - the coarse-grid redistribution of Section 2.2 / Algorithm 2 re-read for
 *     one GPU: every level below a threshold runs inside one persistent
 *     thread block, or one thread-block cluster, instead of one kernel launch
 *     per operation; a cost model in the spirit of Section 3 (Eq. (Vmodel))
 *     with measured parameters picks the threshold and the number of blocks.
 *
 * Conventions (all entry points):
 *   - Grid arrays passed in or out are dense, row-major, shape (ny, nx):
 *     element (i, j), 0 <= i < nx (x, fast), 0 <= j < ny, at offset j*nx + i.
 *   - "_dev" pointers are CUDA device pointers owned by the caller; "_host"
 *     pointers are host memory owned by the caller.  The library never frees
 *     caller memory.  Coefficients are copied into the hierarchy, so the
 *     caller may free or reuse k after bmg_setup returns (stream-ordered).
 *   - Every call is ordered on the given stream (NULL = legacy default
 *     stream).  A call that returns data to a host pointer synchronises the
 *     stream before returning.
 *   - Return value: BMG_OK (0) or a negative BMG_E* code; no call aborts, and
 *     no call falls back to the CPU.  bmg_strerror() gives a message.
 *   - Sizes: nx, ny >= 2.  Coarse point I is fine point 2I (1-based), so a
 *     side of n points coarsens to floor(n / 2) ((n - 1) / 2 for the 2^m - 1
 *     sides, which keep every level of that form; on an even side the last
 *     fine point is a coarse point).  Levels are coarsened while the smaller
 *     side exceeds 3; the coarsest level must have at most BMG_MAX_COARSEST
 *     unknowns.  Batched problems (bmg_batch_*) keep sides 2^m - 1.
 */
#ifndef BOXMG_H
#define BOXMG_H

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; declared here so the header needs no CUDA. */
typedef struct CUstream_st *bmg_stream_t;

typedef struct bmg_hierarchy bmg_hierarchy; /* opaque, library-owned */

enum {
  BMG_OK = 0,
  BMG_EINVAL = -1,   /* bad argument: size, NaN/Inf or non-positive k, level */
  BMG_ENOMEM = -2,   /* device allocation failed                            */
  BMG_ECUDA = -3,    /* a CUDA runtime call failed                          */
  BMG_ENOCONV = -4,  /* max_cycles reached before the tolerance             */
  BMG_ENAN = -5,     /* the residual norm became NaN or Inf                 */
  BMG_ETIMEOUT = -6  /* a bounded device-side wait gave up                  */
};

enum { BMG_FP64 = 0, BMG_FP32_REFINE = 1 };

/* Solvers: the V-cycle iteration of Algorithm 1, or conjugate gradients
 * preconditioned by one symmetric V(nu, nu) cycle (an extension: the paper
 * iterates V-cycles).  BMG_SOLVER_PCG needs nu1 == nu2 >= 1 and
 * interp_residual_term == 0, which make the cycle a symmetric positive
 * definite preconditioner.  The CG recurrences are FP64; with precision
 * BMG_FP32_REFINE the cycle runs on the FP32 hierarchy (r / ||r|| cast down,
 * ||r|| e cast back), which can cost iterations on high-contrast fields. */
enum { BMG_SOLVER_VCYCLE = 0, BMG_SOLVER_PCG = 1 };

/* Smoothers: multicolour point Gauss-Seidel (red-black on the 5-point finest
 * level, four colours on the 9-point levels; the paper's smoother), or zebra
 * line Gauss-Seidel along x (every row solved exactly, odd rows first), along
 * y (the columns), or alternating (x-lines then y-lines) -- Section 2's
 * alternating line smoothing for anisotropic problems.  Line smoothers run on
 * every level; post-smoothing takes the steps in reverse order, so with
 * nu1 == nu2 the cycle stays symmetric. */
enum { BMG_SMOOTH_POINT = 0, BMG_SMOOTH_XLINE = 1, BMG_SMOOTH_YLINE = 2, BMG_SMOOTH_ALTLINE = 3 };

#define BMG_MAX_COARSEST 1024

typedef struct {
  int nu1;                  /* pre-smoothing sweeps (Algorithm 1), default 2  */
  int nu2;                  /* post-smoothing sweeps, default 1               */
  int precision;            /* BMG_FP64 or BMG_FP32_REFINE                    */
  int interp_residual_term; /* 1: add r/C at non-coarse points when
                               interpolating (Section 3, interpolation
                               equations); 0: x += P x_c (Algorithm 1)       */
  int coarse_threshold;     /* levels l < threshold run inside the persistent
                               coarse kernel (1 <= threshold <= L); -1: chosen
                               by the cost model                              */
  int max_cycles;           /* cap on V-cycles (or refinement steps), 200    */
  int log_coefficients;     /* 1: the coefficient array holds theta = log k and
                               the assembly uses k = exp(theta) (adjoint
                               gradients with respect to theta); 0: holds k */
  int solver;               /* BMG_SOLVER_VCYCLE (default) or BMG_SOLVER_PCG  */
  double aniso_r;           /* diffusion tensor D = diag(k / r, k r) per cell
                               (Section 5 uses r ~ 16); 1: isotropic (default) */
  double cell_aspect;       /* cell aspect hy / hx (nx x ny cells of the unit
                               square: nx / ny); 1: square cells (default)    */
  double bc_beta[4];        /* boundary condition of the west, east, south and
                               north wall: < 0 (default -1): u = 0; >= 0: the
                               Robin condition k du/dn + alpha u = 0 with
                               beta = alpha times the cell width normal to
                               that wall (0: Neumann, no flux).  Not all four
                               may be Neumann (the operator would be singular) */
  int smoother;             /* BMG_SMOOTH_* (default BMG_SMOOTH_POINT); line
                               smoothers are not available to the batched
                               solver                                         */
  int coarse_ctas;          /* thread blocks that run the levels below the
                               threshold: 1 = one block; 2..16 = one
                               thread-block cluster of that many blocks, the
                               phases separated by the hardware cluster
                               barrier (point smoother only; sizes above 8
                               need the device's non-portable cluster
                               support); -1 (default) = chosen by the cost
                               model together with the threshold            */
} bmg_options;

typedef struct {
  int cycles;        /* V-cycles run (FP32_REFINE: refinement steps)          */
  int threshold;     /* level threshold used by the schedule                  */
  double rel_resid;  /* final ||b - A x||_2 / ||b||_2, computed in FP64       */
  double setup_ms;   /* wall time of bmg_setup                                 */
  double solve_ms;   /* wall time of the last bmg_solve                        */
  int coarse_ctas;   /* thread blocks running the levels below the threshold  */
} bmg_info;

/* Fill *opt with the defaults above. */
void bmg_default_options(bmg_options *opt);

/* Message for a BMG_* code (static storage). */
const char *bmg_strerror(int code);

/* Details of the last failed call made by this thread (which device check
 * fired, on which level), or "" (thread-local storage, valid until the next
 * call). */
const char *bmg_last_error(void);

/* BoxMG setup (Section 2; Section 5 discretisation).
 * k_dev: cell coefficients k > 0 (or theta = log k when
 * opt->log_coefficients), dense (ny, nx) float64, device.
 * Assembles the fine 5-point operator (harmonic face means, 2k on Dirichlet
 * faces, scaled by h^2; with opt->aniso_r and opt->cell_aspect, x faces carry
 * the harmonic mean of k / r times hy / hx and y faces that of k r times
 * hx / hy, boundary faces 2 (k / r) hy / hx and 2 k r hx / hy, times
 * beta / (2 k_n + beta) on a wall with Robin coefficient beta, k_n = k / r
 * or k r the coefficient normal to it), builds P_l
 * and A_{l-1} = P_l^T A_l P_l on every
 * level, factors A_0, and fixes the level schedule.  With precision
 * BMG_FP32_REFINE the coarse hierarchy (P and RAP) is built in FP32 from an
 * FP32 copy of the fine operator; the FP64 fine operator is kept for the
 * outer residual.  On success *out owns all device memory of the hierarchy.
 * Errors: BMG_EINVAL (sizes, NaN/Inf or k <= 0 found on the device, options),
 * BMG_ENOMEM, BMG_ECUDA.  *out is NULL on error. */
int bmg_setup(const double *k_dev, int nx, int ny, const bmg_options *opt,
              bmg_stream_t stream, bmg_hierarchy **out);

/* Solve A x = b with V-cycles (Algorithm 1) until
 * ||b - A x||_2 / ||b||_2 <= tol (checked before the first cycle and after
 * every cycle) or max_cycles cycles ran.  With solver BMG_SOLVER_PCG: with
 * preconditioned conjugate gradients (r = b - A x, z = M^{-1} r, p = z; per
 * iteration q = A p, alpha = r.z / p.q, x += alpha p, r -= alpha q, stop
 * test on the updated r, z = M^{-1} r, beta = r.z' / r.z, p = z + beta p;
 * M^{-1} is one V(nu, nu) cycle from zero), max_cycles capping the
 * iterations and info->cycles counting them.
 * FP64 V-cycles with point smoothing on a prescaled finest level (nx >= 1024)
 * take the residual after a cycle inside the next cycle's first fine sweep:
 * after the cycle's last sweep one colour satisfies its equation exactly, so
 * that sweep's second colour phase sees the whole residual, evaluated as
 * C (b/C + sum (a/C) x_nb - x) with the level's prescaled coefficients.  The
 * output of that sweep is dropped when the loop stops (one extra sweep per
 * solve); the iterate is the same bits as without it.
 * b_dev: dense (ny, nx) float64, device.  x_dev: dense (ny, nx) float64,
 * device; on entry the initial guess, on exit the solution.  info may be
 * NULL.  Synchronises the stream (the cycle count and residual return to the
 * host).  Errors: BMG_ENOCONV (x holds the last iterate), BMG_ENAN,
 * BMG_ETIMEOUT, BMG_ECUDA, BMG_EINVAL (tol <= 0 or NULL pointers). */
int bmg_solve(bmg_hierarchy *h, const double *b_dev, double *x_dev, double tol,
              bmg_info *info, bmg_stream_t stream);

/* Relative residuals of the last bmg_solve: entry 0 before the first cycle,
 * entry c after cycle c (at most BMG_MAX_HISTORY entries are kept).  Copies
 * min(n, capacity) values to host_out and stores the count in *n. */
#define BMG_MAX_HISTORY 4096
int bmg_residual_history(const bmg_hierarchy *h, double *host_out, int capacity, int *n);

/* Change the cycle cap of later bmg_solve calls on h (>= 0). */
int bmg_set_max_cycles(bmg_hierarchy *h, int max_cycles);

/* End-to-end convenience: copy k and b from pinned (or pageable) host memory,
 * set up, solve, and copy x back, all on `stream`.  Equivalent to
 * bmg_setup + bmg_solve + bmg_destroy with device buffers the call allocates
 * and frees.  x_host holds the initial guess on entry. */
int bmg_solve_host(const double *k_host, const double *b_host, double *x_host,
                   int nx, int ny, const bmg_options *opt, double tol,
                   bmg_info *info, bmg_stream_t stream);

/* Release every device resource of the hierarchy (NULL is allowed). */
void bmg_destroy(bmg_hierarchy *h);

/* ---- Introspection (parity checks against the CPU oracle) ---------------- */

/* Number of levels L; level L-1 is the finest, level 0 the coarsest. */
int bmg_num_levels(const bmg_hierarchy *h, int *nlevels);

/* Grid size of a level. */
int bmg_level_shape(const bmg_hierarchy *h, int level, int *nx, int *ny);
/* *out = 1 when the red-black sweep of level `level` runs on the prescaled
 * operator (the 5-point FP64 finest level swept by the TMA-staged kernel:
 * b/C and the couplings divided by C stored beside the operator, four fused
 * multiply-adds per point update; the same Gauss-Seidel step with different
 * rounding), else 0. */
int bmg_level_prescaled(const bmg_hierarchy *h, int level, int *out);

/* A_level as five dense (ny, nx) float64 planes, concatenated, in host
 * memory: C, W, S, SW, NW, where W(i,j) = -A[(i,j),(i-1,j)],
 * S(i,j) = -A[(i,j),(i,j-1)], SW(i,j) = -A[(i,j),(i-1,j-1)],
 * NW(i,j) = -A[(i,j),(i-1,j+1)]; E, N, NE, SE follow by symmetry.  The
 * finest level has SW = NW = 0.  FP32 hierarchies are widened to float64.
 * host_out holds 5*nx*ny doubles. */
int bmg_level_stencil(const bmg_hierarchy *h, int level, double *host_out);

/* Interpolation weights of P_level (coarse level-1 -> level), 1 <= level,
 * as eight dense (ncy+1, ncx+1) float64 planes in host memory, ncx, ncy the
 * coarse sizes.  Plane entry (I, J), 0 <= I <= ncx, 0 <= J <= ncy, with
 * 1-based fine indices:
 *   0 xw, 1 xe : x-edge point (2I+1, 2J) -> coarse (I, J), (I+1, J)
 *   2 ys, 3 yn : y-edge point (2I, 2J+1) -> coarse (I, J), (I, J+1)
 *   4 csw, 5 cse, 6 cnw, 7 cne : centre point (2I+1, 2J+1) -> coarse
 *                (I, J), (I+1, J), (I, J+1), (I+1, J+1)
 * Entries that name no fine point (xw at J = 0, ys at I = 0) are 0.
 * host_out holds 8*(ncx+1)*(ncy+1) doubles. */
int bmg_level_interp(const bmg_hierarchy *h, int level, double *host_out);

/* Lower-triangular Cholesky factor of the coarsest operator A_0, dense
 * N0 x N0 row-major float64 in host memory (N0 = nx0 * ny0, unknown index
 * j*nx0 + i). */
int bmg_coarse_factor(const bmg_hierarchy *h, double *host_out, int n0_capacity);

/* ---- Single operations on one level (for per-kernel parity and timing) -- */
/* Each takes dense (ny, nx) float64 device arrays of that level and runs the
 * same device code as the V-cycle on them.  FP64 hierarchies only. */

/* nu multicolour Gauss-Seidel sweeps on level `level`, in place on x_dev
 * (Section 3 smoothing; colours forward, or reversed if reverse != 0). */
int bmg_op_relax(bmg_hierarchy *h, int level, double *x_dev, const double *b_dev,
                 int nu, int reverse, bmg_stream_t stream);

/* r = b - A_level x (Algorithm 1). */
int bmg_op_residual(bmg_hierarchy *h, int level, const double *x_dev,
                    const double *b_dev, double *r_dev, bmg_stream_t stream);

/* bc = P_level^T r  (r on level `level`, bc on level-1; Algorithm 1). */
int bmg_op_restrict(bmg_hierarchy *h, int level, const double *r_dev,
                    double *bc_dev, bmg_stream_t stream);

/* x += P_level xc  (xc on level-1, x on level `level`; Algorithm 1). */
int bmg_op_interp(bmg_hierarchy *h, int level, const double *xc_dev,
                  double *x_dev, bmg_stream_t stream);

/* ---- Adjoint gradient (extension: differentiation) ---------------------- */

/* dtheta_c = -d(lam^T A(theta) u)/d theta_c for k = exp(theta), the
 * backward of the Section 5 assembly contracted with the state u and the
 * adjoint lam (both dense (ny, nx) float64, device):
 *   dtheta_c = -k_c [ sum_{faces f of c} dA_f/dk_c (u_c - u_n)(lam_c - lam_n)
 *                     + sum_{boundary faces} 2 u_c lam_c ],
 *   dA_f/dk_c = 2 k_n^2 / (k_c + k_n)^2.
 * With lam solving A lam = u - u_obs this is dL/dtheta for
 * L = 0.5 ||u - u_obs||^2.  Uses the k given to bmg_setup.  Isotropic square
 * cells with u = 0 on every wall only (aniso_r = cell_aspect = 1, all
 * bc_beta < 0; else BMG_EINVAL). */
int bmg_assemble_backward(bmg_hierarchy *h, const double *u_dev,
                          const double *lam_dev, double *dtheta_dev,
                          bmg_stream_t stream);

/* ---- Level schedule (single-GPU reading of Section 2.2 / Algorithm 2) ----- */

/* Measure the cost-model parameters on the current device (the analogue of
 * the Section 3 machine parameters alpha, beta, gamma) and use them for every
 * later threshold choice in this process.  params_out (may be NULL) receives
 * 10 doubles: launch latency [us], in-block barrier phase [us], streaming
 * bandwidth [GB/s], FP64 and FP32 FMA rates of the whole GPU [GFLOP/s],
 * one-block L2 bandwidth [GB/s], one-block FP64 and FP32 rates [GFLOP/s],
 * cluster-barrier phase [us] and the cluster size it was measured with (the
 * largest the coarse kernel can use; 1 and the default phase time when the
 * device has no thread-block clusters).
 * Allocates and frees 1 GiB of scratch; synchronises the stream. */
int bmg_calibrate(bmg_stream_t stream, double *params_out);

/* Largest value bmg_options.coarse_ctas may take on the current device for
 * the given precision (BMG_FP64 or BMG_FP32_REFINE): the largest thread-block
 * cluster (a power of two <= 16) the cluster coarse kernel can be launched
 * with, 1 when the device has no thread-block clusters.  No device work
 * besides attribute queries. */
int bmg_max_coarse_ctas(int precision, int *out);

/* Model-predicted time [us] of one V-cycle of h with the given threshold
 * (levels l < threshold inside the persistent kernel, run by as many blocks
 * as h uses, see bmg_info.coarse_ctas). */
int bmg_predict_cycle_us(const bmg_hierarchy *h, int threshold, double *us);

/* ---- Batched solves (many independent problems) -------------------------- */

typedef struct bmg_batch bmg_batch; /* opaque, library-owned */

/* Set up nprob independent square problems at once: problem p has side n[p]
 * (2^m - 1) and coefficients k_dev[p] (dense n[p] x n[p] float64, device).
 * k_dev and n are host arrays.  Each problem is solved with FP32 V-cycles
 * (Algorithm 1) inside FP64 iterative refinement (opt->precision is ignored),
 * or, with opt->solver BMG_SOLVER_PCG (nu1 == nu2, no r/C term), with FP64
 * conjugate gradients preconditioned by one symmetric FP32 V(nu, nu) cycle
 * (r / ||r|| cast down, ||r|| e cast back), all problems' iterations
 * advanced together; levels of side <= 31 run in the persistent coarse
 * kernel, one thread block per problem.  Setup also picks the tile shape of the batched sweeps for
 * every level side by timing the candidates on this batch (cached per
 * process, and in the file named by the environment variable BMG_TUNE_CACHE
 * if set) and records the refinement loop as one CUDA graph.  Errors as
 * bmg_setup, naming the failing problem in bmg_last_error. */
int bmg_batch_setup(int nprob, const double *const *k_dev, const int *n,
                    const bmg_options *opt, bmg_stream_t stream, bmg_batch **out);

/* Solve every problem to ||b - A x||_2 / ||b||_2 <= tol with ONE launch of
 * the refinement-loop graph: every V-cycle operation is one launch over all
 * problems that have a level of that side, problems that have converged
 * drop out, and the loop ends when none is left.  b_dev[p], x_dev[p]: host
 * arrays of device pointers to dense n[p] x n[p] float64 arrays (x: initial
 * guess in, solution out).  per_prob (may be NULL) receives nprob bmg_info
 * (cycles = refinement steps of that problem).  Returns BMG_OK, or
 * BMG_ENOCONV / BMG_ENAN if any problem ended that way. */
int bmg_batch_solve(bmg_batch *b, const double *const *b_dev, double *const *x_dev,
                    double tol, bmg_info *per_prob, bmg_stream_t stream);

/* Number of problems of a batch. */
int bmg_batch_size(const bmg_batch *b, int *nprob);

/* Release a batch (NULL is allowed). */
void bmg_batch_destroy(bmg_batch *b);

/* ---- Domain decomposition (Section 2.1) and redistribution (Algorithm 2) --
 *
 * One rank's part of a distributed hierarchy.  The ranks form a px x py
 * processor grid (Section 2.1); on every distributed level a rank owns one
 * rectangular block of points, stored with a one-point ring that holds the
 * neighbours' values (the width-1 halo).  A part holds nlev levels, part
 * level 0 (the gather level of Algorithm 2, vectors only) up to part level
 * nlev - 1 (the finest).  The caller moves ring and block data between ranks
 * (halo exchange, gather_rhs, scatter_sol) with bmg_dd_copy and bmg_dd_block
 * and runs the coarse levels below the gather level on one rank with
 * bmg_op_vcycle_from.  Blocks must start at 0-based global indices that are
 * multiples of 2^(nlev - 1) in both directions, so that local and global
 * point parities (colours, coarse points) agree on every level.  All device
 * work is ordered on the given stream. */

typedef struct bmg_dd_part bmg_dd_part;  /* opaque, library-owned */

enum { BMG_DD_X = 0, BMG_DD_B = 1, BMG_DD_R = 2 };              /* vectors      */
enum { BMG_DD_WEST = 0, BMG_DD_EAST = 1, BMG_DD_SOUTH = 2, BMG_DD_NORTH = 3 };

/* Create one rank's part.  nx[k], ny[k]: owned block size on part level k
 * (>= 1).  nine[k]: 1 if part level k has a 9-point operator, 0 for the
 * 5-point finest level.  stencil_host[k] (k >= 1; entry 0 ignored): host
 * doubles (5, ny[k] + 2, nx[k] + 2), the planes C, W, S, SW, NW (the
 * negated couplings of bmg_level_stencil) of the block and its ring, zero
 * outside the domain.  interp_host[k] (k >= 1): host doubles
 * (8, ny[k-1] + 2, nx[k-1] + 2), the eight interpolation planes of
 * bmg_level_interp (weights stored at coarse points, Section 3) on the
 * coarser block with its ring.  Copies everything; vectors start at zero.
 * Synchronises the stream.  BMG_EINVAL for empty blocks or missing planes. */
int bmg_dd_part_create(int nlev, const int *nx, const int *ny, const int *nine,
                       const double *const *stencil_host,
                       const double *const *interp_host, bmg_stream_t stream,
                       bmg_dd_part **out);

/* Release a part (NULL is allowed). */
void bmg_dd_part_destroy(bmg_dd_part *p);

/* One colour of multicolour Gauss-Seidel on the owned points of part level
 * k >= 1, in place (colour 0..1 red-black on a 5-point level, 0..3 on a
 * 9-point level, in the forward order of the full-level smoother).  The ring
 * of x must hold the neighbours' current values (halo exchange per colour,
 * Algorithm 2). */
int bmg_dd_relax_colour(bmg_dd_part *p, int k, int colour, bmg_stream_t stream);

/* r = b - A x on the owned points of part level k >= 1 (x ring current). */
int bmg_dd_residual(bmg_dd_part *p, int k, bmg_stream_t stream);

/* b = P^T r on the owned points of part level k - 1, x there set to zero
 * (r's ring current; restriction needs no other communication, Section 3). */
int bmg_dd_restrict(bmg_dd_part *p, int k, bmg_stream_t stream);

/* x_k += P x_{k-1} on the owned points of part level k (the coarse x and
 * its ring current). */
int bmg_dd_interp(bmg_dd_part *p, int k, bmg_stream_t stream);

/* out2_host[0] = sum of r^2, out2_host[1] = sum of b^2 over the owned points
 * of part level k >= 1, in a fixed order; synchronises the stream. */
int bmg_dd_norms(bmg_dd_part *p, int k, double *out2_host, bmg_stream_t stream);

/* Halo strips of vector `vec` (BMG_DD_X/B/R) of part level k.  dir 0 (get)
 * copies the owned edge line next to `side` into buf_dev; dir 1 (put) copies
 * buf_dev into the ring line on that side.  West/east lines are columns of
 * ny[k] values (rows 1..ny); south/north lines are rows of nx[k] + 2 values
 * (ring columns included, so a west/east exchange followed by a south/north
 * exchange fills the ring corners).  buf_dev: caller-owned device memory. */
int bmg_dd_copy(bmg_dd_part *p, int k, int vec, int side, int dir, double *buf_dev,
                bmg_stream_t stream);

/* Whole block of `vec` on part level k to (dir 0) or from (dir 1) a dense
 * row-major device array: ring == 0: the owned (ny, nx) points; ring == 1:
 * (ny + 2, nx + 2) including the ring. */
int bmg_dd_block(bmg_dd_part *p, int k, int vec, int dir, int ring, double *dense_dev,
                 bmg_stream_t stream);

/* x = one V-cycle (Algorithm 1, the hierarchy's nu1, nu2, smoother and level
 * schedule) on levels 0..level of h for A_level x = b from x = 0: the cycle
 * the rank holding an agglomerated coarse problem runs (Algorithm 2, after
 * gather_rhs).  b_dev, x_dev: dense (ny, nx) float64 device arrays of that
 * level.  FP64 point-smoother hierarchies; 0 <= level < number of levels. */
int bmg_op_vcycle_from(bmg_hierarchy *h, int level, const double *b_dev, double *x_dev,
                       bmg_stream_t stream);

/* ---- Allocation-free residual check --------------------------------------- */

/* ||b - A(k) x||_2 and ||b||_2 for the 5-point cell-centred operator of k
 * (the operator bmg_setup assembles with aniso_r = cell_aspect = 1 and u = 0
 * on every wall), written
 * to norms_dev[0] and
 * norms_dev[1] (device memory, 2 doubles).  This entry point has no
 * counterpart in the paper: it exists for callers that cannot allocate
 * device memory -- programs whose device memory is all handed out by their
 * own pool, and latency-critical loops that cannot afford the device-wide
 * synchronisation a cudaMalloc/cudaFree pair can cause.  Such callers cannot
 * create a hierarchy, but can check a solution with this call.
 * k_dev, x_dev, b_dev: dense (ny, nx) float64 device arrays, caller-owned.
 * The call allocates nothing: its reduction scratch (one pair of partial sums
 * per grid row) is a static device array of 2 x 16384 doubles (256 KiB) that
 * every GPU loading the library holds until the process exits, so ny may be
 * at most 16384 (BMG_EINVAL beyond, see bmg_last_error).  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) and
 * keeps it for the rest of the process; make that first call before any
 * stream capture, and do not use this call on a device after
 * cudaDeviceReset (the kept address belongs to the context that was torn
 * down).  All calls share the array and
 * each call overwrites every slot it reads, so nothing carries over between
 * calls; calls that overlap on the GPU (different streams, or different
 * threads) race on the array and must be serialised by the caller. */
int bmg_residual_norm_noalloc(const double *k_dev, const double *x_dev,
                              const double *b_dev, int nx, int ny,
                              double *norms_dev, bmg_stream_t stream);

/* Failure-detection self-test (no counterpart in the paper).  The TMA-staged
 * sweeps wait for their bulk copies on mbarriers; every such wait gives up
 * after about one second, records DEV_TIMEOUT in the solve's device error
 * word and lets the kernel return, so a solve ends with BMG_ETIMEOUT instead
 * of hanging the GPU.  This call runs that same bounded wait, in one thread
 * of a one-block kernel, on a barrier phase that expects bytes no copy ever
 * delivers.  Returns BMG_ETIMEOUT after about one second (the expected
 * result), BMG_OK if the wait completed (it cannot), BMG_ENOMEM/BMG_ECUDA on
 * a CUDA error.  Allocates and frees 4 bytes of device memory; synchronises
 * `stream`. */
int bmg_selftest_bounded_wait(bmg_stream_t stream);

/* ---- Observability ------------------------------------------------------ */

/* Total kernel launches this library has issued in this process. */
long long bmg_kernel_launches(void);

/* Kernel classes that can be timed live with CUDA events (class numbers;
 * bit (1 << class) in a mask). */
enum { BMG_PROF_FINE_SMOOTH = 1, BMG_PROF_FINE_RESID = 2, BMG_PROF_FINE_INTERP = 3,
       BMG_PROF_COARSE = 4, BMG_PROF_LEVELS = 5, BMG_PROF_NORM = 6, BMG_PROF_CYCLE = 7,
       BMG_PROF_KRYLOV = 8 };

/* Bracket every launch of each kernel class whose bit is set in `mask` with
 * a pair of CUDA events on its stream (up to 65536 per class) and reset all
 * records; mask 0 stops recording.  Classes: fine-level sweeps (one bracket
 * per full sweep), fine-level residual, fine-level interpolation, the
 * persistent coarse kernel, all other levels' full-grid work of one V-cycle,
 * the convergence norm (where the stop test is taken inside the next
 * cycle's first fine sweep: that sweep and the stop test, which the
 * fine-sweep class then leaves out), one whole V-cycle, and the
 * conjugate-gradient vector
 * kernels of BMG_SOLVER_PCG (A p with p.q, the x/r update with r.r, r.z with
 * the scalars, and p = z + beta p; one bracket per iteration). */
int bmg_profile_set(int mask);

/* Synchronise the recorded events of class `which` and return the number of
 * brackets and their summed device time in milliseconds. */
int bmg_profile_read(int which, int *launches, double *total_ms);

#ifdef __cplusplus
}
#endif
#endif /* BOXMG_H */
