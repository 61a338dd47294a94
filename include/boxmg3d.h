/* C ABI of the 3D BoxMG V-cycle (GB300, sm_103a).
 *
 * The 3D form of the solver in boxmg.h: the 7-point cell-centred finite-volume
 * operator of -div(k grad u) = f with u = 0 on the boundary of the unit cube
 * (Section 5's Eqs. (diffusion), (diffusion_bc) in three dimensions; cubic
 * cells, integrated form divided by h, so b is used as given), operator-induced
 * interpolation (Section 2; the 3D interpolation whose cost Section 3 models),
 * Galerkin coarse operators A_{l-1} = P^T A_l P (27-point), multicolour point
 * Gauss-Seidel (red-black on the 7-point finest level, eight colours on the
 * 27-point levels; post-smoothing in reverse colour order), a dense Cholesky
 * solve on the coarsest level, and V(nu1, nu2) cycles (Algorithm 1) until
 * ||b - A x||_2 / ||b||_2 <= tol.
 *
 * Interpolation weights (the paper gives none; the 2D readings extended): a
 * fine point between coarse points in one direction takes its equation
 * collapsed onto that direction (couplings on each side summed, those within
 * its transverse plane moved to the diagonal); in two directions, its equation
 * collapsed along the third with its edge neighbours replaced by their
 * interpolants; in all three, its full equation with every non-coarse
 * neighbour replaced by its interpolant.  Constant k gives the trilinear
 * weights.  Non-M-matrix rows are lumped first as in 2D.
 *
 * Layout of host/device arrays: (nz, ny, nx) float64, x fastest.  Sides: any
 * nx, ny, nz >= 2; a side of n points coarsens to floor(n / 2) while the
 * smallest side exceeds 3; the coarsest level may hold at most
 * BMG_MAX_COARSEST unknowns.  All calls are stream-ordered on `stream`;
 * device pointers are caller-owned; coefficients are copied into the
 * hierarchy.  Return codes are those of boxmg.h (0 = BMG_OK, negative on
 * failure, bmg_last_error() for details); there is no CPU fallback.
 */
#ifndef BOXMG3D_H
#define BOXMG3D_H

#include "boxmg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bmg3_hierarchy bmg3_hierarchy; /* opaque, library-owned */

/* Setup: assemble, build P_l and A_{l-1} level by level, factor the
 * coarsest operator.  k_dev: (nz, ny, nx) float64 cell coefficients > 0,
 * device.  opt: nu1, nu2, max_cycles and precision are used (BMG_FP64, or
 * BMG_FP32_REFINE: the hierarchy is built in FP64 and also kept as an FP32
 * copy, operator, 1/C and interpolation rounded once, on which each solve
 * step runs one FP32 V-cycle inside FP64 iterative refinement) and solver
 * (BMG_SOLVER_VCYCLE, or BMG_SOLVER_PCG: conjugate gradients on the finest
 * operator in FP64, preconditioned by one symmetric V(nu, nu) cycle from
 * zero, which needs nu1 == nu2; with BMG_FP32_REFINE that cycle runs on the
 * FP32 copies); smoother must be BMG_SMOOTH_POINT and the anisotropy, aspect
 * and wall options their defaults (BMG_EINVAL otherwise); NULL for the
 * defaults.  BMG_EINVAL for bad sizes or non-positive / non-finite k. */
int bmg3_setup(const double *k_dev, int nx, int ny, int nz, const bmg_options *opt,
               bmg_stream_t stream, bmg3_hierarchy **out);

/* V-cycles from the initial guess in x_dev (overwritten) until the relative
 * residual is at most tol, on device arrays of (nz, ny, nx) float64.
 * BMG_FP32_REFINE: each step computes r = b - A x in FP64, runs one FP32
 * V-cycle on A e = r / s from e = 0 (s the previous residual norm, so the
 * FP32 right-hand side is of order one) and updates x += s e in FP64; the
 * stop test is the FP64 relative residual.
 * BMG_SOLVER_PCG: CG iterations in the oracle's textbook order; the stop test
 * uses the recursively updated residual.
 * FP64 V-cycles with nu1, nu2 >= 1 take the residual after a cycle inside the
 * next cycle's first fine sweep (the cycle's last colour is unchanged by it;
 * C (x_new - x_old) at the other colour is the residual), which writes out of
 * place, so the iterate returned is the one the residual belongs to: the same
 * bits as with a separate residual pass (one extra half sweep per solve).
 * info (may be NULL): cycles (refinement steps, or CG iterations) run, final
 * relative residual, solve wall time.  BMG_ENOCONV after max_cycles, BMG_ENAN if the residual is
 * not finite. */
int bmg3_solve(bmg3_hierarchy *h, const double *b_dev, double *x_dev, double tol, bmg_info *info,
               bmg_stream_t stream);

void bmg3_destroy(bmg3_hierarchy *h);

/* Introspection for parity checks (synchronous, host output). */
int bmg3_num_levels(const bmg3_hierarchy *h, int *n);
int bmg3_level_shape(const bmg3_hierarchy *h, int level, int *nx, int *ny, int *nz);
/* 14 planes of nx*ny*nz values of level `level`: the diagonal C, then the
 * negated off-diagonals a_d = -A[p, p + d] for the 13 offsets
 * d = (di, dj, dk) with dk = -1 (di, dj in -1..1, di fastest), then
 * dk = 0, dj = -1 (di in -1..1), then (-1, 0, 0).  The couplings to the other
 * 13 offsets are those of the neighbour (symmetry). */
int bmg3_level_stencil(const bmg3_hierarchy *h, int level, double *host_out);
/* 8 planes of nx*ny*nz values on level `level` (>= 1): the weights of each
 * fine point to its parent coarse points.  Plane m = 4 cz + 2 cy + cx; per
 * direction, a fine point at 1-based index i has the single parent i / 2 when
 * i is even (c = 0) and the parents (i - 1) / 2 (c = 0) and (i + 1) / 2 (c = 1)
 * when i is odd (a parent index 0 or beyond the coarse side lies outside the
 * grid and carries the Dirichlet value 0). */
int bmg3_level_interp(const bmg3_hierarchy *h, int level, double *host_out);

#ifdef __cplusplus
}
#endif

#endif /* BOXMG3D_H */
