"""Plain FP64 CPU oracle of the BoxMG V-cycle for 2D heterogeneous diffusion.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this module.  The library's product
path never calls it, and it shares no code with the CUDA path.

What it computes (Reisner, Olson, Moulton, "Scaling Structured Multigrid to
500K+ Cores through Coarse-Grid Redistribution"):

* ``assemble_fv5``   -- the standard 5-point cell-centred finite-volume
  discretisation of Eq. (diffusion) with the homogeneous Dirichlet condition
  of Eq. (diffusion_bc) (Section 5).  Face coefficients are harmonic means
  2 k1 k2 / (k1 + k2); a boundary face contributes 2 k to the diagonal.  The
  operator is scaled by h^2 (square cells), so the right-hand side b is used
  as given.
* ``interpolation``  -- operator-induced interpolation P (Section 2): weights
  from the operator, stored per fine point, computed by collapsing the fine
  stencil (flux continuity, Dendy's black-box construction).  Coarse point I
  is fine point 2I (1-based); coarsening by 2 (Section 2).
* ``galerkin``       -- the variational coarse operator A_{l-1} = P^T A_l P
  (Section 2), formed literally as a sparse triple product; the result is
  checked to be a 9-point stencil.
* ``cholesky`` / ``cholesky_solve`` -- the coarsest-grid direct solve, with
  the factor computed once in setup (Section 3, Eq. for T_cgsolve).
* ``relax``          -- multicolour point Gauss-Seidel (Section 2, Section 3
  Eq. for T_smooth, Section 5): red-black on the 5-point finest level, four
  colours on 9-point coarse levels.
* ``relax_lines``    -- zebra line Gauss-Seidel, alternating x- and y-lines
  (Section 2 names alternating line smoothing as the smoother anisotropy
  calls for; Section 7 leaves line smoothers to future work): every line of
  one colour is solved exactly, its tridiagonal system built from the
  couplings along the line and a right-hand side holding the current values
  of the neighbouring lines.
* ``residual``, restriction R = P^T, interpolate-and-correct -- Algorithm 1,
  with the optional r/C term of the interpolation equations in Section 3.
* ``vcycle`` / ``solve`` -- Algorithm 1, iterated until the relative residual
  ||b - A x||_2 / ||b||_2 is at most ``tol``.
* ``pcg``            -- conjugate gradients preconditioned by one symmetric
  V(nu, nu) cycle (the V-cycle used as a preconditioner rather than as the
  iteration; the paper solves with V-cycles alone).
* ``assembly_vjp`` / ``adjoint_gradient`` -- the gradient of
  L = 0.5 ||u - u_obs||^2 with respect to log-coefficients through the adjoint
  equation A lambda = u - u_obs (A is symmetric), with exact sparse solves.

Readings where the paper is silent (each is also listed in the design notes):
* interpolation weights: x-edge point w_W = (a_W + a_SW + a_NW) / (C - a_S - a_N)
  (and the mirror for E); y-edge point w_S = (a_S + a_SW + a_SE) / (C - a_W - a_E)
  (and the mirror for N); cell-centre point: the fine equation at the point
  with the four edge neighbours replaced by their interpolants.  Here a_X
  are the negated off-diagonal entries of the fine row.
* rows that are not M-matrix rows (the paper mentions BoxMG heuristics for
  non-zero row sums without stating them): before collapsing, a coupling
  with a_X < 0 (a positive matrix entry) is lumped into the diagonal and a
  negative row sum sigma = C - sum_X a_X is dropped, i.e. the formulas above
  are applied to a_X+ = max(a_X, 0) and C_eff = C - sum_X min(a_X, 0) -
  min(sigma, 0).  On rows with all a_X >= 0 and sigma >= 0 (every row of the
  assembled operator) C_eff = C exactly and nothing changes.  Galerkin
  operators of high-contrast fields develop such rows once the coefficient
  blocks are narrower than a coarse cell; without this the collapse
  denominators turn negative there.
* colour order: red = (i + j) even (1-based), first; four colours
  (i mod 2, j mod 2) in the order (1,1), (0,1), (1,0), (0,0).  Pre-smoothing
  runs the colours forward, post-smoothing in reverse.
* line smoothing: zebra order, the odd lines (1-based) first; a line's
  system is solved exactly (a banded solve).  "x-lines" are the rows (lines
  along x, implicit in the W/E couplings), "y-lines" the columns.  The
  alternating smoother runs x-lines then y-lines; post-smoothing runs the
  reverse (y-lines then x-lines, each with the colours reversed), so the
  V-cycle stays symmetric.  The smoother is used on every level.
* residual norm: the Euclidean norm; the stop test is applied after each
  full cycle (and once before the first).
* sizes: any nx, ny >= 2; a side of n points coarsens to floor(n / 2)
  (coarse point I is fine point 2I), and coarsening stops once the smaller
  side is at most 3.  2^m - 1 sides keep every level of that form.

Data layout: every grid quantity is a float64 array of shape (ny, nx),
``a[j, i]`` with i the x index (fast).  A stencil is a dict of nine planes,
'C' and the eight negated off-diagonals 'W','E','S','N','SW','SE','NW','NE'
(``st['E'][j, i] = -A[(i, j), (i + 1, j)]``), zero where the neighbour lies
outside the domain.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

# direction -> (di, dj) offset of the neighbour in (x, y)
OFFSETS = {
    "W": (-1, 0), "E": (1, 0), "S": (0, -1), "N": (0, 1),
    "SW": (-1, -1), "SE": (1, -1), "NW": (-1, 1), "NE": (1, 1),
}
DIRS = tuple(OFFSETS)


# ---------------------------------------------------------------------------
# Discretisation (Section 5, Eqs. (diffusion), (diffusion_bc))
# ---------------------------------------------------------------------------

def harmonic_face(k1: np.ndarray, k2: np.ndarray) -> np.ndarray:
    """Face coefficient between two square cells: the series conductance of
    two half cells, 2 k1 k2 / (k1 + k2)."""
    return 2.0 * k1 * k2 / (k1 + k2)


def boundary_face(dirichlet: np.ndarray, k_normal: np.ndarray, beta) -> np.ndarray:
    """Coefficient of a boundary face.  ``dirichlet`` is the Dirichlet face
    coefficient (the wall half a cell from the centre: 2 k_n times the face
    length over the cell width) and ``beta`` selects the condition on that
    side: None for u = 0 (Dirichlet, the value as given), or beta >= 0 for
    the Robin condition k du/dn + alpha u = 0 with beta = alpha times the
    cell width normal to the wall: eliminating the wall value gives the
    series conductance dirichlet * beta / (2 k_n + beta); beta = 0 is the
    Neumann condition (no flux)."""
    if beta is None:
        return dirichlet
    return dirichlet * (beta / (2.0 * k_normal + beta))


def assemble_fv5(k: np.ndarray, r: float = 1.0, aspect: float = 1.0, bc=None) -> dict:
    """5-point cell-centred FV operator for -div(D grad u) = f, u = 0 on the
    boundary of the unit square (Section 5, Eqs. (diffusion),
    (diffusion_bc)), in integrated form (for square cells: scaled by h^2).

    D = diag(k / r, k r) per cell (Section 5 uses a constant D with r ~ 16;
    r = 1 is isotropic diffusion with coefficient k), on cells of aspect
    hy / hx = ``aspect`` (nx x ny cells of the unit square: aspect nx / ny).
    Interior x faces carry the harmonic mean of the two cells' k / r times
    hy / hx, y faces that of k r times hx / hy; a boundary face sits half a
    cell from the cell centre and carries 2 (k / r) hy / hx or 2 k r hx / hy.
    The diagonal C is the sum of the cell's four face coefficients.  With
    r = aspect = 1 every factor is an exact 1.  ``bc`` = (west, east, south,
    north), each None (u = 0, the default) or a Robin/Neumann beta (see
    boundary_face); not all four may be Neumann (the operator would be
    singular).
    """
    bc = (None, None, None, None) if bc is None else tuple(bc)
    if len(bc) != 4 or any(b is not None and not (np.isfinite(b) and b >= 0) for b in bc):
        raise ValueError("bc: four entries, each None or a finite beta >= 0")
    if all(b is not None and b == 0 for b in bc):
        raise ValueError("Neumann on every side: the operator is singular")
    k = np.asarray(k, dtype=np.float64)
    ny, nx = k.shape
    inv_r, inv_a = 1.0 / r, 1.0 / aspect
    kx, ky = k * inv_r, k * r
    st = {d: np.zeros((ny, nx)) for d in ("C",) + DIRS}
    ax = harmonic_face(kx[:, :-1], kx[:, 1:]) * aspect     # face between i and i+1
    ay = harmonic_face(ky[:-1, :], ky[1:, :]) * inv_a      # face between j and j+1
    st["E"][:, :-1] = ax
    st["W"][:, 1:] = ax
    st["N"][:-1, :] = ay
    st["S"][1:, :] = ay
    bw = np.zeros((ny, nx))                          # boundary face coefficients
    bw[:, 0] += boundary_face(2.0 * kx[:, 0] * aspect, kx[:, 0], bc[0])
    bw[:, -1] += boundary_face(2.0 * kx[:, -1] * aspect, kx[:, -1], bc[1])
    bw[0, :] += boundary_face(2.0 * ky[0, :] * inv_a, ky[0, :], bc[2])
    bw[-1, :] += boundary_face(2.0 * ky[-1, :] * inv_a, ky[-1, :], bc[3])
    st["C"] = st["W"] + st["E"] + st["S"] + st["N"] + bw
    return st


def shifted(xp: np.ndarray, d: str, ny: int, nx: int,
            rows=slice(None), cols=slice(None)) -> np.ndarray:
    """Neighbour values x[j + dj, i + di] read from the zero-padded array
    ``xp`` (one ghost cell on every side), restricted to rows/cols of the
    unpadded grid."""
    di, dj = OFFSETS[d]
    v = xp[1 + dj:1 + dj + ny, 1 + di:1 + di + nx]
    return v[rows, cols]


def apply(st: dict, x: np.ndarray) -> np.ndarray:
    """y = A x for a stencil in plane form."""
    ny, nx = x.shape
    xp = np.pad(x, 1)
    y = st["C"] * x
    for d in DIRS:
        y = y - st[d] * shifted(xp, d, ny, nx)
    return y


def residual(st: dict, x: np.ndarray, b: np.ndarray) -> np.ndarray:
    """r = b - A x (Algorithm 1)."""
    return b - apply(st, x)


def stencil_to_csr(st: dict) -> sp.csr_matrix:
    """The matrix of a plane-form stencil; unknown (i, j) has index j*nx + i."""
    ny, nx = st["C"].shape
    idx = np.arange(nx * ny).reshape(ny, nx)
    rows = [idx.ravel()]
    cols = [idx.ravel()]
    vals = [st["C"].ravel()]
    for d, (di, dj) in OFFSETS.items():
        j0, j1 = max(0, -dj), ny - max(0, dj)
        i0, i1 = max(0, -di), nx - max(0, di)
        r = idx[j0:j1, i0:i1]
        c = idx[j0 + dj:j1 + dj, i0 + di:i1 + di]
        v = -st[d][j0:j1, i0:i1]
        rows.append(r.ravel())
        cols.append(c.ravel())
        vals.append(v.ravel())
    a = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nx * ny, nx * ny))
    return a.tocsr()


def csr_to_stencil(a: sp.spmatrix, nx: int, ny: int) -> dict:
    """Plane form of a matrix whose pattern is at most 9-point; raises if an
    entry couples unknowns more than one cell apart."""
    a = a.tocoo()
    jr, ir = np.divmod(a.row, nx)
    jc, ic = np.divmod(a.col, nx)
    di = ic - ir
    dj = jc - jr
    if np.any(np.abs(di) > 1) or np.any(np.abs(dj) > 1):
        raise ValueError("operator is not a 9-point stencil")
    st = {d: np.zeros((ny, nx)) for d in ("C",) + DIRS}
    diag = (di == 0) & (dj == 0)
    np.add.at(st["C"], (jr[diag], ir[diag]), a.data[diag])
    for d, (ddi, ddj) in OFFSETS.items():
        m = (di == ddi) & (dj == ddj)
        np.add.at(st[d], (jr[m], ir[m]), -a.data[m])
    return st


# ---------------------------------------------------------------------------
# Operator-induced interpolation (Section 2; weights stored per point as in
# the interpolation stencil of Section 3)
# ---------------------------------------------------------------------------

def coarse_size(n: int) -> int:
    """Standard coarsening by 2: coarse point I is fine point 2I (1-based),
    so a side of n fine points has floor(n / 2) coarse points ((n - 1) / 2
    for the 2^m - 1 sides; for an even n the last fine point is a coarse
    point)."""
    return n // 2


def collapse_stencil(st: dict) -> dict:
    """The stencil the interpolation formulas are applied to: couplings with
    a_X < 0 lumped into the diagonal and a negative row sum dropped,
    a_X+ = max(a_X, 0), C_eff = C - sum_X min(a_X, 0) - min(sigma, 0) with
    sigma = C - sum_X a_X.  Identical to ``st`` on M-matrix rows with
    sigma >= 0."""
    total = 0.0
    for d in DIRS:
        total = total + st[d]
    sigma = st["C"] - total
    neg = 0.0
    for d in DIRS:
        neg = neg + np.minimum(st[d], 0.0)
    out = {d: np.maximum(st[d], 0.0) for d in DIRS}
    out["C"] = (st["C"] - neg) - np.minimum(sigma, 0.0)
    return out


def edge_weights(st: dict):
    """Weights of the two kinds of edge points.

    x-edge points lie on a coarse row between two coarse points (1-based i
    odd, j even; 0-based rows 1::2, cols 0::2).  Collapsing the fine row in y
    gives the 1D flux balance (C - a_S - a_N) u = (a_W + a_SW + a_NW) u_W +
    (a_E + a_SE + a_NE) u_E.  y-edge points (0-based rows 0::2, cols 1::2)
    are the mirror image.  Returns (xw, xe, ys, yn).
    """
    xs = (slice(1, None, 2), slice(0, None, 2))
    den = st["C"][xs] - st["S"][xs] - st["N"][xs]
    xw = (st["W"][xs] + st["SW"][xs] + st["NW"][xs]) / den
    xe = (st["E"][xs] + st["SE"][xs] + st["NE"][xs]) / den
    ysl = (slice(0, None, 2), slice(1, None, 2))
    den = st["C"][ysl] - st["W"][ysl] - st["E"][ysl]
    ys = (st["S"][ysl] + st["SW"][ysl] + st["SE"][ysl]) / den
    yn = (st["N"][ysl] + st["NW"][ysl] + st["NE"][ysl]) / den
    return xw, xe, ys, yn


def interpolation(st: dict) -> sp.csr_matrix:
    """Operator-induced interpolation P_l from level l-1 (coarse) to level l.

    Returns a CSR matrix of shape (nx*ny, ncx*ncy).  Rows are fine unknowns,
    columns interior coarse unknowns; weights towards ghost coarse points
    (outside the domain, value 0) are dropped.  The formulas act on
    ``collapse_stencil(st)``.
    """
    st = collapse_stencil(st)
    ny, nx = st["C"].shape
    ncx, ncy = coarse_size(nx), coarse_size(ny)
    fidx = np.arange(nx * ny).reshape(ny, nx)

    def cidx(q, p):
        """Flat coarse index of 0-based coarse (row q, col p); -1 for ghosts."""
        q = np.asarray(q)
        p = np.asarray(p)
        ok = (q >= 0) & (q < ncy) & (p >= 0) & (p < ncx)
        return np.where(ok, q * ncx + p, -1)

    rows, cols, vals = [], [], []

    def add(frows, ccols, w):
        frows, ccols, w = np.broadcast_arrays(frows, ccols, w)
        keep = ccols >= 0
        rows.append(frows[keep])
        cols.append(ccols[keep])
        vals.append(w[keep])

    # coarse points: injection (0-based fine rows 1::2, cols 1::2)
    q, p = np.meshgrid(np.arange(ncy), np.arange(ncx), indexing="ij")
    add(fidx[1::2, 1::2], cidx(q, p), np.ones((ncy, ncx)))

    xw, xe, ys, yn = edge_weights(st)
    # fine points of odd 1-based index along x and y: (n + 1) // 2 of them
    # (ncx + 1 for the 2^m - 1 sides, ncx for an even side)
    nex, ney = (nx + 1) // 2, (ny + 1) // 2
    # x-edge point (row 2q+1, col 2p): west coarse (q, p-1), east (q, p)
    q, p = np.meshgrid(np.arange(ncy), np.arange(nex), indexing="ij")
    add(fidx[1::2, 0::2], cidx(q, p - 1), xw)
    add(fidx[1::2, 0::2], cidx(q, p), xe)
    # y-edge point (row 2q, col 2p+1): south coarse (q-1, p), north (q, p)
    q, p = np.meshgrid(np.arange(ney), np.arange(ncx), indexing="ij")
    add(fidx[0::2, 1::2], cidx(q - 1, p), ys)
    add(fidx[0::2, 1::2], cidx(q, p), yn)

    # cell-centre point (row 2q, col 2p).  Its W/E neighbours are y-edge
    # points (q, p-1) and (q, p); its S/N neighbours are x-edge points
    # (q-1, p) and (q, p).  Edge weights of neighbours outside the grid are
    # taken as 0; their a-coefficients are 0 anyway (Dirichlet).
    ysp = np.pad(ys, ((0, 0), (1, 1)))   # ysp[q, p'] = ys[q, p'-1]
    ynp = np.pad(yn, ((0, 0), (1, 1)))
    xwp = np.pad(xw, ((1, 1), (0, 0)))   # xwp[q', p] = xw[q'-1, p]
    xep = np.pad(xe, ((1, 1), (0, 0)))
    cs = (slice(0, None, 2), slice(0, None, 2))
    c = st["C"][cs]
    aw, ae, as_, an = st["W"][cs], st["E"][cs], st["S"][cs], st["N"][cs]
    q, p = np.meshgrid(np.arange(ney), np.arange(nex), indexing="ij")
    ys_w, ys_e = ysp[:, 0:nex], ysp[:, 1:nex + 1]       # W nbr (q,p-1), E nbr (q,p)
    yn_w, yn_e = ynp[:, 0:nex], ynp[:, 1:nex + 1]
    xw_s, xw_n = xwp[0:ney, :], xwp[1:ney + 1, :]       # S nbr (q-1,p), N nbr (q,p)
    xe_s, xe_n = xep[0:ney, :], xep[1:ney + 1, :]
    w_sw = (st["SW"][cs] + aw * ys_w + as_ * xw_s) / c
    w_se = (st["SE"][cs] + ae * ys_e + as_ * xe_s) / c
    w_nw = (st["NW"][cs] + aw * yn_w + an * xw_n) / c
    w_ne = (st["NE"][cs] + ae * yn_e + an * xe_n) / c
    f = fidx[0::2, 0::2]
    add(f, cidx(q - 1, p - 1), w_sw)
    add(f, cidx(q - 1, p), w_se)
    add(f, cidx(q, p - 1), w_nw)
    add(f, cidx(q, p), w_ne)

    pm = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(nx * ny, ncx * ncy))
    return pm.tocsr()


def galerkin(st: dict, p: sp.csr_matrix) -> dict:
    """Variational coarse operator P^T A P (Section 2) as a sparse triple
    product; returned in plane form (raises unless it is 9-point)."""
    ny, nx = st["C"].shape
    a = stencil_to_csr(st)
    ac = (p.T @ (a @ p)).tocsr()
    return csr_to_stencil(ac, coarse_size(nx), coarse_size(ny))


# ---------------------------------------------------------------------------
# Coarsest-grid direct solve (Section 3, cost model of the coarse solve:
# a Cholesky factorisation computed and stored in setup)
# ---------------------------------------------------------------------------

def cholesky(m: np.ndarray) -> np.ndarray:
    """Lower-triangular L with L L^T = m (column-by-column Cholesky)."""
    n = m.shape[0]
    lo = np.zeros_like(m, dtype=np.float64)
    for j in range(n):
        s = m[j, j] - lo[j, :j] @ lo[j, :j]
        if not s > 0.0:
            raise ValueError("coarsest operator is not positive definite")
        lo[j, j] = np.sqrt(s)
        for i in range(j + 1, n):
            lo[i, j] = (m[i, j] - lo[i, :j] @ lo[j, :j]) / lo[j, j]
    return lo


def cholesky_solve(lo: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Solve L L^T x = b by forward then backward substitution."""
    n = lo.shape[0]
    y = np.zeros(n)
    for i in range(n):
        y[i] = (b[i] - lo[i, :i] @ y[:i]) / lo[i, i]
    x = np.zeros(n)
    for i in range(n - 1, -1, -1):
        x[i] = (y[i] - lo[i + 1:, i] @ x[i + 1:]) / lo[i, i]
    return x


# ---------------------------------------------------------------------------
# Multicolour Gauss-Seidel (Section 2 smoothing; Section 3 T_smooth with n_c
# colours; Section 5 four-colour Gauss-Seidel)
# ---------------------------------------------------------------------------

# Each colour is a union of the four parity sub-lattices, named by 0-based
# (row parity, col parity).  1-based (i mod 2, j mod 2) = (1, 1) is 0-based
# (even col, even row).
RB_ORDER = (((0, 0), (1, 1)),            # red: (i + j) even
            ((0, 1), (1, 0)))            # black
FOUR_ORDER = (((0, 0),),                 # (i mod 2, j mod 2) = (1, 1)
              ((0, 1),),                 # (0, 1): i even, j odd  -> col odd, row even
              ((1, 0),),                 # (1, 0): i odd, j even  -> col even, row odd
              ((1, 1),))                 # (0, 0)


def is_five_point(st: dict) -> bool:
    return all(not np.any(st[d]) for d in ("SW", "SE", "NW", "NE"))


def colour_order(st: dict):
    """Red-black on a 5-point level (the assembled finest level), four
    colours on a 9-point level (every Galerkin coarse level)."""
    return RB_ORDER if is_five_point(st) else FOUR_ORDER


def relax(st: dict, x: np.ndarray, b: np.ndarray, nu: int, order,
          reverse: bool = False) -> None:
    """``nu`` multicolour Gauss-Seidel sweeps in place.  Within one colour no
    two points are coupled, so each sub-lattice update reads only values of
    other colours: x_p <- (b_p + sum_X a_X x_{p+X}) / C_p."""
    ny, nx = x.shape
    seq = tuple(reversed(order)) if reverse else tuple(order)
    for _ in range(nu):
        for colour in seq:
            for (pj, pi) in colour:
                rows = slice(pj, None, 2)
                cols = slice(pi, None, 2)
                xp = np.pad(x, 1)
                s = b[rows, cols].copy()
                for d in DIRS:
                    s += st[d][rows, cols] * shifted(xp, d, ny, nx, rows, cols)
                x[rows, cols] = s / st["C"][rows, cols]


# ---------------------------------------------------------------------------
# Zebra line Gauss-Seidel (Section 2: alternating line smoothing for
# anisotropic problems)
# ---------------------------------------------------------------------------

# The couplings that stay implicit in a line's system, per line direction.
LINE_DIRS = {"x": ("W", "E"), "y": ("S", "N")}
SMOOTHERS = ("point", "x", "y", "xy")


def line_colour(st: dict, x: np.ndarray, b: np.ndarray, direction: str,
                colour: int) -> None:
    """Solve every line of one colour exactly, in place.  ``colour`` 0 is
    the odd lines (1-based), 0-based rows (x-lines) or columns (y-lines)
    0, 2, 4, ...  Lines of one colour do not couple (the stencil reaches
    one line over), so they are solved together as one banded system with
    no coupling across the seams between lines."""
    import scipy.linalg
    if direction == "y":
        stt = {"C": st["C"].T, "W": st["S"].T, "E": st["N"].T, "S": st["W"].T,
               "N": st["E"].T, "SW": st["SW"].T, "NE": st["NE"].T,
               "SE": st["NW"].T, "NW": st["SE"].T}
        xt = x.T.copy()
        line_colour(stt, xt, b.T, "x", colour)
        x[:] = xt.T
        return
    ny, nx = x.shape
    rows = slice(colour, None, 2)
    xp = np.pad(x, 1)
    rhs = b[rows, :].copy()
    for d in DIRS:
        if d in LINE_DIRS["x"]:
            continue
        rhs += st[d][rows, :] * shifted(xp, d, ny, nx, rows, slice(None))
    n = rhs.size
    ab = np.zeros((3, n))
    ab[0, 1:] = -st["E"][rows, :].ravel()[:-1]   # A[k, k+1]; zero at a row's end
    ab[1] = st["C"][rows, :].ravel()
    ab[2, :-1] = -st["W"][rows, :].ravel()[1:]   # A[k+1, k]; zero at a row's start
    x[rows, :] = scipy.linalg.solve_banded((1, 1), ab, rhs.ravel()).reshape(rhs.shape)


def relax_lines(st: dict, x: np.ndarray, b: np.ndarray, nu: int, smoother: str,
                reverse: bool = False) -> None:
    """``nu`` line Gauss-Seidel sweeps in place: ``smoother`` "x", "y" or
    "xy" (x-lines then y-lines).  Forward: each direction's colours 0 then
    1; reverse: the whole sequence backwards."""
    seq = [(d, c) for d in smoother for c in (0, 1)]
    if reverse:
        seq = seq[::-1]
    for _ in range(nu):
        for d, c in seq:
            line_colour(st, x, b, d, c)


def smooth(h, st: dict, x: np.ndarray, b: np.ndarray, nu: int, reverse: bool) -> None:
    """The hierarchy's smoother: multicolour point Gauss-Seidel or line
    Gauss-Seidel."""
    if h.smoother == "point":
        relax(st, x, b, nu, colour_order(st), reverse=reverse)
    else:
        relax_lines(st, x, b, nu, h.smoother, reverse=reverse)


# ---------------------------------------------------------------------------
# Hierarchy and V-cycle (Algorithm 1)
# ---------------------------------------------------------------------------

@dataclass
class Level:
    st: dict                       # A_l in plane form
    p: sp.csr_matrix | None = None  # P_l: level l-1 -> level l (None on level 0)

    @property
    def shape(self):
        return self.st["C"].shape


@dataclass
class Hierarchy:
    levels: list                   # levels[0] coarsest ... levels[L-1] finest
    chol: np.ndarray               # Cholesky factor of A_0
    nu1: int = 2
    nu2: int = 1
    interp_residual_term: bool = False
    smoother: str = "point"        # "point", "x", "y" or "xy" (see smooth)
    stats: dict = field(default_factory=dict)

    @property
    def nlevels(self):
        return len(self.levels)


def valid_size(n: int) -> bool:
    return n >= 2


def level_shapes(nx: int, ny: int):
    """[(nx, ny) finest, ..., coarsest]: coarsen both sides (n -> floor(n/2))
    while the smaller side exceeds 3 (2^m - 1 sides end at 3; other sides at
    2 or 3)."""
    if not (valid_size(nx) and valid_size(ny)):
        raise ValueError("grid sides must be at least 2")
    out = [(nx, ny)]
    while min(nx, ny) > 3:
        nx, ny = coarse_size(nx), coarse_size(ny)
        out.append((nx, ny))
    return out


def setup(k: np.ndarray, nu1: int = 2, nu2: int = 1,
          interp_residual_term: bool = False, r: float = 1.0, aspect: float = 1.0,
          bc=None, smoother: str = "point") -> Hierarchy:
    """BoxMG setup: assemble the fine operator (``r``, ``aspect``, ``bc`` as
    in assemble_fv5), then for each level build P_l from A_l and
    A_{l-1} = P_l^T A_l P_l; factor A_0 (Section 2).  ``smoother`` picks
    point or line Gauss-Seidel (see smooth)."""
    if smoother not in SMOOTHERS:
        raise ValueError(f"smoother must be one of {SMOOTHERS}")
    ny, nx = k.shape
    shapes = level_shapes(nx, ny)
    if not np.all(np.isfinite(k)) or np.any(k <= 0):
        raise ValueError("coefficients must be finite and positive")
    if not (np.isfinite(r) and r > 0 and np.isfinite(aspect) and aspect > 0):
        raise ValueError("r and the cell aspect must be finite and positive")
    st = assemble_fv5(k, r, aspect, bc)
    fine_to_coarse = [Level(st)]
    for _ in shapes[1:]:
        p = interpolation(st)
        st_c = galerkin(st, p)
        fine_to_coarse[-1].p = p
        fine_to_coarse.append(Level(st_c))
        st = st_c
    levels = fine_to_coarse[::-1]          # levels[0] coarsest
    a0 = stencil_to_csr(levels[0].st).toarray()
    return Hierarchy(levels=levels, chol=cholesky(a0), nu1=nu1, nu2=nu2,
                     interp_residual_term=interp_residual_term, smoother=smoother)


def vcycle(h: Hierarchy, x: np.ndarray, b: np.ndarray) -> None:
    """One V(nu1, nu2) cycle of Algorithm 1, updating the finest x in place."""
    nl = h.nlevels
    xs = [None] * nl
    bs = [None] * nl
    rs = [None] * nl
    xs[nl - 1], bs[nl - 1] = x, b
    for l in range(nl - 1, 0, -1):
        lev = h.levels[l]
        smooth(h, lev.st, xs[l], bs[l], h.nu1, reverse=False)
        rs[l] = residual(lev.st, xs[l], bs[l])
        nyc, nxc = h.levels[l - 1].shape
        bs[l - 1] = (lev.p.T @ rs[l].ravel()).reshape(nyc, nxc)
        xs[l - 1] = np.zeros((nyc, nxc))
    xs[0][:] = cholesky_solve(h.chol, bs[0].ravel()).reshape(xs[0].shape)
    for l in range(1, nl):
        lev = h.levels[l]
        corr = (lev.p @ xs[l - 1].ravel()).reshape(xs[l].shape)
        if h.interp_residual_term:
            # Section 3 interpolation equations: add r/C at every fine point
            # that is not a coarse point (injection points get no r/C).
            rc = rs[l] / lev.st["C"]
            rc[1::2, 1::2] = 0.0
            corr = corr + rc
        xs[l] += corr
        smooth(h, lev.st, xs[l], bs[l], h.nu2, reverse=True)


@dataclass
class SolveResult:
    x: np.ndarray
    cycles: int
    rel_resid: float
    history: list
    converged: bool


def solve(h: Hierarchy, b: np.ndarray, x0: np.ndarray | None = None,
          tol: float = 1e-10, max_cycles: int = 200) -> SolveResult:
    """Iterate V-cycles until ||b - A x||_2 / ||b||_2 <= tol (checked before
    the first cycle and after each one) or ``max_cycles`` cycles ran."""
    fine = h.levels[-1].st
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bn = float(np.linalg.norm(b))
    if bn == 0.0:
        x[:] = 0.0
        return SolveResult(x, 0, 0.0, [0.0], True)
    rel = float(np.linalg.norm(residual(fine, x, b))) / bn
    hist = [rel]
    cycles = 0
    while rel > tol and cycles < max_cycles:
        vcycle(h, x, b)
        cycles += 1
        rel = float(np.linalg.norm(residual(fine, x, b))) / bn
        hist.append(rel)
        if not np.isfinite(rel):
            break
    return SolveResult(x, cycles, rel, hist, bool(rel <= tol))


# ---------------------------------------------------------------------------
# Conjugate gradients preconditioned by one symmetric V-cycle
# ---------------------------------------------------------------------------

def vcycle_precond(h: Hierarchy, r: np.ndarray) -> np.ndarray:
    """z = M^{-1} r: one V(nu, nu) cycle of Algorithm 1 on A z = r from z = 0.
    With nu1 = nu2, forward colours before the coarse correction and the
    reverse order after it, R = P^T and an exact coarsest solve, M^{-1} is a
    symmetric linear operator."""
    z = np.zeros_like(r)
    vcycle(h, z, r)
    return z


def pcg(h: Hierarchy, b: np.ndarray, x0: np.ndarray | None = None, tol: float = 1e-10,
        max_iter: int = 500, precond=None) -> SolveResult:
    """Preconditioned conjugate gradients on A x = b (A the finest operator of
    h), in the textbook order:
        r = b - A x, z = M^{-1} r, p = z, rz = r.z; then per iteration
        q = A p, alpha = rz / p.q, x += alpha p, r -= alpha q, stop test,
        z = M^{-1} r, rz' = r.z, beta = rz' / rz, p = z + beta p.
    The stop test ||r||_2 / ||b||_2 <= tol uses the updated r and is applied
    before the first iteration and after each one.  ``precond`` maps r to z;
    the default is one symmetric V-cycle (h.nu1 == h.nu2 required), None
    for it, or ``"identity"`` for plain conjugate gradients."""
    fine = h.levels[-1].st
    if precond is None:
        if h.nu1 != h.nu2 or h.interp_residual_term:
            raise ValueError("the V-cycle preconditioner needs nu1 == nu2 and no r/C term")
        precond = lambda r: vcycle_precond(h, r)  # noqa: E731
    elif precond == "identity":
        precond = lambda r: r.copy()  # noqa: E731
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bn = float(np.linalg.norm(b))
    if bn == 0.0:
        x[:] = 0.0
        return SolveResult(x, 0, 0.0, [0.0], True)
    r = residual(fine, x, b)
    rel = float(np.linalg.norm(r)) / bn
    hist = [rel]
    it = 0
    if rel <= tol:
        return SolveResult(x, 0, rel, hist, True)
    z = precond(r)
    p = z.copy()
    rz = float(np.sum(r * z))
    while it < max_iter:
        q = apply(fine, p)
        pq = float(np.sum(p * q))
        alpha = rz / pq
        x += alpha * p
        r -= alpha * q
        it += 1
        rel = float(np.linalg.norm(r)) / bn
        hist.append(rel)
        if rel <= tol or not np.isfinite(rel):
            break
        z = precond(r)
        rz_new = float(np.sum(r * z))
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return SolveResult(x, it, rel, hist, bool(rel <= tol))


# ---------------------------------------------------------------------------
# Adjoint gradient with respect to log-coefficients
# ---------------------------------------------------------------------------

def assembly_vjp(k: np.ndarray, u: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """g_c = -d(lam^T A(theta) u)/d theta_c with k = exp(theta).

    A = sum over interior faces f=(p,q) of a_f (e_p - e_q)(e_p - e_q)^T plus
    sum over boundary faces of 2 k_p e_p e_p^T, so
    lam^T A u = sum_f a_f (u_p - u_q)(lam_p - lam_q) + sum_bf 2 k_p u_p lam_p.
    With da/dk1 = 2 k2^2 / (k1 + k2)^2 and dk/dtheta = k:
    g_c = -k_c [ sum_{faces of c} da_f/dk_c (u_c - u_n)(lam_c - lam_n)
                 + (number of boundary faces of c) * 2 u_c lam_c ].
    """
    k = np.asarray(k, dtype=np.float64)
    ny, nx = k.shape
    g = np.zeros((ny, nx))
    # x faces between (i, j) and (i+1, j)
    k1, k2 = k[:, :-1], k[:, 1:]
    prod = (u[:, :-1] - u[:, 1:]) * (lam[:, :-1] - lam[:, 1:])
    s = (k1 + k2) ** 2
    g[:, :-1] += 2.0 * k2 * k2 / s * prod
    g[:, 1:] += 2.0 * k1 * k1 / s * prod
    # y faces
    k1, k2 = k[:-1, :], k[1:, :]
    prod = (u[:-1, :] - u[1:, :]) * (lam[:-1, :] - lam[1:, :])
    s = (k1 + k2) ** 2
    g[:-1, :] += 2.0 * k2 * k2 / s * prod
    g[1:, :] += 2.0 * k1 * k1 / s * prod
    # boundary faces
    nb = np.zeros((ny, nx))
    nb[:, 0] += 1
    nb[:, -1] += 1
    nb[0, :] += 1
    nb[-1, :] += 1
    g += nb * 2.0 * u * lam
    return -k * g


def direct_solve(k: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Exact (sparse LU) solution of the assembled system, for small grids."""
    import scipy.sparse.linalg as spla
    a = stencil_to_csr(assemble_fv5(k)).tocsc()
    return spla.spsolve(a, b.ravel()).reshape(b.shape)


def loss(theta: np.ndarray, b: np.ndarray, u_obs: np.ndarray) -> float:
    """L = 0.5 ||u(theta) - u_obs||^2 with u the exact solution."""
    u = direct_solve(np.exp(theta), b)
    return 0.5 * float(np.sum((u - u_obs) ** 2))


def adjoint_gradient(theta: np.ndarray, b: np.ndarray, u_obs: np.ndarray):
    """dL/dtheta via the adjoint equation A lam = u - u_obs (A symmetric),
    with exact sparse solves.  Returns (grad, u, lam)."""
    k = np.exp(theta)
    u = direct_solve(k, b)
    lam = direct_solve(k, u - u_obs)
    return assembly_vjp(k, u, lam), u, lam
