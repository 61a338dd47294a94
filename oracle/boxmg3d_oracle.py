"""Plain FP64 CPU oracle of the BoxMG V-cycle for 3D heterogeneous diffusion.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this module.  The library's product
path never calls it, and it shares no code with the CUDA path.

The paper (Reisner, Olson, Moulton) measures BoxMG in 2D and models its 3D
interpolation cost (Section 3, the 3D form of T_interp); this module extends
the 2D oracle's readings to three dimensions:

* ``assemble_fv7``  -- the 7-point cell-centred finite-volume operator of
  -div(k grad u) = f with u = 0 on the boundary of the unit cube (the 3D form
  of Section 5's Eqs. (diffusion), (diffusion_bc)): harmonic-mean faces,
  2 k on a boundary face, scaled by h (cubic cells), so b is used as given.
* ``interpolation`` -- operator-induced interpolation, coarse point I = fine
  point 2I per direction (1-based), by collapsing the fine stencil onto the
  coarse directions: a fine point between coarse points in one direction
  (edge point) takes the 1D collapse of its equation (everything on each
  side summed, the couplings within its own transverse plane moved to the
  diagonal); one between coarse points in two directions (face point) takes
  its equation collapsed along the third direction, with its edge neighbours
  replaced by their interpolants; one between coarse points in all three
  (cell centre) takes its full equation with every non-coarse neighbour
  replaced by its interpolant.  With constant k these are exactly the
  trilinear weights 1/2, 1/4, 1/8.  Rows that are not M-matrix rows get the
  2D oracle's lumping (positive matrix entries and a negative row sum moved
  to the diagonal) before collapsing.
* ``galerkin`` -- A_{l-1} = P^T A_l P as a sparse triple product, checked to
  be a 27-point stencil.
* ``relax`` -- multicolour point Gauss-Seidel: red-black on the 7-point
  finest level, eight colours (the parities of i, j, k) on 27-point levels,
  colours in order of the colour index 4 (k-1 mod 2) + 2 (j-1 mod 2) +
  (i-1 mod 2) forward for pre-smoothing and reversed for post-smoothing.
* ``vcycle`` / ``solve`` -- Algorithm 1 with a dense Cholesky solve on the
  coarsest level; stop on ||b - Ax||_2 / ||b||_2 <= tol after each cycle.
* ``vcycle_precond`` / ``pcg`` -- conjugate gradients on the finest operator
  preconditioned by one symmetric V(nu, nu) cycle from zero (an extension;
  the 2D oracle's textbook order).

Sizes: any side >= 2; a side of n points coarsens to floor(n / 2); coarsening
stops once the smallest side is at most 3.

Data layout: grid arrays have shape (nz, ny, nx), a[k, j, i] with i fastest;
unknown (i, j, k) has index (k * ny + j) * nx + i.  Operators are scipy CSR
matrices.
"""
from __future__ import annotations

from dataclasses import dataclass
from itertools import product

import numpy as np
import scipy.sparse as sp

from oracle.boxmg_oracle import cholesky, cholesky_solve

OFFS = [d for d in product((-1, 0, 1), repeat=3) if d != (0, 0, 0)]  # (di, dj, dk)


# ---------------------------------------------------------------------------
# Discretisation
# ---------------------------------------------------------------------------

def assemble_fv7(k: np.ndarray) -> sp.csr_matrix:
    """7-point cell-centred FV operator for -div(k grad u) on the unit cube,
    u = 0 on the boundary, cubic cells, scaled by h: face coefficient
    2 k1 k2 / (k1 + k2) between cells, 2 k on a boundary face, C = sum of the
    six face coefficients."""
    k = np.asarray(k, dtype=np.float64)
    nz, ny, nx = k.shape
    n = nx * ny * nz
    idx = np.arange(n).reshape(nz, ny, nx)
    rows, cols, vals = [], [], []
    diag = np.zeros((nz, ny, nx))
    for axis in range(3):
        a = np.moveaxis(k, 2 - axis, 0)          # axis 0 of a is the face normal
        face = 2.0 * a[:-1] * a[1:] / (a[:-1] + a[1:])
        fa = np.moveaxis(face, 0, 2 - axis)
        sl_lo = [slice(None)] * 3
        sl_hi = [slice(None)] * 3
        sl_lo[2 - axis] = slice(0, -1)
        sl_hi[2 - axis] = slice(1, None)
        lo, hi = idx[tuple(sl_lo)], idx[tuple(sl_hi)]
        rows += [lo.ravel(), hi.ravel()]
        cols += [hi.ravel(), lo.ravel()]
        vals += [-fa.ravel(), -fa.ravel()]
        diag[tuple(sl_lo)] += fa
        diag[tuple(sl_hi)] += fa
        # boundary faces at both ends of this axis
        first = [slice(None)] * 3
        last = [slice(None)] * 3
        first[2 - axis] = 0
        last[2 - axis] = -1
        diag[tuple(first)] += 2.0 * k[tuple(first)]
        diag[tuple(last)] += 2.0 * k[tuple(last)]
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n)).tocsr()


def coarse_size(n: int) -> int:
    """A side of n points coarsens to floor(n / 2): coarse point I is fine
    point 2I (1-based)."""
    return n // 2


def level_shapes(nx: int, ny: int, nz: int):
    if min(nx, ny, nz) < 2:
        raise ValueError("grid sides must be at least 2")
    out = [(nx, ny, nz)]
    while min(nx, ny, nz) > 3:
        nx, ny, nz = coarse_size(nx), coarse_size(ny), coarse_size(nz)
        out.append((nx, ny, nz))
    return out


# ---------------------------------------------------------------------------
# Operator-induced interpolation
# ---------------------------------------------------------------------------

def _row_couplings(a: sp.csr_matrix, shape, p):
    """Diagonal and the negated off-diagonals of row p by offset (di, dj, dk),
    after the lumping of non-M-matrix rows: positive matrix entries and a
    negative row sum go to the diagonal."""
    nx, ny, nz = shape
    k0, rem = divmod(p, nx * ny)
    j0, i0 = divmod(rem, nx)
    cpl = {}
    diag = 0.0
    for q, v in zip(a.indices[a.indptr[p]:a.indptr[p + 1]], a.data[a.indptr[p]:a.indptr[p + 1]]):
        if q == p:
            diag += v
            continue
        k1, rem1 = divmod(int(q), nx * ny)
        j1, i1 = divmod(rem1, nx)
        cpl[(i1 - i0, j1 - j0, k1 - k0)] = -v
    sigma = diag - sum(cpl.values())
    neg = sum(min(v, 0.0) for v in cpl.values())
    ceff = diag - neg - min(sigma, 0.0)
    return ceff, {d: max(v, 0.0) for d, v in cpl.items()}


def interpolation(a: sp.csr_matrix, shape) -> sp.csr_matrix:
    """P: coarse (floor(n/2) per side) -> fine, by the collapsed equations
    described in the module docstring."""
    nx, ny, nz = shape
    cx, cy, cz = coarse_size(nx), coarse_size(ny), coarse_size(nz)

    def cidx(I, J, K):
        return (K * cy + J) * cx + I

    def fidx(i, j, k):                        # 0-based fine
        return (k * ny + j) * nx + i

    def coarse_of(i, j, k):
        """The coarse point at fine (0-based) (i, j, k), or None (not a
        coarse point, or outside the grid)."""
        if not (0 <= i < nx and 0 <= j < ny and 0 <= k < nz):
            return None
        if i % 2 == 1 and j % 2 == 1 and k % 2 == 1:
            I, J, K = (i - 1) // 2, (j - 1) // 2, (k - 1) // 2
            if I < cx and J < cy and K < cz:
                return cidx(I, J, K)
        return None

    rows = {}                                  # fine index -> {coarse index: weight}

    def value(i, j, k):
        """Interpolant of fine (i, j, k) (0-based) as {coarse: weight}; the
        empty dict outside the grid (zero Dirichlet values)."""
        if not (0 <= i < nx and 0 <= j < ny and 0 <= k < nz):
            return {}
        return rows[fidx(i, j, k)]

    # A fine point's type: which 0-based coordinates are even, i.e. fall
    # between coarse points (1-based odd).
    pts = [(i, j, k) for k in range(nz) for j in range(ny) for i in range(nx)]
    by_count = {0: [], 1: [], 2: [], 3: []}
    for (i, j, k) in pts:
        between = (i % 2 == 0) + (j % 2 == 0) + (k % 2 == 0)
        by_count[between].append((i, j, k))
    for (i, j, k) in by_count[0]:
        c = coarse_of(i, j, k)
        rows[fidx(i, j, k)] = {c: 1.0} if c is not None else {}
    for nb in (1, 2, 3):
        for (i, j, k) in by_count[nb]:
            p = fidx(i, j, k)
            ceff, cpl = _row_couplings(a, shape, p)
            free = [(i % 2 == 0), (j % 2 == 0), (k % 2 == 0)]   # directions between coarse points
            # collapse every direction the point is coarse-aligned in: a
            # coupling's offset in such a direction is set to 0
            coll = {}
            den = ceff
            for d, v in cpl.items():
                dd = tuple(d[t] if free[t] else 0 for t in range(3))
                if dd == (0, 0, 0):
                    den -= v
                else:
                    coll[dd] = coll.get(dd, 0.0) + v
            out = {}
            for dd, v in coll.items():
                if v == 0.0:
                    continue
                for c, w in value(i + dd[0], j + dd[1], k + dd[2]).items():
                    out[c] = out.get(c, 0.0) + v * w
            if den <= 0.0:
                raise ValueError(f"interpolation denominator <= 0 at fine point {(i, j, k)}")
            rows[p] = {c: w / den for c, w in out.items()}
    r, c, v = [], [], []
    for p, row in rows.items():
        for q, w in row.items():
            r.append(p)
            c.append(q)
            v.append(w)
    return sp.coo_matrix((v, (r, c)), shape=(nx * ny * nz, cx * cy * cz)).tocsr()


def galerkin(a: sp.csr_matrix, p: sp.csr_matrix, coarse_shape) -> sp.csr_matrix:
    """A_c = P^T A P, checked to be a 27-point stencil."""
    ac = (p.T @ (a @ p)).tocsr()
    ac.eliminate_zeros()
    nx, ny, nz = coarse_shape
    coo = ac.tocoo()
    kr, rr = np.divmod(coo.row, nx * ny)
    jr, ir = np.divmod(rr, nx)
    kc, rc = np.divmod(coo.col, nx * ny)
    jc, ic = np.divmod(rc, nx)
    if (np.abs(ic - ir).max(initial=0) > 1 or np.abs(jc - jr).max(initial=0) > 1
            or np.abs(kc - kr).max(initial=0) > 1):
        raise ValueError("coarse operator is not a 27-point stencil")
    return ac


# ---------------------------------------------------------------------------
# Multicolour Gauss-Seidel
# ---------------------------------------------------------------------------

def is_seven_point(a: sp.csr_matrix, shape) -> bool:
    nx, ny, nz = shape
    coo = a.tocoo()
    d = np.abs(coo.col - coo.row)
    return bool(np.all(np.isin(d, (0, 1, nx, nx * ny))))


def colours(shape, seven: bool):
    """Colour index per unknown, and the number of colours: red-black
    ((i + j + k) parity) on the 7-point level, the eight parities
    4 (k mod 2) + 2 (j mod 2) + (i mod 2) (0-based) otherwise."""
    nx, ny, nz = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    if seven:
        return ((i + j + k) % 2).ravel(), 2
    return (4 * (k % 2) + 2 * (j % 2) + (i % 2)).ravel(), 8


def relax(a: sp.csr_matrix, shape, x: np.ndarray, b: np.ndarray, nu: int,
          reverse: bool = False) -> None:
    """nu multicolour Gauss-Seidel sweeps in place (x, b flat).  No two
    points of one colour are coupled, so each colour is one simultaneous
    update x_c <- (b_c - A_{c,other} x_other) / diag_c."""
    col, nc = colours(shape, is_seven_point(a, shape))
    diag = a.diagonal()
    off = (a - sp.diags(diag)).tocsr()
    order = list(range(nc))
    if reverse:
        order.reverse()
    sets = [np.nonzero(col == c)[0] for c in range(nc)]
    for _ in range(nu):
        for c in order:
            s = sets[c]
            x[s] = (b[s] - off[s] @ x) / diag[s]


# ---------------------------------------------------------------------------
# Hierarchy and V-cycle
# ---------------------------------------------------------------------------

@dataclass
class Level3:
    a: sp.csr_matrix
    shape: tuple
    p: sp.csr_matrix | None = None     # interpolation from the next coarser level


@dataclass
class Hierarchy3:
    levels: list                       # levels[0] coarsest ... levels[-1] finest
    chol: np.ndarray
    nu1: int = 2
    nu2: int = 1


def setup(k: np.ndarray, nu1: int = 2, nu2: int = 1) -> Hierarchy3:
    nz, ny, nx = k.shape
    if not np.all(np.isfinite(k)) or np.any(k <= 0):
        raise ValueError("coefficients must be finite and positive")
    shapes = level_shapes(nx, ny, nz)
    a = assemble_fv7(k)
    fine_first = [Level3(a, shapes[0])]
    for s in shapes[1:]:
        prev = fine_first[-1]
        p = interpolation(prev.a, prev.shape)
        prev.p = p
        fine_first.append(Level3(galerkin(prev.a, p, s), s))
    levels = fine_first[::-1]
    return Hierarchy3(levels=levels, chol=cholesky(levels[0].a.toarray()), nu1=nu1, nu2=nu2)


def vcycle(h: Hierarchy3, x: np.ndarray, b: np.ndarray) -> None:
    L = len(h.levels)
    xs, bs = [None] * L, [None] * L
    xs[-1], bs[-1] = x, b
    for l in range(L - 1, 0, -1):
        lev = h.levels[l]
        relax(lev.a, lev.shape, xs[l], bs[l], h.nu1)
        r = bs[l] - lev.a @ xs[l]
        bs[l - 1] = lev.p.T @ r
        xs[l - 1] = np.zeros(bs[l - 1].size)
    xs[0][:] = cholesky_solve(h.chol, bs[0])
    for l in range(1, L):
        lev = h.levels[l]
        xs[l] += lev.p @ xs[l - 1]
        relax(lev.a, lev.shape, xs[l], bs[l], h.nu2, reverse=True)


@dataclass
class SolveResult3:
    x: np.ndarray
    cycles: int
    rel_resid: float
    history: list
    converged: bool


def solve(h: Hierarchy3, b: np.ndarray, tol: float = 1e-10, max_cycles: int = 200) -> SolveResult3:
    """V-cycles from x = 0 until ||b - Ax|| / ||b|| <= tol (b of shape
    (nz, ny, nx) or flat); returns x in b's shape."""
    shape = np.shape(b)
    bf = np.asarray(b, dtype=np.float64).ravel()
    a = h.levels[-1].a
    x = np.zeros_like(bf)
    bn = float(np.linalg.norm(bf))
    if bn == 0.0:
        return SolveResult3(x.reshape(shape), 0, 0.0, [0.0], True)
    rel = float(np.linalg.norm(bf - a @ x)) / bn
    hist = [rel]
    cyc = 0
    while rel > tol and cyc < max_cycles:
        vcycle(h, x, bf)
        cyc += 1
        rel = float(np.linalg.norm(bf - a @ x)) / bn
        hist.append(rel)
        if not np.isfinite(rel):
            break
    return SolveResult3(x.reshape(shape), cyc, rel, hist, bool(rel <= tol))


# ---------------------------------------------------------------------------
# Conjugate gradients preconditioned by one symmetric V-cycle
# ---------------------------------------------------------------------------

def vcycle_precond(h: Hierarchy3, r: np.ndarray) -> np.ndarray:
    """z = M^{-1} r (flat vectors): one V(nu, nu) cycle of Algorithm 1 on
    A z = r from z = 0.  With nu1 = nu2, the post-smoothing colours reversed,
    R = P^T and an exact coarsest solve, M^{-1} is symmetric and positive
    definite."""
    z = np.zeros_like(r)
    vcycle(h, z, r)
    return z


def pcg(h: Hierarchy3, b: np.ndarray, tol: float = 1e-10, max_iter: int = 500,
        precond=None) -> SolveResult3:
    """Preconditioned conjugate gradients on A x = b from x = 0, in the
    textbook order:
        r = b - A x, z = M^{-1} r, p = z, rz = r.z; then per iteration
        q = A p, alpha = rz / p.q, x += alpha p, r -= alpha q, stop test,
        z = M^{-1} r, rz' = r.z, beta = rz' / rz, p = z + beta p.
    The stop test ||r||_2 / ||b||_2 <= tol uses the updated r, before the
    first iteration and after each one.  ``precond``: None for one symmetric
    V-cycle (nu1 == nu2 required), or "identity" for plain conjugate
    gradients.  Returns x in b's shape; `cycles` counts iterations."""
    if precond is None:
        if h.nu1 != h.nu2:
            raise ValueError("the V-cycle preconditioner needs nu1 == nu2")
        precond = lambda r: vcycle_precond(h, r)  # noqa: E731
    elif precond == "identity":
        precond = lambda r: r.copy()  # noqa: E731
    shape = np.shape(b)
    bf = np.asarray(b, dtype=np.float64).ravel()
    a = h.levels[-1].a
    x = np.zeros_like(bf)
    bn = float(np.linalg.norm(bf))
    if bn == 0.0:
        return SolveResult3(x.reshape(shape), 0, 0.0, [0.0], True)
    r = bf - a @ x
    rel = float(np.linalg.norm(r)) / bn
    hist = [rel]
    it = 0
    if rel <= tol:
        return SolveResult3(x.reshape(shape), 0, rel, hist, True)
    z = precond(r)
    p = z.copy()
    rz = float(r @ z)
    while it < max_iter:
        q = a @ p
        alpha = rz / float(p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        rel = float(np.linalg.norm(r)) / bn
        hist.append(rel)
        if rel <= tol or not np.isfinite(rel):
            break
        z = precond(r)
        rz_new = float(r @ z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return SolveResult3(x.reshape(shape), it, rel, hist, bool(rel <= tol))
