"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, exact rational arithmetic done independently, invariants, library
routines on special cases, brute force on tiny grids, or convergence orders.
Together they are meant to fail for a dropped term, a wrong sign, a wrong
index or a transposed operand anywhere in the oracle.
"""
from fractions import Fraction as F

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import boxmg_oracle as O
from paper_1803_02481_gb300 import inputs


# ---------------------------------------------------------------------------
# Assembly (Section 5, Eqs. (diffusion), (diffusion_bc))
# ---------------------------------------------------------------------------

def test_assembly_constant_k_closed_form():
    """k = 1: interior row [-1; -1 4 -1; -1]; a boundary face adds 2k, so an
    edge cell has C = 3 + 2 = 5 and a corner cell C = 2 + 4 = 6; no coupling
    leaves the domain."""
    st = O.assemble_fv5(np.ones((5, 6)))
    assert np.all(st["C"][1:-1, 1:-1] == 4.0)
    assert st["C"][0, 2] == 5.0 and st["C"][2, 0] == 5.0 and st["C"][-1, 2] == 5.0
    assert st["C"][0, 0] == 6.0 and st["C"][-1, -1] == 6.0 and st["C"][0, -1] == 6.0
    for d in ("W", "E", "S", "N"):
        inner = st[d][1:-1, 1:-1]
        assert np.all(inner == 1.0)
    assert np.all(st["W"][:, 0] == 0) and np.all(st["E"][:, -1] == 0)
    assert np.all(st["S"][0, :] == 0) and np.all(st["N"][-1, :] == 0)
    for d in ("SW", "SE", "NW", "NE"):
        assert not np.any(st[d])


def _mms_layered_error(n, k1, k2):
    """u = sin(2 pi x) sin(pi y) / k(x), k = k1 left of x = 1/2, k2 right.
    u is continuous (zero at x = 1/2), the flux k u_x = 2 pi cos(2 pi x)
    sin(pi y) is continuous and non-zero there, and -div(k grad u) =
    5 pi^2 sin(2 pi x) sin(pi y) on both sides."""
    h = 1.0 / n
    xc = (np.arange(n) + 0.5) * h
    x, y = np.meshgrid(xc, xc)
    k = np.where(x < 0.5, k1, k2)
    u = np.sin(2 * np.pi * x) * np.sin(np.pi * y) / k
    f = 5 * np.pi ** 2 * np.sin(2 * np.pi * x) * np.sin(np.pi * y)
    uh = O.direct_solve(k, h * h * f)
    return np.abs(uh - u).max() / np.abs(u).max()


def test_assembly_second_order_across_interface():
    """Harmonic-mean faces give O(h^2) across a coefficient jump aligned with
    cell faces (an arithmetic mean would give O(h))."""
    errs = [_mms_layered_error(n, 1.0, 100.0) for n in (16, 32, 64)]
    for e0, e1 in zip(errs, errs[1:]):
        assert 3.6 < e0 / e1 < 4.4
    assert errs[-1] < 1e-3


def test_assembly_second_order_smooth_k():
    """u = sin(pi x) sin(pi y), k = exp(x + 2y):
    f = k (2 pi^2 u - pi cos(pi x) sin(pi y) - 2 pi sin(pi x) cos(pi y))."""
    def err(n):
        h = 1.0 / n
        xc = (np.arange(n) + 0.5) * h
        x, y = np.meshgrid(xc, xc)
        k = np.exp(x + 2 * y)
        u = np.sin(np.pi * x) * np.sin(np.pi * y)
        f = k * (2 * np.pi ** 2 * u - np.pi * np.cos(np.pi * x) * np.sin(np.pi * y)
                 - 2 * np.pi * np.sin(np.pi * x) * np.cos(np.pi * y))
        return np.abs(O.direct_solve(k, h * h * f) - u).max()
    errs = [err(n) for n in (16, 32, 64)]
    for e0, e1 in zip(errs, errs[1:]):
        assert 3.6 < e0 / e1 < 4.4


def test_operator_symmetric_positive_definite():
    rng = np.random.default_rng(11)
    k = 10.0 ** rng.uniform(-3, 3, size=(9, 12))
    a = O.stencil_to_csr(O.assemble_fv5(k)).toarray()
    assert np.array_equal(a, a.T)
    assert np.linalg.eigvalsh(a).min() > 0


# ---------------------------------------------------------------------------
# Operator-induced interpolation (Section 2)
# ---------------------------------------------------------------------------

def _hat(n_fine, n_coarse, idx):
    """1D piecewise-linear hat of coarse node ``idx`` (0-based) evaluated at
    the fine cell centres of [0, 1].  Coarse node I (1-based) sits at fine
    cell centre 2I, i.e. x = (2I - 0.5) h; the boundary x = 0, 1 is a node
    with value 0 (Dirichlet)."""
    h = 1.0 / n_fine
    xf = (np.arange(n_fine) + 0.5) * h
    nodes = np.concatenate([[0.0], (2 * np.arange(1, n_coarse + 1) - 0.5) * h, [1.0]])
    vals = np.zeros(n_coarse + 2)
    vals[idx + 1] = 1.0
    return np.interp(xf, nodes, vals)


@pytest.mark.parametrize("nx, ny", [(15, 7), (16, 8), (14, 9), (6, 5)])
def test_interpolation_constant_k_is_bilinear(nx, ny):
    """k = 1: every column of P is the tensor product of 1D hats on the
    coarse nodes plus the boundary (weights 1, 1/2, 1/4 inside; the fine
    point between the wall and the first coarse node gets 1/3, a corner
    1/9).  On an even side the last fine point is itself a coarse node next
    to the wall; the edge points on that last fine line collapse the wall's
    Dirichlet face into their denominator (flux balance), so they (and the
    centre points beside them, which use their weights) are left out of
    the hat comparison and the edge points are checked against that closed
    form instead: k = 1 gives 1/4, and 1/5 next to a corner."""
    st = O.assemble_fv5(np.ones((ny, nx)))
    p = O.interpolation(st).toarray()
    ncx, ncy = nx // 2, ny // 2
    keep = np.ones((ny, nx), dtype=bool)      # the centre points next to that
    if nx % 2 == 0:                            # line use its edge weights too
        keep[:, -2:] = False
    if ny % 2 == 0:
        keep[-2:, :] = False
    for q in range(ncy):
        for pp in range(ncx):
            expect = np.outer(_hat(ny, ncy, q), _hat(nx, ncx, pp))
            got = p[:, q * ncx + pp].reshape(ny, nx)
            np.testing.assert_allclose(got[keep], expect[keep], rtol=0, atol=1e-15)
    if nx % 2 == 0:
        # y-edge points (row j odd, 1-based) on the last column: weight to
        # the coarse node above and below; denominators 4 (5 at a wall row)
        col = p.reshape(ny, nx, ncy * ncx)[:, -1, :]
        for j in range(1, ny + 1, 2):
            den = 4.0 + (j == 1) + (j == ny)
            for qq in (j // 2 - 1, j // 2):          # coarse rows below / above (0-based)
                if 0 <= qq < ncy:
                    assert abs(col[j - 1, qq * ncx + ncx - 1] - 1.0 / den) <= 1e-15


def test_interpolation_layered_medium_flux_weights():
    """k depending on x only: an interior x-edge point between coarse nodes
    takes the series-conductance (flux-continuous) weights a_w / (a_w + a_e)
    and a_e / (a_w + a_e); a y-edge point takes 1/2, 1/2; a cell-centre point
    the product of the two."""
    rng = np.random.default_rng(3)
    nx, ny = 15, 15
    kx = 10.0 ** rng.uniform(-3, 3, size=nx)
    k = np.repeat(kx[None, :], ny, axis=0)
    st = O.assemble_fv5(k)
    p = O.interpolation(st).toarray()
    ncx = 7
    face = 2 * kx[:-1] * kx[1:] / (kx[:-1] + kx[1:])   # face between i and i+1
    j0 = 7                                             # 0-based row 7 = coarse row 3
    q = 3
    for i0 in range(2, nx - 2, 2):                     # x-edge points, 0-based even
        aw, ae = face[i0 - 1], face[i0]
        # C - a_S - a_N cancels the y couplings: rounding is relative to C
        tol = 8e-16 * st["C"][j0, i0] / (aw + ae)
        row = p[j0 * nx + i0].reshape(-1)
        pw, pe = i0 // 2 - 1, i0 // 2
        assert abs(row[q * ncx + pw] - aw / (aw + ae)) < tol
        assert abs(row[q * ncx + pe] - ae / (aw + ae)) < tol
        # the cell-centre point one row below: product with 1/2 in y
        rowc = p[(j0 - 1) * nx + i0]
        assert abs(rowc[q * ncx + pw] - 0.5 * aw / (aw + ae)) < tol
        assert abs(rowc[(q - 1) * ncx + pe] - 0.5 * ae / (aw + ae)) < tol
    for i0 in range(1, nx - 1, 2):                     # y-edge points
        row = p[(j0 - 1) * nx + i0]
        assert abs(row[q * ncx + i0 // 2] - 0.5) < 1e-14
        assert abs(row[(q - 1) * ncx + i0 // 2] - 0.5) < 1e-14


def test_interpolation_rows_sum_to_one_where_row_sum_zero():
    """Where A's row sum vanishes (interior), the weights of the interior
    edge/centre points sum to 1: constants are interpolated exactly."""
    rng = np.random.default_rng(5)
    k = 10.0 ** rng.uniform(-2, 2, size=(31, 31))
    st = O.assemble_fv5(k)
    p = O.interpolation(st)
    s = np.asarray(p.sum(axis=1)).reshape(31, 31)
    np.testing.assert_allclose(s[2:-2, 2:-2], 1.0, atol=1e-14)


def test_operator_induced_beats_bilinear_on_contrast():
    """On a 10^8-contrast block field the two-grid error reduction with
    operator-induced P is far better than with the constant-k (bilinear) P.
    A wrong index or swapped weight in P destroys the gap."""
    rng = np.random.default_rng(2)
    n = 15
    k = inputs.block_field(rng, n, n, 4, -4, 4)
    st = O.assemble_fv5(k)

    def rate(p):
        a = O.stencil_to_csr(st)
        lu = spla.splu((p.T @ a @ p).tocsc())
        x = np.random.default_rng(0).standard_normal((n, n))
        b = np.zeros((n, n))
        for _ in range(30):
            n0 = np.sqrt(x.ravel() @ (a @ x.ravel()))
            O.relax(st, x, b, 2, O.RB_ORDER)
            r = -(a @ x.ravel())
            x += (p @ lu.solve(p.T @ r)).reshape(n, n)
            O.relax(st, x, b, 1, O.RB_ORDER, reverse=True)
            n1 = np.sqrt(x.ravel() @ (a @ x.ravel()))
        return n1 / n0

    good = rate(O.interpolation(st))
    bilinear = rate(O.interpolation(O.assemble_fv5(np.ones((n, n)))))
    assert good < 0.25
    assert bilinear > 0.5


# ---------------------------------------------------------------------------
# Galerkin coarse operator (Section 2)
# ---------------------------------------------------------------------------

def _conv(s1, s2):
    out = {}
    for (a, b), v in s1.items():
        for (c, d), w in s2.items():
            out[(a + c, b + d)] = out.get((a + c, b + d), 0) + v * w
    return out


def _galerkin_symbol(alpha, pi):
    """Interior (infinite-grid) Galerkin stencil of a constant stencil alpha
    with a symmetric prolongation stencil pi: A_c(D) = (pi * alpha * pi)(2D),
    computed with exact rationals."""
    full = _conv(_conv(pi, alpha), pi)
    return {(dx // 2, dy // 2): v for (dx, dy), v in full.items()
            if dx % 2 == 0 and dy % 2 == 0 and v != 0}


BILINEAR = {(dx, dy): F(2 - abs(dx), 2) * F(2 - abs(dy), 2)
            for dx in (-1, 0, 1) for dy in (-1, 0, 1)}
LAPLACE5 = {(0, 0): F(4), (1, 0): F(-1), (-1, 0): F(-1), (0, 1): F(-1), (0, -1): F(-1)}


def _oracle_interior(st):
    ny, nx = st["C"].shape
    j, i = ny // 2, nx // 2
    m = {(0, 0): st["C"][j, i]}
    for d, (di, dj) in O.OFFSETS.items():
        m[(di, dj)] = -st[d][j, i]
    return m


def test_rap_constant_k_closed_form_two_levels():
    lev1 = _galerkin_symbol(LAPLACE5, BILINEAR)
    # the familiar closed form [[-1/4,-1/2,-1/4],[-1/2,3,-1/2],[-1/4,-1/2,-1/4]]
    assert lev1[(0, 0)] == 3 and lev1[(1, 0)] == F(-1, 2) and lev1[(1, 1)] == F(-1, 4)
    lev2 = _galerkin_symbol(lev1, BILINEAR)
    assert lev2[(0, 0)] == F(11, 4) and lev2[(1, 0)] == F(-3, 8) and lev2[(1, 1)] == F(-5, 16)
    h = O.setup(np.ones((63, 63)))
    for l, expect in ((h.nlevels - 2, lev1), (h.nlevels - 3, lev2)):
        got = _oracle_interior(h.levels[l].st)
        for key, v in expect.items():
            assert got[key] == float(v), (l, key)
    # interior P of the level-1 operator is bilinear again
    p = O.interpolation(h.levels[h.nlevels - 2].st)
    assert p[15 * 31 + 14, 7 * 15 + 6] == 0.5        # x-edge, row 15 col 14
    assert p[14 * 31 + 14, 7 * 15 + 6] == 0.25       # centre


def test_rap_is_symmetric_nine_point_with_zero_interior_row_sums():
    rng = np.random.default_rng(7)
    k = inputs.block_field(rng, 63, 63, 8, -4, 4)
    h = O.setup(k)
    for l in range(h.nlevels - 1):
        st = h.levels[l].st
        ny, nx = st["C"].shape
        scale = np.abs(st["C"]).max()
        # full symmetry of the stored 9-point planes
        assert np.allclose(st["W"][:, 1:], st["E"][:, :-1], rtol=0, atol=1e-13 * scale)
        assert np.allclose(st["S"][1:, :], st["N"][:-1, :], rtol=0, atol=1e-13 * scale)
        assert np.allclose(st["SW"][1:, 1:], st["NE"][:-1, :-1], rtol=0, atol=1e-13 * scale)
        assert np.allclose(st["NW"][:-1, 1:], st["SE"][1:, :-1], rtol=0, atol=1e-13 * scale)
        rs = st["C"] - sum(st[d] for d in O.DIRS)
        if ny > 4:
            assert np.abs(rs[2:-2, 2:-2]).max() <= 1e-12 * scale
        assert np.all(rs >= -1e-12 * scale)                 # diagonally dominant rows
        a = O.stencil_to_csr(st).toarray()
        assert np.linalg.eigvalsh(a).min() > 0


def test_rap_pattern_check_rejects_wider_coupling():
    import scipy.sparse as sp
    a = sp.lil_matrix((9, 9))
    a[0, 0] = 1.0
    a[0, 2] = 1.0                                         # two cells apart in x
    with pytest.raises(ValueError):
        O.csr_to_stencil(a.tocsr(), 3, 3)


def test_two_grid_galerkin_orthogonality():
    """After an exact coarse-grid correction the restricted residual
    vanishes: P^T (b - A (x + P A_c^{-1} P^T r)) = 0."""
    rng = np.random.default_rng(9)
    k = 10.0 ** rng.uniform(-2, 2, size=(31, 31))
    st = O.assemble_fv5(k)
    p = O.interpolation(st)
    ac = O.stencil_to_csr(O.galerkin(st, p)).toarray()
    a = O.stencil_to_csr(st)
    b = rng.uniform(-1, 1, 31 * 31)
    x = rng.uniform(-1, 1, 31 * 31)
    r = b - a @ x
    x2 = x + p @ np.linalg.solve(ac, p.T @ r)
    rr = p.T @ (b - a @ x2)
    assert np.abs(rr).max() <= 1e-12 * np.abs(p.T @ r).max()


# ---------------------------------------------------------------------------
# Coarsest direct solve
# ---------------------------------------------------------------------------

def test_cholesky_matches_lapack():
    rng = np.random.default_rng(4)
    h = O.setup(inputs.block_field(rng, 31, 31, 4, -4, 4))
    a0 = O.stencil_to_csr(h.levels[0].st).toarray()
    np.testing.assert_allclose(h.chol, np.linalg.cholesky(a0), rtol=1e-13, atol=1e-13 * np.abs(a0).max())
    b = rng.uniform(-1, 1, a0.shape[0])
    np.testing.assert_allclose(O.cholesky_solve(h.chol, b), np.linalg.solve(a0, b), rtol=1e-11)


# ---------------------------------------------------------------------------
# Smoother and V-cycle (Algorithm 1)
# ---------------------------------------------------------------------------

def _gs_loop(st, x, b, order, reverse=False):
    """Pointwise Gauss-Seidel visiting colours in order and, inside a colour,
    the points in reverse lexicographic order (any in-colour order must give
    the same result because same-coloured points do not couple)."""
    ny, nx = x.shape
    seq = list(reversed(order)) if reverse else list(order)
    for colour in seq:
        pts = [(j, i) for j in range(ny) for i in range(nx) if (j % 2, i % 2) in colour]
        for (j, i) in reversed(pts):
            s = b[j, i]
            for d, (di, dj) in O.OFFSETS.items():
                jj, ii = j + dj, i + di
                if 0 <= jj < ny and 0 <= ii < nx:
                    s += st[d][j, i] * x[jj, ii]
            x[j, i] = s / st["C"][j, i]


@pytest.mark.parametrize("nine_point", [False, True])
def test_multicolour_gs_matches_pointwise_loop(nine_point):
    rng = np.random.default_rng(12)
    k = 10.0 ** rng.uniform(-2, 2, size=(15, 15))
    h = O.setup(k)
    st = h.levels[-2].st if nine_point else h.levels[-1].st
    order = O.colour_order(st)
    assert order == (O.FOUR_ORDER if nine_point else O.RB_ORDER)
    ny, nx = st["C"].shape
    b = rng.uniform(-1, 1, (ny, nx))
    x0 = rng.uniform(-1, 1, (ny, nx))
    for reverse in (False, True):
        x1 = x0.copy()
        O.relax(st, x1, b, 1, order, reverse=reverse)
        x2 = x0.copy()
        _gs_loop(st, x2, b, order, reverse=reverse)
        np.testing.assert_allclose(x1, x2, rtol=1e-14, atol=1e-15)


def test_gs_is_gauss_seidel_not_jacobi():
    """The second colour must see the first colour's new values: one red
    sweep then one black sweep differs from a Jacobi update."""
    rng = np.random.default_rng(1)
    st = O.assemble_fv5(np.ones((7, 7)))
    b = rng.uniform(-1, 1, (7, 7))
    x = np.zeros((7, 7))
    O.relax(st, x, b, 1, O.RB_ORDER)
    red = np.add.outer(np.arange(7), np.arange(7)) % 2 == 0
    np.testing.assert_allclose(x[red], b[red] / st["C"][red], rtol=1e-15)
    assert not np.allclose(x[~red], b[~red] / st["C"][~red])


@pytest.mark.parametrize("n", [7, 15, 31])
def test_vcycle_converges_to_direct_solution(n):
    rng = np.random.default_rng(100 + n)
    k = 10.0 ** rng.uniform(-2, 2, size=(n, n))
    b = rng.uniform(-1, 1, (n, n))
    h = O.setup(k)
    res = O.solve(h, b, tol=1e-13, max_cycles=400)
    assert res.converged
    xd = O.direct_solve(k, b)
    assert np.abs(res.x - xd).max() <= 1e-10 * np.abs(xd).max()


def test_rectangular_grid_solves():
    rng = np.random.default_rng(21)
    k = 10.0 ** rng.uniform(-1, 1, size=(15, 63))
    b = rng.uniform(-1, 1, (15, 63))
    h = O.setup(k)
    assert [lv.shape for lv in h.levels] == [(3, 15), (7, 31), (15, 63)]
    res = O.solve(h, b, tol=1e-12)
    assert res.converged
    assert np.abs(res.x - O.direct_solve(k, b)).max() <= 1e-9 * np.abs(res.x).max()


def test_poisson_vcycle_rate_is_textbook():
    """V(2,1) with red-black GS on the 5-point Poisson problem contracts the
    residual by roughly an order of magnitude per cycle."""
    pr = inputs.constant_problem(127)
    h = O.setup(pr["k"])
    res = O.solve(h, pr["b"], tol=1e-10)
    assert res.converged and res.cycles <= 13
    rates = np.array(res.history[2:]) / np.array(res.history[1:-1])
    assert rates.max() < 0.2


def test_residual_term_variant_converges_and_differs():
    rng = np.random.default_rng(8)
    k = 10.0 ** rng.uniform(-1, 1, size=(31, 31))
    b = rng.uniform(-1, 1, (31, 31))
    r0 = O.solve(O.setup(k), b, tol=1e-11)
    r1 = O.solve(O.setup(k, interp_residual_term=True), b, tol=1e-11)
    assert r0.converged and r1.converged
    assert r0.history[1] != r1.history[1]
    np.testing.assert_allclose(r0.x, r1.x, rtol=0, atol=1e-9 * np.abs(r0.x).max())


def test_zero_rhs_and_bad_input():
    h = O.setup(np.ones((7, 7)))
    res = O.solve(h, np.zeros((7, 7)))
    assert res.cycles == 0 and res.rel_resid == 0.0
    with pytest.raises(ValueError):
        O.setup(np.ones((1, 7)))          # a side needs at least 2 cells
    with pytest.raises(ValueError):
        O.setup(-np.ones((7, 7)))
    k = np.ones((7, 7))
    k[3, 3] = np.nan
    with pytest.raises(ValueError):
        O.setup(k)


# ---------------------------------------------------------------------------
# Adjoint gradient
# ---------------------------------------------------------------------------

def test_adjoint_gradient_matches_central_differences():
    rng = np.random.default_rng(13)
    n = 8
    theta = rng.normal(0.0, 1.0, (n, n))
    b = rng.uniform(-1, 1, (n, n))
    u_obs = O.direct_solve(np.exp(theta + 0.1 * rng.normal(size=(n, n))), b)
    g, _, _ = O.adjoint_gradient(theta, b, u_obs)
    eps = 1e-6
    fd = np.zeros_like(theta)
    for j in range(n):
        for i in range(n):
            tp = theta.copy()
            tm = theta.copy()
            tp[j, i] += eps
            tm[j, i] -= eps
            fd[j, i] = (O.loss(tp, b, u_obs) - O.loss(tm, b, u_obs)) / (2 * eps)
    assert np.abs(fd - g).max() <= 1e-6 * np.abs(g).max()


def test_compliance_identity():
    """For L = b^T u the adjoint is u itself, so dL/dtheta_c =
    -k_c sum_f da_f/dk_c (u_c - u_n)^2 (- 2 k_c u_c^2 per boundary face): all
    entries are <= 0; check against central differences."""
    rng = np.random.default_rng(14)
    n = 6
    theta = rng.normal(0.0, 1.0, (n, n))
    b = rng.uniform(-1, 1, (n, n))
    u = O.direct_solve(np.exp(theta), b)
    g = O.assembly_vjp(np.exp(theta), u, u)
    assert np.all(g <= 0)
    eps = 1e-6
    for (j, i) in [(0, 0), (2, 3), (5, 1), (3, 3)]:
        tp = theta.copy()
        tm = theta.copy()
        tp[j, i] += eps
        tm[j, i] -= eps
        fd = (b.ravel() @ O.direct_solve(np.exp(tp), b).ravel()
              - b.ravel() @ O.direct_solve(np.exp(tm), b).ravel()) / (2 * eps)
        assert abs(fd - g[j, i]) <= 1e-6 * np.abs(g).max()


# ---------------------------------------------------------------------------
# Reading for non-M-matrix Galerkin rows (lumping before collapsing)
# ---------------------------------------------------------------------------

def test_collapse_is_identity_on_m_matrix_rows():
    rng = np.random.default_rng(41)
    st = O.assemble_fv5(10.0 ** rng.uniform(-4, 4, size=(15, 15)))
    cs = O.collapse_stencil(st)
    for d in ("C",) + O.DIRS:
        assert np.array_equal(cs[d], st[d]), d


def test_lumped_rows_keep_constants_and_bounded_weights():
    """A 9-point operator whose rows have zero row sum but some positive
    off-diagonal matrix entries (a_X < 0): lumping keeps the interpolation of
    constants exact (interior P rows sum to 1) and the weights in [0, 1]."""
    rng = np.random.default_rng(42)
    n = 15
    st = {d: np.zeros((n, n)) for d in ("C",) + O.DIRS}
    for d in O.DIRS:
        st[d] = rng.uniform(0.2, 1.0, (n, n))
    st["SW"] = rng.uniform(-0.3, 0.3, (n, n))          # mixed-sign corners
    # symmetric partners
    st["E"][:, :-1] = st["W"][:, 1:]
    st["N"][:-1, :] = st["S"][1:, :]
    st["NE"][:-1, :-1] = st["SW"][1:, 1:]
    st["SE"][1:, :-1] = st["NW"][:-1, 1:]
    for d, (di, dj) in O.OFFSETS.items():               # no coupling out of the grid
        if di < 0:
            st[d][:, 0] = 0
        if di > 0:
            st[d][:, -1] = 0
        if dj < 0:
            st[d][0, :] = 0
        if dj > 0:
            st[d][-1, :] = 0
    st["C"] = sum(st[d] for d in O.DIRS)               # zero row sums
    assert (st["SW"] < 0).any()
    p = O.interpolation(st)
    assert p.data.min() >= 0.0 and p.data.max() <= 1.0 + 1e-15
    s = np.asarray(p.sum(axis=1)).reshape(n, n)
    np.testing.assert_allclose(s[2:-2, 2:-2], 1.0, atol=1e-13)


def test_high_contrast_galerkin_levels_stay_interpolable():
    """Blocks of 10^[-4,4] narrower than a coarse cell make the Galerkin
    operators lose the M-matrix property; every interpolation weight must
    still lie in [0, 1] on every level."""
    pr = inputs.block_problem(255, seed=1, block=16, lo=-4, hi=4)
    h = O.setup(pr["k"])
    saw_negative = False
    for l in range(1, h.nlevels):
        st = h.levels[l].st
        saw_negative |= any((st[d] < 0).any() for d in O.DIRS)
        p = h.levels[l].p
        assert p.data.min() >= 0.0 and p.data.max() <= 1.0 + 1e-12, l
    assert saw_negative


# ---------------------------------------------------------------------------
# Conjugate gradients preconditioned by one symmetric V-cycle
# ---------------------------------------------------------------------------

def _one_d_operator(n):
    """The 1-D cell-centred Dirichlet operator of unit coefficient: 2 on the
    diagonal, 3 at both ends (a boundary face carries 2k), -1 off it."""
    t = np.diag(np.full(n, 2.0)) - np.diag(np.ones(n - 1), 1) - np.diag(np.ones(n - 1), -1)
    t[0, 0] = t[-1, -1] = 3.0
    return t


def test_cg_converges_in_as_many_steps_as_distinct_eigenvalues():
    # For k = 1 the 5-point operator is the Kronecker sum T (+) T, whose
    # eigenvectors are v_i (x) v_j with eigenvalues mu_i + mu_j.  Conjugate
    # gradients from x = 0 on a right-hand side with components along three
    # eigenvectors of three distinct eigenvalues is exact after three steps.
    n = 15
    mu, v = np.linalg.eigh(_one_d_operator(n))
    pairs = [(0, 0), (2, 5), (7, 11)]
    assert len({round(mu[i] + mu[j], 9) for i, j in pairs}) == 3
    b = sum((c * np.outer(v[:, j], v[:, i])) for c, (i, j) in zip((1.0, -0.5, 2.0), pairs))
    h = O.setup(np.ones((n, n)), nu1=1, nu2=1)
    r = O.pcg(h, b, tol=1e-13, max_iter=10, precond="identity")
    assert r.cycles == 3
    assert r.history[2] > 1e-3 and r.history[3] < 1e-12
    assert np.abs(O.apply(h.levels[-1].st, r.x) - b).max() < 1e-12 * np.abs(b).max()


def _block_field(n, seed):
    return inputs.block_problem(seed=seed, block=4, lo=-3, hi=3, nx=n, ny=n)


def test_symmetric_vcycle_preconditioner_is_symmetric_positive_definite():
    pr = _block_field(31, 11)
    rng = np.random.default_rng(12)
    u, w = rng.normal(size=(31, 31)), rng.normal(size=(31, 31))
    h = O.setup(pr["k"], nu1=1, nu2=1)
    mu, mw = O.vcycle_precond(h, u), O.vcycle_precond(h, w)
    scale = np.linalg.norm(u) * np.linalg.norm(mw)
    assert abs(np.sum(mu * w) - np.sum(u * mw)) <= 1e-13 * scale
    assert np.sum(mu * u) > 0 and np.sum(mw * w) > 0
    # V(2,1) is not symmetric: the same check fails by many orders of magnitude
    h21 = O.setup(pr["k"], nu1=2, nu2=1)
    z = np.zeros_like(u)
    O.vcycle(h21, z, u)
    z2 = np.zeros_like(w)
    O.vcycle(h21, z2, w)
    assert abs(np.sum(z * w) - np.sum(u * z2)) > 1e-6 * np.linalg.norm(u) * np.linalg.norm(z2)


@pytest.mark.parametrize("n", [15, 31])
def test_pcg_converges_to_direct_solution(n):
    pr = _block_field(n, 13)
    h = O.setup(pr["k"], nu1=1, nu2=1)
    r = O.pcg(h, pr["b"], tol=1e-12)
    xd = O.direct_solve(pr["k"], pr["b"])
    assert r.converged
    assert np.abs(r.x - xd).max() <= 1e-9 * np.abs(xd).max()
    # the updated residual tracks the true one
    rel_true = np.linalg.norm(O.residual(h.levels[-1].st, r.x, pr["b"])) / np.linalg.norm(pr["b"])
    assert rel_true <= 1e-11


def test_pcg_needs_fewer_iterations_than_vcycles_on_contrast():
    pr = inputs.block_problem(seed=1, block=8, lo=-4, hi=4, nx=63, ny=63)
    h = O.setup(pr["k"], nu1=1, nu2=1)
    rp = O.pcg(h, pr["b"], tol=1e-10)
    rv = O.solve(O.setup(pr["k"], nu1=1, nu2=1), pr["b"], tol=1e-10, max_cycles=2000)
    assert rp.converged and rv.converged
    assert rp.cycles < rv.cycles / 2


def test_pcg_rejects_unsymmetric_cycle():
    h = O.setup(np.ones((7, 7)), nu1=2, nu2=1)
    with pytest.raises(ValueError):
        O.pcg(h, np.ones((7, 7)))


# ---------------------------------------------------------------------------
# The paper's workload: D = diag(1/r, r) on stretched cells (Section 5)
# ---------------------------------------------------------------------------

def test_anisotropic_stretched_assembly_closed_form():
    # k = 1, r = 4, cells of aspect hy/hx = 2 on a 5 x 3 grid: x faces carry
    # (1/4) * 2 = 1/2, y faces 4 * (1/2) = 2; boundary faces twice that.
    st = O.assemble_fv5(np.ones((3, 5)), r=4.0, aspect=2.0)
    half, two = F(1, 2), F(2)
    for j in range(3):
        for i in range(5):
            w = half if i > 0 else 0
            e = half if i < 4 else 0
            s = two if j > 0 else 0
            n = two if j < 2 else 0
            bnd = (2 * half) * ((i == 0) + (i == 4)) + (2 * two) * ((j == 0) + (j == 2))
            assert st["W"][j, i] == w and st["E"][j, i] == e
            assert st["S"][j, i] == s and st["N"][j, i] == n
            assert st["C"][j, i] == w + e + s + n + bnd


def test_compensating_anisotropy_gives_an_isotropic_discrete_operator():
    # Section 5: with r equal to the cell aspect the couplings in x and y are
    # equal (the grid stretching is compensated), here with r = aspect = 16
    st = O.assemble_fv5(np.ones((7, 15)), r=16.0, aspect=16.0)
    assert np.all(st["W"][:, 1:] == 1.0) and np.all(st["S"][1:, :] == 1.0)
    iso = O.assemble_fv5(np.ones((7, 15)))
    for d in ("C", "W", "E", "S", "N"):
        assert np.array_equal(st[d], iso[d])


def test_anisotropic_stretched_assembly_is_second_order():
    # u = sin(pi x) sin(pi y) on the unit square, D = diag(1/r, r) with
    # r = 3, nx = 2 ny cells (aspect 2); b = f(x_c) hx hy, f = (1/r + r) pi^2 u
    r = 3.0
    errs = []
    for ny in (8, 16, 32):
        nx = 2 * ny
        hx, hy = 1.0 / nx, 1.0 / ny
        xc = (np.arange(nx) + 0.5) * hx
        yc = (np.arange(ny) + 0.5) * hy
        u = np.outer(np.sin(np.pi * yc), np.sin(np.pi * xc))
        b = (1.0 / r + r) * np.pi ** 2 * u * hx * hy
        st = O.assemble_fv5(np.ones((ny, nx)), r=r, aspect=nx / ny)
        uh = spla.spsolve(O.stencil_to_csr(st).tocsc(), b.ravel()).reshape(ny, nx)
        errs.append(np.abs(uh - u).max())
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.7


def test_paper_workload_vcycle_converges_like_poisson():
    # 255 x 15 cells of the unit square (aspect 17) with r = 17: the
    # compensating anisotropy keeps point-smoothed V(2,1) cycles fast
    rng = np.random.default_rng(21)
    b = rng.uniform(-1, 1, (15, 255))
    h = O.setup(np.ones((15, 255)), r=17.0, aspect=17.0)
    res = O.solve(h, b, tol=1e-10, max_cycles=100)
    assert res.converged and res.cycles <= 20
    # without the compensation (isotropic D on the same stretched cells) the
    # point smoother stalls
    h_iso = O.setup(np.ones((15, 255)), aspect=17.0)
    res_iso = O.solve(h_iso, b, tol=1e-10, max_cycles=100)
    assert res_iso.cycles > 3 * res.cycles



# ---------------------------------------------------------------------------
# General grid sizes (sides other than 2^m - 1)
# ---------------------------------------------------------------------------

def test_level_shapes_for_general_sides():
    assert O.level_shapes(16, 8) == [(16, 8), (8, 4), (4, 2)]
    assert O.level_shapes(100, 60) == [(100, 60), (50, 30), (25, 15), (12, 7), (6, 3)]
    assert O.level_shapes(255, 15) == [(255, 15), (127, 7), (63, 3)]
    assert O.level_shapes(3, 40) == [(3, 40)]


def test_coarsening_reproduces_the_papers_enumeration_example():
    """The paper's redistribution-enumeration example (Section 4) coarsens a
    9088 x 568 fine grid to a 1136 x 71 global coarse grid: three halvings
    of both sides.  Sides that are not of the form 2^m - 1 coarsen to
    floor(n / 2) here; (n - 1) / 2 would give 1135 x 70."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "coarsening_9088x568.txt")
    rows = [line.split() for line in open(path) if line.strip() and not line.startswith("#")]
    (fnx, fny, cnx, cny), = [tuple(int(v) for v in r) for r in rows]
    shapes = O.level_shapes(fnx, fny)
    assert shapes[3] == (cnx, cny)
    assert all(O.valid_size(n) for s in shapes for n in s)


@pytest.mark.parametrize("nx, ny", [(20, 13), (32, 32), (10, 6), (4, 4), (37, 18)])
def test_vcycle_converges_to_direct_solution_general_sides(nx, ny):
    rng = np.random.default_rng(nx * 100 + ny)
    k = 10.0 ** rng.uniform(-2, 2, size=(ny, nx))
    b = rng.uniform(-1, 1, (ny, nx))
    h = O.setup(k)
    for lv in h.levels[:-1]:
        st = lv.st
        scale = np.abs(st["C"]).max()
        assert np.allclose(st["W"][:, 1:], st["E"][:, :-1], rtol=0, atol=1e-13 * scale)
        assert np.allclose(st["SW"][1:, 1:], st["NE"][:-1, :-1], rtol=0, atol=1e-13 * scale)
        assert np.linalg.eigvalsh(O.stencil_to_csr(st).toarray()).min() > 0
    res = O.solve(h, b, tol=1e-13, max_cycles=400)
    assert res.converged
    xd = O.direct_solve(k, b)
    assert np.abs(res.x - xd).max() <= 1e-10 * np.abs(xd).max()


def test_poisson_rate_on_even_sides_is_grid_independent():
    rates = []
    for n in (32, 64, 128):
        rng = np.random.default_rng(n)
        h = O.setup(np.ones((n, n)))
        res = O.solve(h, rng.uniform(-1, 1, (n, n)), tol=1e-10, max_cycles=100)
        rates.append((res.history[-1] / res.history[0]) ** (1.0 / res.cycles))
    assert max(rates) < 0.3 and max(rates) - min(rates) < 0.05


# ---------------------------------------------------------------------------
# Neumann and Robin boundaries
# ---------------------------------------------------------------------------

def _mms_error(u_exact, f, bc, n):
    h = 1.0 / n
    xc = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(xc, xc)
    st = O.assemble_fv5(np.ones((n, n)), bc=bc)
    b = f(X, Y) * h * h
    uh = spla.spsolve(O.stencil_to_csr(st).tocsc(), b.ravel()).reshape(n, n)
    return np.abs(uh - u_exact(X, Y)).max()


def test_neumann_sides_are_second_order():
    # u = cos(pi x) sin(pi y): no flux through x = 0, 1; u = 0 at y = 0, 1
    u = lambda x, y: np.cos(np.pi * x) * np.sin(np.pi * y)  # noqa: E731
    f = lambda x, y: 2 * np.pi ** 2 * u(x, y)  # noqa: E731
    e = [_mms_error(u, f, (0.0, 0.0, None, None), n) for n in (16, 32, 64)]
    assert e[0] / e[1] > 3.7 and e[1] / e[2] > 3.8


def test_robin_sides_are_second_order():
    # u = g(x) sin(pi y), g = 1 + x - x^2, meets k du/dn + alpha u = 0 with
    # alpha = 1 at x = 0 and x = 1 (k = 1); beta = alpha * h
    g = lambda x: 1 + x - x * x  # noqa: E731
    u = lambda x, y: g(x) * np.sin(np.pi * y)  # noqa: E731
    f = lambda x, y: (2 + np.pi ** 2 * g(x)) * np.sin(np.pi * y)  # noqa: E731
    e = []
    for n in (16, 32, 64):
        e.append(_mms_error(u, f, (1.0 / n, 1.0 / n, None, None), n))
    assert e[0] / e[1] > 3.7 and e[1] / e[2] > 3.8


def test_boundary_face_limits_and_closed_form():
    k = np.ones((3, 4))
    d = O.assemble_fv5(k)
    n = O.assemble_fv5(k, bc=(0.0, None, None, None))
    big = O.assemble_fv5(k, bc=(1e300, None, None, None))
    # Neumann removes the wall face (2 k) from the west column's diagonal
    assert np.array_equal(n["C"][:, 0], d["C"][:, 0] - 2.0)
    assert np.array_equal(n["C"][:, 1:], d["C"][:, 1:])
    # beta -> infinity is the Dirichlet face
    assert np.allclose(big["C"], d["C"], rtol=1e-15, atol=0)
    # beta = 2 with k = 1: 2 * 2 / (2 + 2) = 1
    rb = O.assemble_fv5(k, bc=(None, 2.0, None, None))
    assert np.array_equal(rb["C"][:, -1], d["C"][:, -1] - 1.0)
    with pytest.raises(ValueError):
        O.assemble_fv5(k, bc=(0.0, 0.0, 0.0, 0.0))
    with pytest.raises(ValueError):
        O.assemble_fv5(k, bc=(-1.0, None, None, None))


@pytest.mark.parametrize("bc", [(0.0, 0.0, None, 0.5), (None, 0.0, 0.0, 0.0), (0.1, 2.0, 0.0, None)])
def test_vcycle_with_mixed_boundaries_converges_to_direct_solution(bc):
    rng = np.random.default_rng(61)
    k = 10.0 ** rng.uniform(-2, 2, size=(31, 31))
    b = rng.uniform(-1, 1, (31, 31))
    h = O.setup(k, bc=bc)
    res = O.solve(h, b, tol=1e-13, max_cycles=400)
    a = O.stencil_to_csr(O.assemble_fv5(k, bc=bc)).tocsc()
    xd = spla.spsolve(a, b.ravel()).reshape(31, 31)
    assert res.converged
    assert np.abs(res.x - xd).max() <= 1e-9 * np.abs(xd).max()


# ---------------------------------------------------------------------------
# Zebra line Gauss-Seidel (Section 2: alternating line smoothing for
# anisotropic problems)
# ---------------------------------------------------------------------------

def _line_sets(nx, ny, direction, colour):
    """Unknown indices (j * nx + i) of the lines of one colour."""
    idx = np.arange(nx * ny).reshape(ny, nx)
    return (idx[colour::2, :] if direction == "x" else idx[:, colour::2]).ravel()


def _dense_block_gs(st, x, b, smoother, reverse):
    """Block Gauss-Seidel with the lines of one colour as one block, by dense
    linear algebra: x_I = A_II^{-1} (b_I - A_I,rest x_rest)."""
    ny, nx = x.shape
    a = O.stencil_to_csr(st).toarray()
    seq = [(d, c) for d in smoother for c in (0, 1)]
    if reverse:
        seq = seq[::-1]
    xv, bv = x.ravel().copy(), b.ravel()
    for d, c in seq:
        idx = _line_sets(nx, ny, d, c)
        rest = np.setdiff1d(np.arange(nx * ny), idx)
        rhs = bv[idx] - a[np.ix_(idx, rest)] @ xv[rest]
        xv[idx] = np.linalg.solve(a[np.ix_(idx, idx)], rhs)
    return xv.reshape(ny, nx)


@pytest.mark.parametrize("smoother", ["x", "y", "xy"])
@pytest.mark.parametrize("nine_point", [False, True])
def test_line_relaxation_is_dense_block_gauss_seidel(smoother, nine_point):
    """One line sweep equals block Gauss-Seidel by dense solves, on a 5-point
    fine operator and on a 9-point Galerkin level of a rectangular grid, in
    both directions of traversal."""
    rng = np.random.default_rng(40)
    k = 10.0 ** rng.uniform(-2, 2, size=(13, 18))
    h = O.setup(k, r=3.0, aspect=0.5)
    st = h.levels[-2].st if nine_point else h.levels[-1].st
    assert O.is_five_point(st) != nine_point
    ny, nx = st["C"].shape
    b = rng.uniform(-1, 1, (ny, nx))
    x0 = rng.uniform(-1, 1, (ny, nx))
    for reverse in (False, True):
        x1 = x0.copy()
        O.relax_lines(st, x1, b, 1, smoother, reverse=reverse)
        x2 = _dense_block_gs(st, x0, b, smoother, reverse)
        np.testing.assert_allclose(x1, x2, rtol=1e-12, atol=1e-13 * np.abs(x2).max())


@pytest.mark.parametrize("direction", ["x", "y"])
def test_line_relaxation_zeroes_the_residual_of_the_last_colour(direction):
    """After a zebra sweep the equations of every line of the colour solved
    last hold exactly; those of the first colour do not."""
    rng = np.random.default_rng(41)
    k = 10.0 ** rng.uniform(-3, 3, size=(16, 11))
    st = O.setup(k).levels[-2].st
    ny, nx = st["C"].shape
    b = rng.uniform(-1, 1, (ny, nx))
    x = rng.uniform(-1, 1, (ny, nx))
    O.relax_lines(st, x, b, 1, direction)
    r = O.residual(st, x, b)
    last = (slice(1, None, 2), slice(None)) if direction == "x" else (slice(None), slice(1, None, 2))
    first = (slice(0, None, 2), slice(None)) if direction == "x" else (slice(None), slice(0, None, 2))
    assert np.abs(r[last]).max() <= 1e-13 * np.abs(b).max() * 10
    assert np.abs(r[first]).max() > 1e-3


def test_line_relaxation_solves_decoupled_lines_exactly():
    """With no coupling between rows one x-line sweep is an exact solve (a
    set of independent 1D problems); a y-line sweep of the transposed
    problem likewise."""
    rng = np.random.default_rng(42)
    ny, nx = 6, 9
    a = rng.uniform(0.5, 2.0, (ny, nx + 1))
    st = {d: np.zeros((ny, nx)) for d in ("C",) + O.DIRS}
    st["W"][:, 1:] = a[:, 1:nx]
    st["E"][:, :-1] = a[:, 1:nx]
    st["C"] = st["W"] + st["E"] + a[:, :nx] * 0.5 + 0.1
    b = rng.uniform(-1, 1, (ny, nx))
    xd = spla.spsolve(O.stencil_to_csr(st).tocsc(), b.ravel()).reshape(ny, nx)
    x = rng.uniform(-1, 1, (ny, nx))
    O.relax_lines(st, x, b, 1, "x")
    np.testing.assert_allclose(x, xd, rtol=1e-13, atol=1e-14)
    stt = {"C": st["C"].T, "S": st["W"].T, "N": st["E"].T, "W": st["S"].T, "E": st["N"].T,
           "SW": st["SW"].T, "NE": st["NE"].T, "SE": st["NW"].T, "NW": st["SE"].T}
    xt = rng.uniform(-1, 1, (nx, ny))
    O.relax_lines(stt, xt, b.T.copy(), 1, "y")
    np.testing.assert_allclose(xt, xd.T, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("r", [0.01, 100.0])
def test_line_smoothing_in_the_strong_direction_restores_convergence(r):
    """D = diag(1/r, r) on square cells: with r = 0.01 the x couplings are
    10^4 times the y couplings.  Point Gauss-Seidel with full coarsening
    stalls; lines along the strong direction (and alternating lines) give
    the textbook rate; lines across it stall like points."""
    rng = np.random.default_rng(43)
    n = 63
    b = rng.uniform(-1, 1, (n, n))
    k = np.ones((n, n))
    strong, weak = ("x", "y") if r < 1 else ("y", "x")
    cycles = {}
    for sm in O.SMOOTHERS:
        res = O.solve(O.setup(k, nu1=1, nu2=1, r=r, smoother=sm), b, tol=1e-10, max_cycles=60)
        cycles[sm] = res.cycles if res.converged else None
    assert cycles[strong] is not None and cycles[strong] <= 8
    assert cycles["xy"] is not None and cycles["xy"] <= 8
    assert cycles["point"] is None and cycles[weak] is None


def test_line_smoothed_preconditioner_is_symmetric_and_pcg_converges():
    """With nu1 = nu2 the post-smoothing runs the pre-smoothing's lines in
    reverse, so the V-cycle is a symmetric preconditioner; PCG with it
    reaches the direct solution."""
    pr = _block_field(31, 14)
    rng = np.random.default_rng(44)
    u, w = rng.normal(size=(31, 31)), rng.normal(size=(31, 31))
    h = O.setup(pr["k"], nu1=1, nu2=1, r=4.0, smoother="xy")
    mu, mw = O.vcycle_precond(h, u), O.vcycle_precond(h, w)
    scale = np.linalg.norm(u) * np.linalg.norm(mw)
    assert abs(np.sum(mu * w) - np.sum(u * mw)) <= 1e-13 * scale
    assert np.sum(mu * u) > 0
    res = O.pcg(h, pr["b"], tol=1e-12)
    xd = spla.spsolve(O.stencil_to_csr(O.assemble_fv5(pr["k"], r=4.0)).tocsc(),
                      pr["b"].ravel()).reshape(31, 31)
    assert res.converged
    assert np.abs(res.x - xd).max() <= 1e-9 * np.abs(xd).max()


def test_line_smoothed_vcycle_on_general_sides_and_robin_walls():
    """Line smoothing on even sides with Robin and Neumann walls reaches the
    direct solution."""
    rng = np.random.default_rng(45)
    nx, ny = 20, 14
    k = 10.0 ** rng.uniform(-1, 1, (ny, nx))
    b = rng.uniform(-1, 1, (ny, nx))
    bc = (0.0, 2.0, None, 0.5)
    h = O.setup(k, r=0.2, aspect=2.0, bc=bc, smoother="xy")
    res = O.solve(h, b, tol=1e-12)
    xd = spla.spsolve(O.stencil_to_csr(O.assemble_fv5(k, 0.2, 2.0, bc)).tocsc(),
                      b.ravel()).reshape(ny, nx)
    assert res.converged
    assert np.abs(res.x - xd).max() <= 1e-9 * np.abs(xd).max()


def test_bad_smoother_rejected():
    with pytest.raises(ValueError):
        O.setup(np.ones((7, 7)), smoother="z")
