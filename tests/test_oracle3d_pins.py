"""Pins of the 3D CPU oracle against what the mathematics fixes: closed
forms, manufactured solutions, exact trilinear weights, flux-ratio weights in
layered media, Galerkin symmetry and pattern, two-grid orthogonality, a
brute-force Gauss-Seidel loop and convergence to the direct solution."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import boxmg3d_oracle as O3


def test_assembly_constant_k_closed_form():
    """k = 1: interior C = 6; a boundary face adds 2 in place of a neighbour's
    1 (face cell 7, edge cell 8, corner cell 9); off-diagonals -1."""
    n = 5
    a = O3.assemble_fv7(np.ones((n, n, n)))
    d = a.diagonal().reshape(n, n, n)
    assert d[2, 2, 2] == 6.0 and d[0, 2, 2] == 7.0 and d[0, 0, 2] == 8.0 and d[0, 0, 0] == 9.0
    off = a.toarray() - np.diag(a.diagonal())
    assert set(np.unique(off)) <= {0.0, -1.0}
    assert np.count_nonzero(off[(2 * n + 2) * n + 2]) == 6
    assert abs(a - a.T).max() == 0


def _mms_error(n, k_of_x):
    h = 1.0 / n
    c = (np.arange(n) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    k = k_of_x(x)
    u = np.sin(2 * np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z) / k
    f = 6 * np.pi ** 2 * np.sin(2 * np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
    a = O3.assemble_fv7(k)
    uh = spla.spsolve(a.tocsc(), (h * h * f).ravel()).reshape(n, n, n)
    return np.abs(uh - u).max() / np.abs(u).max()


@pytest.mark.parametrize("layered", [False, True])
def test_assembly_is_second_order(layered):
    """u = sin(2 pi x) sin(pi y) sin(pi z) / k(x) solves -div(k grad u) =
    6 pi^2 sin(2 pi x) sin(pi y) sin(pi z) for k constant and for k jumping
    at x = 1/2 (u = 0 and the flux continuous there); harmonic faces give
    O(h^2) in both cases."""
    kf = (lambda x: np.where(x < 0.5, 1.0, 50.0)) if layered else (lambda x: np.ones_like(x))
    e = [_mms_error(n, kf) for n in (8, 16, 32)]
    for e0, e1 in zip(e, e[1:]):
        assert 3.4 < e0 / e1 < 4.6


def test_interpolation_is_trilinear_at_constant_k():
    """Constant k, 2^m - 1 sides: injection 1 at coarse points, 1/2 at edge
    points, 1/4 at face points, 1/8 at cell centres, exactly; every row of an
    interior fine point sums to 1."""
    n = 15
    shape = (n, n, n)
    a = O3.assemble_fv7(np.ones((n, n, n)))
    p = O3.interpolation(a, shape)
    for f in range(n ** 3):
        k, rem = divmod(f, n * n)
        j, i = divmod(rem, n)
        between = (i % 2 == 0) + (j % 2 == 0) + (k % 2 == 0)
        row = p.getrow(f)
        vals = row.data
        interior = 0 < i < n - 1 and 0 < j < n - 1 and 0 < k < n - 1
        if interior:
            assert len(vals) == 2 ** between
            assert np.all(vals == 0.5 ** between), (i, j, k, vals)
            assert abs(vals.sum() - 1.0) < 1e-15


def test_interpolation_weights_are_flux_ratios_in_layered_media():
    """k varying in x only: an x-edge point's weights are the 1D flux ratios
    a_W / (a_W + a_E), a_E / (a_W + a_E) of its harmonic face coefficients.
    The oracle forms the denominator as C minus the four transverse
    couplings, which cancels terms up to C / (a_W + a_E) times larger than
    the result: the tolerance is a few ulp of that ratio."""
    rng = np.random.default_rng(3)
    n = 15
    kx = 10.0 ** rng.uniform(-3, 3, n)
    k = np.broadcast_to(kx, (n, n, n)).copy()
    a = O3.assemble_fv7(k)
    p = O3.interpolation(a, (n, n, n))
    hm = lambda u, v: 2 * u * v / (u + v)  # noqa: E731
    for (i, j, kk) in [(2, 5, 7), (8, 3, 9), (12, 11, 1)]:
        f = (kk * n + j) * n + i
        aw, ae = hm(kx[i - 1], kx[i]), hm(kx[i], kx[i + 1])
        row = p.getrow(f)
        cols, vals = row.indices, row.data
        c = (n - 1) // 2
        lo = (((kk - 1) // 2) * c + (j - 1) // 2) * c + (i - 2) // 2     # coarse (i-1)
        hi = lo + 1
        got = dict(zip(cols, vals))
        cdiag = a[f, f]
        rtol = 8 * np.finfo(float).eps * cdiag / (aw + ae)
        np.testing.assert_allclose(got[lo], aw / (aw + ae), rtol=rtol)
        np.testing.assert_allclose(got[hi], ae / (aw + ae), rtol=rtol)


def _block_k(shape, seed, block=4, lo=-2, hi=2):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    nb = [-(-s // block) for s in (nz, ny, nx)]
    kb = 10.0 ** rng.uniform(lo, hi, nb)
    return np.repeat(np.repeat(np.repeat(kb, block, 0), block, 1), block, 2)[:nz, :ny, :nx]


@pytest.mark.parametrize("shape", [(15, 15, 15), (31, 15, 7), (12, 9, 7)])
def test_galerkin_is_symmetric_27_point_with_zero_interior_row_sums(shape):
    """Symmetric 27-point coarse operators.  P reproduces constants wherever
    the fine rows have zero row sums, so coarse rows away from the walls sum
    to zero; checked on 2^m - 1 sides (next to an even side the last fine
    line folds the wall's Dirichlet face into its weights, as in 2D)."""
    k = _block_k(shape, 4)
    h = O3.setup(k)
    odd = all((s + 1) & s == 0 for s in shape)
    for l in range(len(h.levels) - 1):
        a = h.levels[l].a
        assert abs(a - a.T).max() <= 1e-12 * abs(a).max()
        nx, ny, nz = h.levels[l].shape
        rs = np.asarray(a.sum(axis=1)).ravel().reshape(nz, ny, nx)
        inner = rs[1:-1, 1:-1, 1:-1]
        if odd and inner.size:
            assert np.abs(inner).max() <= 1e-11 * abs(a).max()
    # the first coarse level is a full 27-point stencil somewhere
    a1 = h.levels[-2].a
    assert a1.getnnz(axis=1).max() == 27


def test_two_grid_galerkin_orthogonality():
    """After an exact coarse correction the residual is orthogonal to the
    range of P: P^T (b - A (x + P A_c^{-1} P^T r)) = 0."""
    shape = (11, 9, 8)
    k = _block_k(shape, 5)
    a = O3.assemble_fv7(k)
    p = O3.interpolation(a, shape)
    ac = O3.galerkin(a, p, tuple(O3.coarse_size(s) for s in shape))
    rng = np.random.default_rng(6)
    b = rng.normal(size=a.shape[0])
    x = rng.normal(size=a.shape[0])
    r = b - a @ x
    x2 = x + p @ spla.spsolve(ac.tocsc(), p.T @ r)
    assert np.abs(p.T @ (b - a @ x2)).max() <= 1e-11 * np.abs(p.T @ r).max()


def _gs_loop(a, shape, x, b, reverse):
    nx, ny, nz = shape
    col, nc = O3.colours(shape, O3.is_seven_point(a, shape))
    order = range(nc - 1, -1, -1) if reverse else range(nc)
    ad = a.toarray()
    for c in order:
        for p in range(len(x)):
            if col[p] != c:
                continue
            s = b[p]
            for q in range(len(x)):
                if q != p:
                    s -= ad[p, q] * x[q]
            x[p] = s / ad[p, p]


@pytest.mark.parametrize("level", [-1, -2])
def test_multicolour_gs_matches_pointwise_loop(level):
    """Red-black on the 7-point level and eight colours on a 27-point level
    equal a point-by-point Gauss-Seidel loop in colour order."""
    k = _block_k((7, 7, 7), 7)
    h = O3.setup(k)
    lev = h.levels[level]
    rng = np.random.default_rng(8)
    n = lev.a.shape[0]
    b = rng.normal(size=n)
    x0 = rng.normal(size=n)
    for rev in (False, True):
        x1 = x0.copy()
        O3.relax(lev.a, lev.shape, x1, b, 1, reverse=rev)
        x2 = x0.copy()
        _gs_loop(lev.a, lev.shape, x2, b, rev)
        np.testing.assert_allclose(x1, x2, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("shape", [(7, 7, 7), (15, 15, 15), (12, 9, 7), (16, 5, 6)])
def test_vcycle_converges_to_direct_solution(shape):
    k = _block_k(shape, 9)
    nx, ny, nz = shape
    b = np.random.default_rng(10).uniform(-1, 1, (nz, ny, nx))
    h = O3.setup(k)
    res = O3.solve(h, b, tol=1e-12)
    xd = spla.spsolve(h.levels[-1].a.tocsc(), b.ravel()).reshape(nz, ny, nx)
    assert res.converged
    assert np.abs(res.x - xd).max() <= 1e-9 * np.abs(xd).max()


def test_poisson_vcycle_rate_is_textbook_and_grid_independent():
    """Constant k: the V(2,1) convergence factor is small and does not grow
    with the grid."""
    rates = []
    for n in (15, 31):
        b = np.random.default_rng(11).uniform(-1, 1, (n, n, n))
        res = O3.solve(O3.setup(np.ones((n, n, n))), b, tol=1e-10)
        hist = res.history
        rates.append((hist[-1] / hist[1]) ** (1.0 / (len(hist) - 2)))
    assert max(rates) < 0.2
    assert rates[1] < rates[0] + 0.05


def test_bad_input_rejected():
    with pytest.raises(ValueError):
        O3.setup(np.ones((1, 4, 4)))
    with pytest.raises(ValueError):
        O3.setup(-np.ones((4, 4, 4)))


def test_level_shapes_3d():
    """Sides n -> floor(n / 2) in every direction while the smallest side
    exceeds 3; 2^m - 1 sides keep that form down to 3 (the 255^3 benchmark
    hierarchy has 7 levels)."""
    assert O3.level_shapes(255, 255, 255) == [(n, n, n) for n in (255, 127, 63, 31, 15, 7, 3)]
    assert O3.level_shapes(45, 20, 70) == [(45, 20, 70), (22, 10, 35), (11, 5, 17), (5, 2, 8)]
    assert O3.level_shapes(12, 9, 7) == [(12, 9, 7), (6, 4, 3)]
    assert O3.level_shapes(3, 40, 40) == [(3, 40, 40)]
    with pytest.raises(ValueError):
        O3.level_shapes(1, 8, 8)


# ---------------------------------------------------------------------------
# Conjugate gradients preconditioned by one symmetric V-cycle (3D)
# ---------------------------------------------------------------------------

def _one_d_operator(n):
    """1-D cell-centred Dirichlet operator of unit coefficient: 2 on the
    diagonal, 3 at both ends (a boundary face carries 2k), -1 off it."""
    t = np.diag(np.full(n, 2.0)) - np.diag(np.ones(n - 1), 1) - np.diag(np.ones(n - 1), -1)
    t[0, 0] = t[-1, -1] = 3.0
    return t


def test_3d_cg_converges_in_as_many_steps_as_distinct_eigenvalues():
    # k = 1: the 7-point operator is the Kronecker sum T (+) T (+) T with
    # eigenvectors v_i (x) v_j (x) v_k and eigenvalues mu_i + mu_j + mu_k; CG
    # from x = 0 on a right-hand side along three eigenvectors of three
    # distinct eigenvalues is exact after three steps
    n = 7
    mu, v = np.linalg.eigh(_one_d_operator(n))
    triples = [(0, 0, 0), (1, 3, 2), (6, 4, 5)]
    assert len({round(mu[i] + mu[j] + mu[k], 9) for i, j, k in triples}) == 3
    b = sum(c * np.einsum("k,j,i->kji", v[:, k], v[:, j], v[:, i])
            for c, (i, j, k) in zip((1.0, -0.5, 2.0), triples))
    h = O3.setup(np.ones((n, n, n)), nu1=1, nu2=1)
    r = O3.pcg(h, b, tol=1e-13, max_iter=10, precond="identity")
    assert r.cycles == 3
    assert r.history[2] > 1e-3 and r.history[3] < 1e-12
    a = h.levels[-1].a
    assert np.abs(a @ r.x.ravel() - b.ravel()).max() < 1e-12 * np.abs(b).max()


def test_3d_symmetric_vcycle_preconditioner_is_symmetric_positive_definite():
    k = _block_k((15, 15, 15), 41, block=4, lo=-3, hi=3)
    rng = np.random.default_rng(42)
    u, w = rng.normal(size=15 ** 3), rng.normal(size=15 ** 3)
    h = O3.setup(k, nu1=1, nu2=1)
    mu, mw = O3.vcycle_precond(h, u), O3.vcycle_precond(h, w)
    scale = np.linalg.norm(u) * np.linalg.norm(mw)
    assert abs(mu @ w - u @ mw) <= 1e-13 * scale
    assert mu @ u > 0 and mw @ w > 0
    # V(2,1) is not symmetric: the same check fails by orders of magnitude
    h21 = O3.setup(k, nu1=2, nu2=1)
    z, z2 = np.zeros_like(u), np.zeros_like(w)
    O3.vcycle(h21, z, u)
    O3.vcycle(h21, z2, w)
    assert abs(z @ w - u @ z2) > 1e-6 * np.linalg.norm(u) * np.linalg.norm(z2)


@pytest.mark.parametrize("shape", [(7, 7, 7), (15, 12, 9)])
def test_3d_pcg_converges_to_direct_solution(shape):
    k = _block_k(shape, 43, block=3, lo=-3, hi=3)
    b = np.random.default_rng(44).uniform(-1, 1, k.shape)
    h = O3.setup(k, nu1=1, nu2=1)
    r = O3.pcg(h, b, tol=1e-12)
    a = h.levels[-1].a
    xd = spla.spsolve(a.tocsc(), b.ravel())
    assert r.converged
    assert np.abs(r.x.ravel() - xd).max() <= 1e-9 * np.abs(xd).max()
    # the recursively updated residual tracks the true one
    assert np.linalg.norm(b.ravel() - a @ r.x.ravel()) / np.linalg.norm(b) <= 1e-11


def test_3d_pcg_needs_fewer_iterations_than_vcycles_and_rejects_unsymmetric_cycle():
    k = _block_k((15, 15, 15), 45, block=4, lo=-4, hi=4)
    b = np.random.default_rng(46).uniform(-1, 1, k.shape)
    rp = O3.pcg(O3.setup(k, nu1=1, nu2=1), b, tol=1e-10)
    rv = O3.solve(O3.setup(k, nu1=1, nu2=1), b, tol=1e-10, max_cycles=2000)
    assert rp.converged and rv.converged and rp.cycles < rv.cycles
    with pytest.raises(ValueError):
        O3.pcg(O3.setup(k, nu1=2, nu2=1), b)
