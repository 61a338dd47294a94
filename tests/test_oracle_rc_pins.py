"""Pins of the oracle's optional r/C term in interpolate-and-correct.

Section 3 (following Dendy 2010) writes the correction as
u <- u + I u_c + r/C, where r is the residual computed before restriction
(after pre-smoothing) and C the fine diagonal; the edge and cell-centre
formulas carry the term, injection at coarse points does not.  Two
consequences of that definition, neither of which re-evaluates the cycle's
own arithmetic, pin the oracle's reading:

1. With exact coarse solves (two levels), no smoothing and an initial error
   in the range of P, the coarse-grid correction removes the error exactly
   (Galerkin A_c = P^T A P), so what is left is the r/C term alone:
   x1 - x* vanishes at coarse points and equals r0/C = (A e0)/C elsewhere.
2. For any number of levels, with nu2 = 0 the update minus r_pre/C at
   non-coarse points is P times the coarse correction, so it is interpolated
   exactly from its own values at the coarse points.

The negative controls plant plausible misreadings in a copy of the oracle's
cycle (checked to be bit-identical to it when nothing is planted) and show
that each one fails at least one pin.
"""
import numpy as np
import pytest

from oracle import boxmg_oracle as O
from paper_1803_02481_gb300 import inputs


def planted_vcycle(h, x, b, mistake=None):
    """The oracle's V-cycle with an optional planted misreading of the r/C
    term:
      'coarse_too'       r/C added at coarse points as well
      'after_correction' r taken after x += P x_c
      'before_smoothing' r taken before pre-smoothing
      'sign'             x -= r/C
      'edges_only'       r/C at edge points but not at cell centres
      'times_c'          r * C instead of r / C
    """
    nl = h.nlevels
    xs, bs, rs, r0s = [None] * nl, [None] * nl, [None] * nl, [None] * nl
    xs[nl - 1], bs[nl - 1] = x, b
    for l in range(nl - 1, 0, -1):
        lev = h.levels[l]
        r0s[l] = O.residual(lev.st, xs[l], bs[l])
        O.smooth(h, lev.st, xs[l], bs[l], h.nu1, reverse=False)
        rs[l] = O.residual(lev.st, xs[l], bs[l])
        nyc, nxc = h.levels[l - 1].shape
        bs[l - 1] = (lev.p.T @ rs[l].ravel()).reshape(nyc, nxc)
        xs[l - 1] = np.zeros((nyc, nxc))
    xs[0][:] = O.cholesky_solve(h.chol, bs[0].ravel()).reshape(xs[0].shape)
    for l in range(1, nl):
        lev = h.levels[l]
        corr = (lev.p @ xs[l - 1].ravel()).reshape(xs[l].shape)
        if h.interp_residual_term:
            r = rs[l]
            if mistake == "before_smoothing":
                r = r0s[l]
            elif mistake == "after_correction":
                r = O.residual(lev.st, xs[l] + corr, bs[l])
            c = lev.st["C"]
            rc = r * c if mistake == "times_c" else r / c
            if mistake != "coarse_too":
                rc[1::2, 1::2] = 0.0
            if mistake == "edges_only":
                rc[0::2, 0::2] = 0.0
            corr = corr + (-rc if mistake == "sign" else rc)
        xs[l] += corr
        O.smooth(h, lev.st, xs[l], bs[l], h.nu2, reverse=True)


MISTAKES = ("coarse_too", "after_correction", "before_smoothing", "sign", "edges_only", "times_c")


def two_level(k, nu1, nu2, rc=True):
    """A hierarchy of the fine level and its Galerkin coarse level only, so
    the coarse solve is exact (Cholesky)."""
    st = O.assemble_fv5(k)
    p = O.interpolation(st)
    stc = O.galerkin(st, p)
    chol = O.cholesky(O.stencil_to_csr(stc).toarray())
    return O.Hierarchy(levels=[O.Level(stc), O.Level(st, p)], chol=chol, nu1=nu1, nu2=nu2,
                       interp_residual_term=rc)


def coarse_mask(shape):
    m = np.zeros(shape, dtype=bool)
    m[1::2, 1::2] = True
    return m


def fields():
    rng = np.random.default_rng(31)
    return {"poisson": np.ones((31, 31)),
            "lognormal": np.exp(2.0 * inputs.gaussian_random_field(rng, 31, 31, 4.0)),
            "blocks": inputs.block_field(rng, 31, 31, 4, -3, 3)}


def pin_range_of_p(k, cycle):
    """Pin 1.  Returns (max |error| at coarse points, max |error - r0/C| at
    the other points, max |r0/C| there)."""
    rng = np.random.default_rng(5)
    h = two_level(k, nu1=0, nu2=0)
    st, p = h.levels[1].st, h.levels[1].p
    ny, nx = st["C"].shape
    a = O.stencil_to_csr(st)
    xstar = rng.uniform(-1, 1, ny * nx)
    v = rng.uniform(-1, 1, p.shape[1])
    e0 = p @ v
    b = (a @ xstar).reshape(ny, nx)
    x = (xstar - e0).reshape(ny, nx)
    cycle(h, x, b)
    # r0 = b - A x0 = A e0 and P^T r0 = A_c v, so the exact coarse solve
    # returns v and P v = e0: x1 = x0 + e0 + r0/C|_F = x* + r0/C|_F
    e1 = x - xstar.reshape(ny, nx)
    expected = (a @ e0).reshape(ny, nx) / st["C"]
    cm = coarse_mask((ny, nx))
    scale = np.abs(expected[~cm]).max()
    return np.abs(e1[cm]).max(), np.abs(e1[~cm] - expected[~cm]).max(), scale


def pin_interpolated_update(k, nlevels_two, cycle, nu1=1):
    """Pin 2.  Returns (max |y_F - (P y_C)_F|, scale of y) for
    y = x1 - x_pre - r_pre/C|_F."""
    rng = np.random.default_rng(6)
    if nlevels_two:
        h = two_level(k, nu1=nu1, nu2=0)
    else:
        h = O.setup(k, nu1=nu1, nu2=0, interp_residual_term=True)
    st, p = h.levels[-1].st, h.levels[-1].p
    ny, nx = st["C"].shape
    a = O.stencil_to_csr(st)
    b = rng.uniform(-1, 1, (ny, nx))
    x0 = rng.uniform(-1, 1, (ny, nx))
    x_pre = x0.copy()
    O.relax(st, x_pre, b, nu1, O.colour_order(st))
    r_pre = b - (a @ x_pre.ravel()).reshape(ny, nx)
    cm = coarse_mask((ny, nx))
    s_r = np.where(cm, 0.0, r_pre / st["C"])
    x1 = x0.copy()
    cycle(h, x1, b)
    y = x1 - x_pre - s_r
    yc = y[1::2, 1::2]
    py = (p @ yc.ravel()).reshape(ny, nx)
    return np.abs(y - py).max(), np.abs(y).max()


def test_planted_copy_is_the_oracle_cycle():
    """With nothing planted the test's copy computes the oracle's cycle bit
    for bit, so the negative controls below differ only by their mistake."""
    rng = np.random.default_rng(3)
    for name, k in fields().items():
        for h in (two_level(k, 2, 1), O.setup(k, interp_residual_term=True), O.setup(k)):
            b = rng.uniform(-1, 1, k.shape)
            x_a = rng.uniform(-1, 1, k.shape)
            x_b = x_a.copy()
            O.vcycle(h, x_a, b)
            planted_vcycle(h, x_b, b)
            assert np.array_equal(x_a, x_b), name


@pytest.mark.parametrize("name", ["poisson", "lognormal", "blocks"])
def test_rc_term_is_all_that_remains_of_an_error_in_range_of_p(name):
    k = fields()[name]
    ce, fe, scale = pin_range_of_p(k, O.vcycle)
    assert scale > 1e-3
    assert ce <= 1e-12 * scale          # coarse points: solved exactly
    assert fe <= 1e-12 * scale          # elsewhere: exactly r0/C


@pytest.mark.parametrize("name", ["poisson", "lognormal", "blocks"])
@pytest.mark.parametrize("nu1", [1, 2])
def test_update_minus_rc_term_is_an_interpolant(name, nu1):
    k = fields()[name]
    for two in (True, False):
        err, scale = pin_interpolated_update(k, two, O.vcycle, nu1)
        assert scale > 1e-3
        assert err <= 1e-12 * scale, (two, err, scale)


def test_update_minus_rc_term_is_an_interpolant_at_c1_size():
    """Pin 2 on the 255^2 Poisson problem and a 255^2 window of a log-normal
    field (seven levels, inexact coarse solves)."""
    rng = np.random.default_rng(2)
    for k in (np.ones((255, 255)), np.exp(2.0 * inputs.gaussian_random_field(rng, 255, 255, 32.0))):
        err, scale = pin_interpolated_update(k, False, O.vcycle)
        assert err <= 1e-12 * scale, (err, scale)


@pytest.mark.parametrize("mistake", MISTAKES)
def test_planted_misreadings_fail_a_pin(mistake):
    """Each misreading of the r/C term, planted in a copy of the oracle's
    cycle, breaks pin 1 or pin 2 on at least one field."""
    def cycle(h, x, b):
        planted_vcycle(h, x, b, mistake)

    broken = False
    for name, k in fields().items():
        ce, fe, scale = pin_range_of_p(k, cycle)
        if ce > 1e-12 * scale or fe > 1e-12 * scale:
            broken = True
        for two in (True, False):
            err, s = pin_interpolated_update(k, two, cycle)
            if err > 1e-12 * s:
                broken = True
    assert broken, mistake


def test_rc_variant_converges_to_the_direct_solution():
    """The r/C variant is a convergent iteration with the same fixed point:
    it reaches the direct solution on the three fields."""
    rng = np.random.default_rng(4)
    for name, k in fields().items():
        b = rng.uniform(-1, 1, k.shape)
        res = O.solve(O.setup(k, interp_residual_term=True), b, tol=1e-12, max_cycles=200)
        assert res.converged, name
        xd = O.direct_solve(k, b)
        assert np.abs(res.x - xd).max() <= 1e-9 * np.abs(xd).max(), name
