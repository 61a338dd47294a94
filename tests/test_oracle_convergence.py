"""Why the 4095^2 block field converges slowly: per-level two-grid rates.

The 4095^2 field has 64 x 64 blocks of k = 10^U, U ~ uniform[-4, 4].  A
scaled model with the same structure (64 blocks per side, the same contrast)
is a 511^2 grid with 8-cell blocks; on it every level's two-grid rate can be
measured on the CPU.  Each rate is the asymptotic A-norm contraction of one
two-grid cycle (nu1 = 2 forward Gauss-Seidel sweeps, exact coarse solve on
the Galerkin level, nu2 = 1 reversed sweep) by power iteration from a
random error.

Measured facts this file keeps true:
* while a coefficient block spans at least four coarse cells the two-grid
  rate is that of Poisson (about 0.15); at two cells it degrades (about
  0.6), and once a block is one coarse cell or narrower it is about 0.95;
* with contrast 10^+-1 instead of 10^+-4 every level stays below 0.35;
* the lumping of non-M-matrix rows before the collapse (the oracle's reading
  of the unstated BoxMG heuristics) does not cause the slow levels: the
  rates without it are the same to within 0.05.
So the slow V-cycle on the full field comes from its coarse levels, where a
coarse cell covers several blocks of 10^8 contrast, not from the lumping.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import boxmg_oracle as O
from paper_1803_02481_gb300 import inputs

N, BLOCK = 511, 8


def two_grid_rate(st, p, stc, nu1=2, nu2=1, iters=25, seed=0):
    """A-norm contraction per two-grid cycle (geometric mean of the last 10
    of `iters` power-iteration steps); the coarse solve is a sparse LU."""
    a = O.stencil_to_csr(st)
    lu = spla.splu(O.stencil_to_csr(stc).tocsc())
    ny, nx = st["C"].shape
    e = np.random.default_rng(seed).uniform(-1, 1, (ny, nx))
    zero = np.zeros((ny, nx))
    order = O.colour_order(st)
    norms = []
    for _ in range(iters):
        O.relax(st, e, zero, nu1, order)              # b = 0: x is the error
        r = -(a @ e.ravel())
        e += (p @ lu.solve(p.T @ r)).reshape(ny, nx)
        O.relax(st, e, zero, nu2, order, reverse=True)
        n = np.sqrt(e.ravel() @ (a @ e.ravel()))
        norms.append(n)
        e /= n
    return float(np.exp(np.mean(np.log(norms[-10:]))))


def level_rates(lo, hi, lump=True):
    """[(level side, coarse cells per block, two-grid rate)] from fine to
    coarse for the scaled model with contrast 10^U(lo, hi)."""
    k = inputs.block_problem(N, seed=1, block=BLOCK, lo=lo, hi=hi)["k"]
    saved = O.collapse_stencil
    if not lump:
        O.collapse_stencil = lambda st: st            # the plain collapse
    try:
        h = O.setup(k)
    finally:
        O.collapse_stencil = saved
    out = []
    for l in range(h.nlevels - 1, 0, -1):
        st = h.levels[l].st
        side = st["C"].shape[1]
        out.append((side, BLOCK * (side + 1) / (N + 1), two_grid_rate(st, h.levels[l].p, h.levels[l - 1].st)))
    return out


@pytest.fixture(scope="module")
def rates_high():
    return level_rates(-4, 4)


def test_two_grid_rates_degrade_where_blocks_are_narrower_than_coarse_cells(rates_high):
    for side, span, rate in rates_high:
        if span >= 4:
            assert rate <= 0.2, (side, span, rate)
        elif span >= 2:
            assert 0.4 <= rate <= 0.75, (side, span, rate)
        elif span >= 0.25:
            assert rate >= 0.9, (side, span, rate)


def test_low_contrast_keeps_every_level_fast():
    for side, span, rate in level_rates(-1, 1):
        assert rate <= 0.35, (side, span, rate)


def test_lumping_is_not_the_cause(rates_high):
    plain = level_rates(-4, 4, lump=False)
    for (side, span, r1), (_, _, r0) in zip(rates_high, plain):
        assert abs(r1 - r0) <= 0.05, (side, r1, r0)
