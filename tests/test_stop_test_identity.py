"""The exactness arguments behind two shortcuts of the GPU cycle -- the stop
test taken inside the next sweep, and the zero-start form of a sweep from
x = 0 -- checked with the oracle's own Gauss-Seidel arithmetic on CPU.

After a sweep in reverse colour order, nothing else touching x:
* the colour updated last satisfies its update exactly: recomputing that
  colour from the unchanged neighbours gives the same bits, so the next
  forward sweep's first colour is a no-op;
* the second colour of that next sweep then changes each of its points by
  r / C, r the residual b - A x of the iterate before the sweep (the first
  colour's residual being zero in that evaluation), so C (x_new - x_old)
  summed in squares over the second colour is ||b - A x||^2 up to rounding.
On a 9-point (four-colour) level the first property holds for the last
colour too.  The same identities are what the GPU sweeps use."""
import numpy as np
import pytest

from oracle import boxmg_oracle as O
from paper_1803_02481_gb300 import inputs


def _level(name):
    if name == "five":
        pr = inputs.block_problem(63, seed=11, block=8, lo=-3, hi=3)
        st = O.assemble_fv5(pr["k"])
        b = pr["b"]
    else:
        h = O.setup(inputs.block_problem(63, seed=12, block=8, lo=-2, hi=2)["k"])
        st = h.levels[-2].st                      # a Galerkin (9-point) level
        b = np.random.default_rng(13).uniform(-1, 1, st["C"].shape)
    return st, b


@pytest.mark.parametrize("name", ["five", "nine"])
def test_first_colour_after_a_reverse_sweep_is_a_no_op(name):
    st, b = _level(name)
    order = O.colour_order(st)
    x = np.random.default_rng(1).uniform(-1, 1, b.shape)
    O.relax(st, x, b, 1, order)
    O.relax(st, x, b, 1, order, reverse=True)     # ends with order[0]
    y = x.copy()
    O.relax(st, y, b, 1, [order[0]])
    assert np.array_equal(x, y)
    # a colour that was not updated last does change
    z = x.copy()
    O.relax(st, z, b, 1, [order[1]])
    assert not np.array_equal(x, z)


def test_second_colour_update_carries_the_residual():
    st, b = _level("five")
    order = O.colour_order(st)
    x = np.random.default_rng(2).uniform(-1, 1, b.shape)
    O.relax(st, x, b, 2, order)
    O.relax(st, x, b, 1, order, reverse=True)
    r = O.residual(st, x, b)
    y = x.copy()
    O.relax(st, y, b, 1, [order[1]])               # the second colour of the next sweep
    fused = np.linalg.norm(st["C"] * (y - x))
    exact = np.linalg.norm(r)
    assert abs(fused - exact) <= 1e-12 * exact
    # the residual at the first colour is zero to rounding, not by structure
    mask = np.zeros(b.shape, dtype=bool)
    for (pj, pi) in order[0]:
        mask[pj::2, pi::2] = True
    assert np.abs(r[mask]).max() <= 1e-12 * np.abs(r).max()


def _colour_of(order, pj, pi):
    for k, colour in enumerate(order):
        if (pj, pi) in colour:
            return k
    raise AssertionError((pj, pi))


@pytest.mark.parametrize("name", ["five", "nine"])
def test_zero_start_sweep_needs_only_the_colours_before(name):
    """A forward sweep from x = 0 (each coarse level's first pre-sweep) gives
    the same values when colour k applies only the neighbour terms of the
    colours updated before it: the zero-start form of the GPU sweeps (four
    colours: 0, 2, 6 and 8 of the 8 terms; two colours: 0 and 4)."""
    st, b = _level(name)
    order = O.colour_order(st)
    x = np.zeros_like(b)
    O.relax(st, x, b, 1, order)
    y = np.zeros_like(b)
    ny, nx = b.shape
    counts = []
    for k, colour in enumerate(order):
        yp = np.pad(y, 1)
        for (pj, pi) in colour:
            rows, cols = slice(pj, None, 2), slice(pi, None, 2)
            s = b[rows, cols].copy()
            used = 0
            for d in O.DIRS:
                di, dj = O.OFFSETS[d]
                if _colour_of(order, (pj + dj) % 2, (pi + di) % 2) < k:
                    s += st[d][rows, cols] * O.shifted(yp, d, ny, nx, rows, cols)
                    used += 1 if np.any(st[d]) else 0
            y[rows, cols] = s / st["C"][rows, cols]
        counts.append(used)
    assert np.array_equal(x, y)
    assert counts == ([0, 2, 6, 8] if name == "nine" else [0, 4])
