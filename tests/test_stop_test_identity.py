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


def _three_d():
    from oracle import boxmg3d_oracle as O3
    rng = np.random.default_rng(21)
    nx, ny, nz = 11, 9, 7
    kb = 10.0 ** rng.uniform(-2, 2, (3, 3, 3))
    k = np.repeat(np.repeat(np.repeat(kb, 4, 0), 4, 1), 4, 2)[:nz, :ny, :nx]
    h = O3.setup(k)
    return O3, h, rng


def test_3d_stop_test_identities():
    """The 3D V-cycle's stop test inside the next fine sweep (k3_gs_norm):
    after a reverse red-black sweep colour 0 is unchanged by its update, and
    C (x_new - x_old) over colour 1 has the norm of b - A x."""
    O3, h, rng = _three_d()
    lv = h.levels[-1]
    a, shape = lv.a, lv.shape
    n = a.shape[0]
    b = rng.uniform(-1, 1, n)
    x = rng.uniform(-1, 1, n)
    O3.relax(a, shape, x, b, 2)
    O3.relax(a, shape, x, b, 1, reverse=True)
    col, nc = O3.colours(shape, True)
    diag = a.diagonal()
    off = (a - O3.sp.diags(diag)).tocsr()
    s0, s1 = np.nonzero(col == 0)[0], np.nonzero(col == 1)[0]
    assert np.array_equal(x[s0], (b[s0] - off[s0] @ x) / diag[s0])
    y1 = (b[s1] - off[s1] @ x) / diag[s1]
    r = b - a @ x
    fused = np.linalg.norm(diag[s1] * (y1 - x[s1]))
    assert abs(fused - np.linalg.norm(r)) <= 1e-12 * np.linalg.norm(r)


def test_3d_zero_start_terms_per_colour():
    """A forward eight-colour sweep of a 27-point (Galerkin) level from
    x = 0 equals the sweep in which colour c uses only the neighbours of
    colours before it -- 0, 2, 6, 8, 18, 20, 24, 26 of the 26 for c = 0..7,
    the kernel's zero_term3 rule."""
    O3, h, rng = _three_d()
    lv = h.levels[-2]
    a, shape = lv.a, lv.shape
    n = a.shape[0]
    b = rng.uniform(-1, 1, n)
    x = np.zeros(n)
    O3.relax(a, shape, x, b, 1)
    col, nc = O3.colours(shape, False)
    assert nc == 8
    diag = a.diagonal()
    off = (a - O3.sp.diags(diag)).tocoo()
    y = np.zeros(n)
    counts = []
    for c in range(8):
        s = np.nonzero(col == c)[0]
        keep = (col[off.row] == c) & (col[off.col] < c)
        part = O3.sp.csr_matrix((off.data[keep], (off.row[keep], off.col[keep])), shape=off.shape)
        y[s] = (b[s] - part[s] @ y) / diag[s]
        # the largest number of terms one point of colour c keeps
        counts.append(int(np.diff(part.tocsr().indptr)[s].max()) if s.size else 0)
    assert np.allclose(x, y, rtol=0, atol=0)
    assert counts == [0, 2, 6, 8, 18, 20, 24, 26]
