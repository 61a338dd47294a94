"""The redundant-halo tiling of the multicolour Gauss-Seidel sweep, on CPU.

The GPU sweeps (the TMA-staged kernel and the tiled kernel) relax each tile
once per sweep: colour phase k is updated on the tile grown by (gx_k, gy_k)
cells from old values staged with nc halo columns and 2 halo rows, and only
the tile's own points are written.  The growth follows from which
sub-lattices a later colour reads (x offset +-1 iff the column parities
differ, y offset +-1 iff the row parities differ):

  red-black (5-point):              (1, 1), (0, 0)
  four colours (0,0),(0,1),(1,0),(1,1) of (row, column) parities, and the
  reverse order (9-point):          (3, 1), (2, 1), (1, 0), (0, 0)

This model of the tiling reproduces the oracle's plain multicolour sweep
bit for bit (same per-point operations in the same order) on ragged grids;
every read it makes lies inside the staged box; a growth one cell too small
anywhere gives different values.
"""
import numpy as np
import pytest

from oracle import boxmg_oracle as O


def growth(nc, k):
    """(gx, gy) of colour phase k of nc, as in the kernels."""
    gx = nc - 1 - k
    gy = (1 if k < 2 else 0) if nc == 4 else nc - 1 - k
    return gx, gy


def random_stencil(nx, ny, nine, seed):
    rng = np.random.default_rng(seed)
    st = {d: np.zeros((ny, nx)) for d in O.DIRS}
    for d in O.DIRS if nine else ("W", "E", "S", "N"):
        st[d] = rng.uniform(0.1, 1.0, (ny, nx))
    st["C"] = sum(st[d] for d in O.DIRS) + rng.uniform(0.5, 1.0, (ny, nx))
    return st


def tiled_sweep(st, x, b, order, tx, ty, grow, halo_x, halo_y):
    """One sweep, tile by tile, each tile from the old iterate only."""
    ny, nx = x.shape
    nc = len(order)
    out = np.zeros_like(x)
    for j0 in range(0, ny, ty):
        for i0 in range(0, nx, tx):
            # staged box: the old iterate, zero outside the domain
            box = {}
            for j in range(j0 - halo_y, j0 + ty + halo_y):
                for i in range(i0 - halo_x, i0 + tx + halo_x):
                    box[(i, j)] = x[j, i] if 0 <= i < nx and 0 <= j < ny else 0.0
            for k, colour in enumerate(order):
                gx, gy = grow(nc, k)
                for j in range(j0 - gy, j0 + ty + gy):
                    for i in range(i0 - gx, i0 + tx + gx):
                        if not (0 <= i < nx and 0 <= j < ny) or (j % 2, i % 2) not in colour:
                            continue
                        s = b[j, i]
                        for d in O.DIRS:
                            di, dj = O.OFFSETS[d]
                            s = s + st[d][j, i] * box[(i + di, j + dj)]   # KeyError: not staged
                        box[(i, j)] = s / st["C"][j, i]
            for j in range(j0, min(j0 + ty, ny)):
                for i in range(i0, min(i0 + tx, nx)):
                    out[j, i] = box[(i, j)]
    return out


CASES = [  # (nx, ny, tile x, tile y)
    (23, 19, 8, 4), (17, 13, 12, 2), (9, 30, 4, 6), (40, 11, 16, 8),
]


@pytest.mark.parametrize("nine", [False, True])
@pytest.mark.parametrize("reverse", [False, True])
@pytest.mark.parametrize("nx, ny, tx, ty", CASES)
def test_tiled_sweep_equals_the_plain_sweep(nx, ny, tx, ty, nine, reverse):
    st = random_stencil(nx, ny, nine, seed=nx * ny + tx)
    rng = np.random.default_rng(ty)
    x = rng.uniform(-1, 1, (ny, nx))
    b = rng.uniform(-1, 1, (ny, nx))
    order = O.FOUR_ORDER if nine else O.RB_ORDER
    seq = tuple(reversed(order)) if reverse else tuple(order)
    nc = len(order)
    got = tiled_sweep(st, x, b, seq, tx, ty, growth, halo_x=nc, halo_y=2)
    ref = x.copy()
    O.relax(st, ref, b, 1, order, reverse=reverse)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("nine", [False, True])
def test_any_smaller_growth_breaks_the_sweep(nine):
    nx, ny, tx, ty = 23, 19, 8, 4
    st = random_stencil(nx, ny, nine, seed=5)
    rng = np.random.default_rng(6)
    x = rng.uniform(-1, 1, (ny, nx))
    b = rng.uniform(-1, 1, (ny, nx))
    order = O.FOUR_ORDER if nine else O.RB_ORDER
    nc = len(order)
    ref = x.copy()
    O.relax(st, ref, b, 1, order)
    for phase in range(nc):
        for axis in (0, 1):
            g = growth(nc, phase)
            if g[axis] == 0:
                continue

            def smaller(n, k, phase=phase, axis=axis):
                gx, gy = growth(n, k)
                if k == phase:
                    gx, gy = (gx - 1, gy) if axis == 0 else (gx, gy - 1)
                return gx, gy

            got = tiled_sweep(st, x, b, order, tx, ty, smaller, halo_x=nc, halo_y=2)
            assert not np.array_equal(got, ref), (phase, axis)
