"""Helpers shared by the GPU parity tests: the oracle side of each workload
(cached per process) and layout mapping between the oracle's matrices and
the library's exported planes.  No arithmetic of the method lives here."""
from __future__ import annotations

import functools

import numpy as np

from oracle import boxmg_oracle as O
from paper_1803_02481_gb300 import inputs

# name -> generator of {"k", "b"} (reduced-size stand-ins of the workloads,
# plus edge shapes: rectangular, smallest, random per-cell)
PROBLEMS = {
    "poisson255": lambda: inputs.constant_problem(255, seed=0),
    "blocks255": lambda: inputs.block_problem(255, seed=1, block=64, lo=-4, hi=4),
    "blocks511_c2": lambda: inputs.block_problem(511, seed=1, block=64, lo=-2, hi=2),
    "lognormal255": lambda: inputs.lognormal_problem(255, seed=2),
    "random63": lambda: {"k": 10.0 ** np.random.default_rng(7).uniform(-2, 2, (63, 63)),
                         "b": np.random.default_rng(8).uniform(-1, 1, (63, 63))},
    "rect127x31": lambda: inputs.block_problem(seed=5, block=8, lo=-3, hi=3, nx=127, ny=31),
    "wide2047x127": lambda: inputs.block_problem(seed=6, block=64, lo=-2, hi=2, nx=2047, ny=127),
    "tiny3": lambda: {"k": np.array([[1.0, 2.0, 3.0], [4.0, 5.0, 6.0], [7.0, 8.0, 9.0]]),
                      "b": np.array([[1.0, -1.0, 0.5], [0.25, 2.0, -3.0], [1.0, 1.0, 1.0]])},
}


@functools.lru_cache(maxsize=None)
def problem(name):
    return PROBLEMS[name]()


@functools.lru_cache(maxsize=None)
def oracle_hierarchy(name):
    return O.setup(problem(name)["k"])


@functools.lru_cache(maxsize=None)
def oracle_solve(name, tol=1e-10):
    return O.solve(oracle_hierarchy(name), problem(name)["b"], tol=tol, max_cycles=400)


def stencil_scale(st):
    """Per-entry scale for stencil comparisons: the larger of the entry and
    the diagonal of its row (off-diagonals can be tiny under 10^8 contrast)."""
    return st["C"]


def interp_planes(p, nxf, nyf):
    """Oracle P (CSR, fine x coarse) in the library's 8-plane layout.
    Returns (planes, valid) with planes[k][J, I] for 0 <= I <= ncx,
    0 <= J <= ncy; valid marks entries whose fine point exists and whose
    coarse target is interior."""
    ncx, ncy = nxf // 2, nyf // 2
    J, I = np.meshgrid(np.arange(ncy + 1), np.arange(ncx + 1), indexing="ij")
    # (fine dx, fine dy, coarse dI, coarse dJ) per plane, fine point
    # (2I + fx, 2J + fy) and coarse target (I + cx, J + cy), 1-based
    spec = [(1, 0, 0, 0), (1, 0, 1, 0), (0, 1, 0, 0), (0, 1, 0, 1),
            (1, 1, 0, 0), (1, 1, 1, 0), (1, 1, 0, 1), (1, 1, 1, 1)]
    planes = np.zeros((8, ncy + 1, ncx + 1))
    valid = np.zeros((8, ncy + 1, ncx + 1), dtype=bool)
    csr = p.tocsr()
    for k, (fx, fy, cx, cy) in enumerate(spec):
        fi, fj = 2 * I + fx, 2 * J + fy
        ci, cj = I + cx, J + cy
        ok = (fi >= 1) & (fi <= nxf) & (fj >= 1) & (fj <= nyf) & (ci >= 1) & (ci <= ncx) \
            & (cj >= 1) & (cj <= ncy)
        f = ((fj - 1) * nxf + (fi - 1))[ok]
        c = ((cj - 1) * ncx + (ci - 1))[ok]
        planes[k][ok] = np.asarray(csr[f, c]).ravel()
        valid[k] = ok
    return planes, valid


def nine_from_five(planes):
    """The library's symmetric 5-plane export (C, W, S, SW, NW) as the
    oracle's 9-plane stencil: E(i,j) = W(i+1,j), N(i,j) = S(i,j+1),
    NE(i,j) = SW(i+1,j+1), SE(i,j) = NW(i+1,j-1)."""
    st = {d: np.array(planes[d], dtype=np.float64) for d in ("C", "W", "S", "SW", "NW")}
    ny, nx = st["C"].shape
    st["E"] = np.zeros((ny, nx))
    st["E"][:, :-1] = st["W"][:, 1:]
    st["N"] = np.zeros((ny, nx))
    st["N"][:-1, :] = st["S"][1:, :]
    st["NE"] = np.zeros((ny, nx))
    st["NE"][:-1, :-1] = st["SW"][1:, 1:]
    st["SE"] = np.zeros((ny, nx))
    st["SE"][1:, :-1] = st["NW"][:-1, 1:]
    return st
