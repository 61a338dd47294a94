"""CPU stand-in for one rank's part of the domain-decomposed solve, for the
multi-rank tests on `gloo` (test infrastructure only; the product path is
the CUDA part).  It holds the same blocks with a one-point ring as the CUDA
part and applies the oracle's per-point arithmetic to them: the Gauss-Seidel
update and the residual accumulate the neighbour terms in the oracle's
direction order, with E, N, NE, SE taken from the neighbours' W, S, SW, NW
(the symmetric storage of the C ABI).  Also the oracle-side adapters: the
global source of the block planes and rank 0's coarse cycle."""
from __future__ import annotations

import numpy as np
import torch

from oracle import boxmg_oracle as O
from paper_1803_02481_gb300.dd import EAST, NORTH, SOUTH, VB, VR, VX, WEST
from tests.parity_helpers import interp_planes

OFF = O.OFFSETS


class OracleSource:
    """level_stencil / level_interp / vcycle_from over an oracle hierarchy,
    with the C ABI's plane conventions."""

    def __init__(self, h):
        self.h = h

    @property
    def nlevels(self):
        return self.h.nlevels

    def level_shape(self, l):
        ny, nx = self.h.levels[l].shape
        return nx, ny

    def level_stencil(self, l):
        st = self.h.levels[l].st
        return {key: st[key] for key in ("C", "W", "S", "SW", "NW")}

    def level_interp(self, l):
        ny, nx = self.h.levels[l].shape
        planes, _ = interp_planes(self.h.levels[l].p, nx, ny)
        return dict(zip(("XW", "XE", "YS", "YN", "CSW", "CSE", "CNW", "CNE"), planes))

    def vcycle_from(self, level, b, x):
        sub = O.Hierarchy(levels=self.h.levels[:level + 1], chol=self.h.chol, nu1=self.h.nu1,
                          nu2=self.h.nu2)
        xx = np.zeros(tuple(b.shape))
        O.vcycle(sub, xx, b.numpy())
        x.copy_(torch.from_numpy(xx))
        return x


class CpuPart:
    torch = torch
    device = torch.device("cpu")

    def __init__(self, payload):
        self.dims = payload["dims"]
        self.nine = payload["nine"]
        n = len(self.dims)
        self.vec = [{v: np.zeros((ny + 2, nx + 2)) for v in (VX, VB, VR)} for nx, ny in self.dims]
        self.st, self.p = [None] * n, [None] * n
        for k in range(1, n):
            planes = payload["stencils"][k]
            st = dict(zip(("C", "W", "S", "SW", "NW"), planes))
            # E(i,j) = W(i+1,j), N(i,j) = S(i,j+1), NE = SW(i+1,j+1), SE = NW(i+1,j-1)
            for d in ("E", "N", "NE", "SE"):
                st[d] = np.zeros_like(st["C"])
            st["E"][:, :-1] = st["W"][:, 1:]
            st["N"][:-1, :] = st["S"][1:, :]
            st["NE"][:-1, :-1] = st["SW"][1:, 1:]
            st["SE"][1:, :-1] = st["NW"][:-1, 1:]
            self.st[k] = st
            self.p[k] = dict(zip(("XW", "XE", "YS", "YN", "CSW", "CSE", "CNW", "CNE"), payload["interps"][k]))

    # -- the arithmetic of one block ------------------------------------------
    def _nbr(self, a, j, i, d):
        di, dj = OFF[d]
        return a[j + dj, i + di]

    def relax_colour(self, k, c):
        nx, ny = self.dims[k]
        st, x, b = self.st[k], self.vec[k][VX], self.vec[k][VB]
        subs = (((0, 0), (1, 1)), ((0, 1), (1, 0)))[c] if not self.nine[k] else (((0, 0),), ((0, 1),),
                                                                                  ((1, 0),), ((1, 1),))[c]
        for pj, pi in subs:
            jj = np.arange(1 + pj, ny + 1, 2)
            ii = np.arange(1 + pi, nx + 1, 2)
            if jj.size == 0 or ii.size == 0:
                continue
            J, I = np.meshgrid(jj, ii, indexing="ij")
            s = b[J, I].copy()
            for d in O.DIRS:
                di, dj = OFF[d]
                s += st[d][J, I] * x[J + dj, I + di]
            x[J, I] = s / st["C"][J, I]

    def residual(self, k):
        nx, ny = self.dims[k]
        st, x, b = self.st[k], self.vec[k][VX], self.vec[k][VB]
        J, I = np.meshgrid(np.arange(1, ny + 1), np.arange(1, nx + 1), indexing="ij")
        y = st["C"][J, I] * x[J, I]
        for d in O.DIRS:
            di, dj = OFF[d]
            y = y - st[d][J, I] * x[J + dj, I + di]
        self.vec[k][VR][J, I] = b[J, I] - y

    def restrict(self, k):
        nxc, nyc = self.dims[k - 1]
        r, P = self.vec[k][VR], self.p[k]
        bc, xc = self.vec[k - 1][VB], self.vec[k - 1][VX]
        Jc, Ic = np.meshgrid(np.arange(1, nyc + 1), np.arange(1, nxc + 1), indexing="ij")
        f, g = 2 * Jc, 2 * Ic
        acc = r[f, g].copy()
        acc += P["XE"][Jc, Ic - 1] * r[f, g - 1] + P["XW"][Jc, Ic] * r[f, g + 1]
        acc += P["YN"][Jc - 1, Ic] * r[f - 1, g] + P["YS"][Jc, Ic] * r[f + 1, g]
        acc += P["CNE"][Jc - 1, Ic - 1] * r[f - 1, g - 1] + P["CNW"][Jc - 1, Ic] * r[f - 1, g + 1]
        acc += P["CSE"][Jc, Ic - 1] * r[f + 1, g - 1] + P["CSW"][Jc, Ic] * r[f + 1, g + 1]
        bc[1:nyc + 1, 1:nxc + 1] = acc
        xc[1:nyc + 1, 1:nxc + 1] = 0.0

    def interp(self, k):
        nx, ny = self.dims[k]
        x, xc, P = self.vec[k][VX], self.vec[k - 1][VX], self.p[k]
        for pj in (0, 1):
            for pi in (0, 1):
                jj = np.arange(2 - pj, ny + 1, 2)        # pj = 0: even j, 1: odd j
                ii = np.arange(2 - pi, nx + 1, 2)
                if jj.size == 0 or ii.size == 0:
                    continue
                j, i = np.meshgrid(jj, ii, indexing="ij")
                J, I = j >> 1, i >> 1
                if not pi and not pj:
                    v = xc[J, I]
                elif not pi:
                    v = P["YS"][J, I] * xc[J, I] + P["YN"][J, I] * xc[J + 1, I]
                elif not pj:
                    v = P["XW"][J, I] * xc[J, I] + P["XE"][J, I] * xc[J, I + 1]
                else:
                    v = (P["CSW"][J, I] * xc[J, I] + P["CSE"][J, I] * xc[J, I + 1]
                         + P["CNW"][J, I] * xc[J + 1, I] + P["CNE"][J, I] * xc[J + 1, I + 1])
                x[j, i] += v

    def norms(self, k):
        nx, ny = self.dims[k]
        r = self.vec[k][VR][1:ny + 1, 1:nx + 1]
        b = self.vec[k][VB][1:ny + 1, 1:nx + 1]
        return float((r * r).sum()), float((b * b).sum())

    # -- data movement --------------------------------------------------------
    def buffer(self, n):
        return torch.empty(n, dtype=torch.float64)

    def strip_len(self, k, side):
        nx, ny = self.dims[k]
        return ny if side in (WEST, EAST) else nx + 2

    def _strip(self, k, vec, side, get):
        nx, ny = self.dims[k]
        a = self.vec[k][vec]
        if side == WEST:
            return a[1:ny + 1, 1 if get else 0]
        if side == EAST:
            return a[1:ny + 1, nx if get else nx + 1]
        if side == SOUTH:
            return a[1 if get else 0, :]
        return a[ny if get else ny + 1, :]

    def get_strip(self, k, vec, side, buf):
        buf.copy_(torch.from_numpy(np.ascontiguousarray(self._strip(k, vec, side, True))))

    def put_strip(self, k, vec, side, buf):
        self._strip(k, vec, side, False)[...] = buf.numpy()

    def get_block(self, k, vec, ring=False):
        nx, ny = self.dims[k]
        a = self.vec[k][vec]
        return torch.from_numpy(np.ascontiguousarray(a if ring else a[1:ny + 1, 1:nx + 1]))

    def put_block(self, k, vec, t, ring=False):
        nx, ny = self.dims[k]
        a = self.vec[k][vec]
        if ring:
            a[...] = t.numpy()
        else:
            a[1:ny + 1, 1:nx + 1] = t.numpy()
