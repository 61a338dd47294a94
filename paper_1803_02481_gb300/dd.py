"""Domain-decomposed solve phase (Section 2.1) with coarse-grid
redistribution by agglomeration (Section 2.2, Algorithm 2).

The ranks form a px x py processor grid.  On each of the `dist_levels`
finest levels every rank owns one rectangular block of points and keeps it,
with a one-point ring of its neighbours' values (the width-1 halo), in a
part of the CUDA library (``bmg_dd_*``).  One V-cycle is Algorithm 2 with
p_l = px * py on the distributed levels and p_l = 1 below them:

* relax: one halo exchange of x before every colour, then the colour;
* residual: a halo exchange of x, r = b - A x;
* restriction: a halo exchange of r, b_{l-1} = P^T r (local otherwise);
* gather_rhs: every rank sends its block of the restricted right-hand side
  of the gather level to rank 0, which runs the rest of the cycle on the
  levels below with the library's single-GPU schedule;
* scatter_sol: rank 0 sends every rank its block of the coarse solution,
  ring included; then interpolation and post-smoothing climb back, with a
  halo exchange of the coarser x before each interpolation;
* the stop test adds the ranks' partial sums of r^2 and b^2 (allreduce).

A halo exchange runs in two phases, west/east (owned rows) and then
south/north (rows including the ring columns, which carry the corners).

Setup is centralised: rank 0 builds the global hierarchy (assembly,
operator-induced interpolation, Galerkin operators, coarsest factor) and
scatters to every rank the planes of its blocks, ring included.  Blocks start
at 0-based global indices that are multiples of 2^dist_levels, so the
colours, coarse points and restriction/interpolation offsets of a block are
those of the full level.

Every numerical step runs in the CUDA library; this module moves blocks
between ranks (``torch.distributed`` or, for several blocks on one GPU, the
in-process ``ThreadComm``) and orders the calls.
"""
from __future__ import annotations

import ctypes
import queue
import threading
from dataclasses import dataclass

import numpy as np

WEST, EAST, SOUTH, NORTH = 0, 1, 2, 3
VX, VB, VR = 0, 1, 2
STENCIL_KEYS = ("C", "W", "S", "SW", "NW")
INTERP_KEYS = ("XW", "XE", "YS", "YN", "CSW", "CSE", "CNW", "CNE")


# ---------------------------------------------------------------------------
# Layout: processor grid and blocks
# ---------------------------------------------------------------------------

def coarse_range(lo: int, hi: int):
    """Coarse points of a 1-based fine range: coarse point I is fine point 2I."""
    return (lo + 1) // 2, hi // 2


def split(n: int, p: int, align: int):
    """p contiguous 1-based ranges covering 1..n, each starting at a 0-based
    index that is a multiple of `align`, sizes as equal as alignment allows."""
    units = -(-n // align)
    if units < p:
        raise ValueError(f"{n} points cannot be split into {p} blocks aligned to {align}")
    base, extra = divmod(units, p)
    out, u = [], 0
    for r in range(p):
        lo = u * align + 1
        u += base + (1 if r < extra else 0)
        out.append((lo, min(u * align, n)))
    return out


@dataclass
class Layout:
    """Processor grid px x py over a hierarchy of `shapes` ((nx, ny) per
    level, coarsest first); the finest `dist_levels` levels are distributed,
    level L - 1 - dist_levels is the gather level."""
    shapes: list
    px: int
    py: int
    dist_levels: int

    def __post_init__(self):
        L = len(self.shapes)
        if not 1 <= self.dist_levels <= L - 1:
            raise ValueError(f"dist_levels must be in 1..{L - 1}")
        self.gather = L - 1 - self.dist_levels
        nxf, nyf = self.shapes[-1]
        align = 2 ** self.dist_levels
        self.xr = [split(nxf, self.px, align)]
        self.yr = [split(nyf, self.py, align)]
        for _ in range(self.dist_levels):        # finest first
            self.xr.append([coarse_range(*r) for r in self.xr[-1]])
            self.yr.append([coarse_range(*r) for r in self.yr[-1]])
        self.xr.reverse()                        # part level 0 = gather level
        self.yr.reverse()
        for k in range(self.dist_levels + 1):
            for lo, hi in self.xr[k] + self.yr[k]:
                if hi < lo:
                    raise ValueError("a block is empty on a distributed level; use fewer ranks or levels")

    @property
    def size(self):
        return self.px * self.py

    @property
    def nlev(self):
        return self.dist_levels + 1

    def coords(self, rank):
        return rank % self.px, rank // self.px

    def block(self, rank, k):
        """((i0, i1), (j0, j1)) 1-based owned ranges of rank on part level k."""
        a, b = self.coords(rank)
        return self.xr[k][a], self.yr[k][b]

    def neighbours(self, rank):
        a, b = self.coords(rank)
        nb = {}
        if a > 0:
            nb[WEST] = rank - 1
        if a < self.px - 1:
            nb[EAST] = rank + 1
        if b > 0:
            nb[SOUTH] = rank - self.px
        if b < self.py - 1:
            nb[NORTH] = rank + self.px
        return nb


def min_block_points(layout: Layout) -> int:
    """Fewest points any rank owns on the coarsest distributed level."""
    k = 1
    return min((i1 - i0 + 1) * (j1 - j0 + 1)
               for r in range(layout.size) for (i0, i1), (j0, j1) in [layout.block(r, k)])


def choose_dist_levels(shapes, px, py, min_local=1024):
    """Parallel coarsening continues while every rank keeps at least
    `min_local` points (the minimum local problem size of Section 2.2); the
    next coarser level is gathered to one rank.  Returns dist_levels."""
    best = 1
    for m in range(1, len(shapes)):
        try:
            lay = Layout(shapes, px, py, m)
        except ValueError:
            break
        if min_block_points(lay) < min_local:
            break
        best = m
    return best


def block_payload(source, layout: Layout, rank: int):
    """The planes rank needs: per part level k >= 1 the stencil of its block
    with ring (5, ny + 2, nx + 2) and the interpolation planes on the coarser
    block with ring (8, nyc + 2, nxc + 2); part level 0 has none."""
    stencils, interps, dims = [None], [None], []
    for k in range(layout.nlev):
        (i0, i1), (j0, j1) = layout.block(rank, k)
        dims.append((i1 - i0 + 1, j1 - j0 + 1))
        if k == 0:
            continue
        lvl = layout.gather + k
        st = source.level_stencil(lvl)
        pl = np.stack([np.pad(st[key], 1) for key in STENCIL_KEYS])
        stencils.append(np.ascontiguousarray(pl[:, j0 - 1:j1 + 2, i0 - 1:i1 + 2]))
        (I0, I1), (J0, J1) = layout.block(rank, k - 1)
        pi = source.level_interp(lvl)             # (ncy + 1, ncx + 1), index 0 = ring
        pp = np.stack([np.pad(pi[key], ((0, 1), (0, 1))) for key in INTERP_KEYS])
        interps.append(np.ascontiguousarray(pp[:, J0 - 1:J1 + 2, I0 - 1:I1 + 2]))
    return {"dims": dims, "stencils": stencils, "interps": interps,
            "nine": [0 if k == layout.nlev - 1 else 1 for k in range(layout.nlev)]}


# ---------------------------------------------------------------------------
# Communicators
# ---------------------------------------------------------------------------

class TorchComm:
    """torch.distributed process group (NCCL on GPUs, gloo on CPUs)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)

    def exchange(self, sends, recvs):
        ops = [self.dist.P2POp(self.dist.isend, t, dst, self.group) for dst, t in sends]
        ops += [self.dist.P2POp(self.dist.irecv, t, src, self.group) for src, t in recvs]
        if ops:
            for req in self.dist.batch_isend_irecv(ops):
                req.wait()

    def allreduce_sum(self, values, device):
        import torch
        t = torch.tensor(values, dtype=torch.float64, device=device)
        self.dist.all_reduce(t, group=self.group)
        return t.tolist()

    def scatter_object(self, objs):
        out = [None]
        self.dist.scatter_object_list(out, objs if self.rank == 0 else None, src=0, group=self.group)
        return out[0]


class PeerFailed(RuntimeError):
    """Another rank of the same ThreadHub failed; this one stopped waiting."""


class ThreadHub:
    """Shared state of `size` ThreadComm ranks living in one process."""

    def __init__(self, size, timeout=60.0):
        self.size = size
        self.q = {(s, d): queue.Queue() for s in range(size) for d in range(size)}
        self.barrier = threading.Barrier(size)
        self.slots = [None] * size
        self.failed = threading.Event()
        self.timeout = timeout

    def get(self, key):
        """Next message on a (src, dst) queue; gives up when a rank has
        failed or after `timeout` seconds."""
        waited = 0.0
        while True:
            if self.failed.is_set():
                raise PeerFailed("a peer rank failed")
            try:
                return self.q[key].get(timeout=0.05)
            except queue.Empty:
                waited += 0.05
                if waited > self.timeout:
                    raise TimeoutError(f"no message from rank {key[0]} to rank {key[1]}")


class ThreadComm:
    """Ranks as threads of one process (several blocks on one GPU, or CPU
    tests): messages are tensor copies through queues, ordered on the
    device stream the threads share, so no kernel ever waits for another."""

    def __init__(self, hub: ThreadHub, rank: int):
        self.hub, self.rank, self.size = hub, rank, hub.size

    def exchange(self, sends, recvs):
        for dst, t in sends:
            self.hub.q[(self.rank, dst)].put(t.clone())
        for src, t in recvs:
            t.copy_(self.hub.get((src, self.rank)))

    def allreduce_sum(self, values, device):
        try:
            self.hub.slots[self.rank] = list(values)
            self.hub.barrier.wait(timeout=self.hub.timeout)
            total = [sum(v[i] for v in self.hub.slots) for i in range(len(values))]
            self.hub.barrier.wait(timeout=self.hub.timeout)
        except threading.BrokenBarrierError:
            raise PeerFailed("a peer rank failed") from None
        return total

    def scatter_object(self, objs):
        if self.rank == 0:
            for d in range(1, self.size):
                self.hub.q[(0, d)].put(objs[d])
            return objs[0]
        return self.hub.get((0, self.rank))


def run_threads(size, fn, timeout=60.0):
    """Run fn(comm) on `size` ThreadComm ranks; returns the per-rank results.
    A rank that raises makes every other rank stop waiting (PeerFailed), and
    the first original error is re-raised."""
    hub = ThreadHub(size, timeout)
    res, err = [None] * size, [None] * size

    def body(r):
        try:
            res[r] = fn(ThreadComm(hub, r))
        except BaseException as e:  # noqa: BLE001 - reported below
            err[r] = e
            hub.failed.set()
            hub.barrier.abort()

    ts = [threading.Thread(target=body, args=(r,)) for r in range(size)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    for e in err:
        if e is not None and not isinstance(e, PeerFailed):
            raise e
    for e in err:
        if e is not None:
            raise e
    return res


# ---------------------------------------------------------------------------
# The CUDA part of one rank
# ---------------------------------------------------------------------------

class CudaPart:
    """One rank's blocks in the CUDA library (bmg_dd_part)."""

    def __init__(self, payload, device=None):
        import torch
        from . import _check, lib
        self.torch, self._check, self._lib = torch, _check, lib
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        dims = payload["dims"]
        n = len(dims)
        self.dims = dims
        nx = (ctypes.c_int * n)(*[d[0] for d in dims])
        ny = (ctypes.c_int * n)(*[d[1] for d in dims])
        nine = (ctypes.c_int * n)(*payload["nine"])
        self._keep = [np.ascontiguousarray(a, dtype=np.float64) if a is not None else None
                      for a in payload["stencils"] + payload["interps"]]
        st = [a.ctypes.data if a is not None else None for a in self._keep[:n]]
        ip = [a.ctypes.data if a is not None else None for a in self._keep[n:]]
        stp = (ctypes.c_void_p * n)(*st)
        ipp = (ctypes.c_void_p * n)(*ip)
        h = ctypes.c_void_p()
        _check(lib().bmg_dd_part_create(n, nx, ny, nine, stp, ipp, self._stream(), ctypes.byref(h)),
               "bmg_dd_part_create")
        self._h = h
        self._keep = None

    _h = None

    def _stream(self):
        return ctypes.c_void_p(self.torch.cuda.current_stream(self.device).cuda_stream)

    def destroy(self):
        if self._h:
            self._lib().bmg_dd_part_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def relax_colour(self, k, c):
        self._check(self._lib().bmg_dd_relax_colour(self._h, k, c, self._stream()), "bmg_dd_relax_colour")

    def residual(self, k):
        self._check(self._lib().bmg_dd_residual(self._h, k, self._stream()), "bmg_dd_residual")

    def restrict(self, k):
        self._check(self._lib().bmg_dd_restrict(self._h, k, self._stream()), "bmg_dd_restrict")

    def interp(self, k):
        self._check(self._lib().bmg_dd_interp(self._h, k, self._stream()), "bmg_dd_interp")

    def norms(self, k):
        out = (ctypes.c_double * 2)()
        self._check(self._lib().bmg_dd_norms(self._h, k, out, self._stream()), "bmg_dd_norms")
        return out[0], out[1]

    def buffer(self, n):
        return self.torch.empty(n, dtype=self.torch.float64, device=self.device)

    def strip_len(self, k, side):
        nx, ny = self.dims[k]
        return ny if side in (WEST, EAST) else nx + 2

    def get_strip(self, k, vec, side, buf):
        self._check(self._lib().bmg_dd_copy(self._h, k, vec, side, 0, ctypes.c_void_p(buf.data_ptr()),
                                            self._stream()), "bmg_dd_copy")

    def put_strip(self, k, vec, side, buf):
        self._check(self._lib().bmg_dd_copy(self._h, k, vec, side, 1, ctypes.c_void_p(buf.data_ptr()),
                                            self._stream()), "bmg_dd_copy")

    def get_block(self, k, vec, ring=False):
        nx, ny = self.dims[k]
        t = self.torch.empty((ny + 2, nx + 2) if ring else (ny, nx), dtype=self.torch.float64,
                             device=self.device)
        self._check(self._lib().bmg_dd_block(self._h, k, vec, 0, int(ring), ctypes.c_void_p(t.data_ptr()),
                                             self._stream()), "bmg_dd_block")
        return t

    def put_block(self, k, vec, t, ring=False):
        nx, ny = self.dims[k]
        shape = (ny + 2, nx + 2) if ring else (ny, nx)
        if tuple(t.shape) != shape or not t.is_contiguous() or t.device != self.device:
            raise TypeError(f"block of shape {shape} on {self.device} expected, got {tuple(t.shape)}")
        self._check(self._lib().bmg_dd_block(self._h, k, vec, 1, int(ring), ctypes.c_void_p(t.data_ptr()),
                                             self._stream()), "bmg_dd_block")


# ---------------------------------------------------------------------------
# The distributed solve (Algorithm 2)
# ---------------------------------------------------------------------------

@dataclass
class DDInfo:
    cycles: int
    rel_resid: float
    history: list


class DDSolver:
    """One rank of the distributed solve.  `part` holds the rank's blocks
    (CudaPart, or any object with the same methods); `coarse` (rank 0 only)
    runs the cycle below the distributed levels: coarse.vcycle_from(level,
    b, x) with full-level (ny, nx) tensors."""

    def __init__(self, comm, layout: Layout, part, coarse=None, nu1=2, nu2=1):
        self.comm, self.layout, self.part, self.coarse = comm, layout, part, coarse
        self.nu1, self.nu2 = nu1, nu2
        self.rank = comm.rank
        self.nb = layout.neighbours(self.rank)
        self.top = layout.nlev - 1
        if self.rank == 0 and coarse is None:
            raise ValueError("rank 0 needs the coarse-level solver")
        # halo buffers per (part level, side): one to send, one to receive
        self.buf = {}
        for k in range(layout.nlev):
            for side in self.nb:
                n = part.strip_len(k, side)
                self.buf[(k, side)] = (part.buffer(n), part.buffer(n))

    def halo(self, k, vec):
        """Width-1 halo exchange of a vector on part level k (Section 2.1)."""
        for sides in ((WEST, EAST), (SOUTH, NORTH)):
            sends, recvs = [], []
            for side in sides:
                if side in self.nb:
                    sb, rb = self.buf[(k, side)]
                    self.part.get_strip(k, vec, side, sb)
                    sends.append((self.nb[side], sb))
                    recvs.append((self.nb[side], rb))
            self.comm.exchange(sends, recvs)
            for side in sides:
                if side in self.nb:
                    self.part.put_strip(k, vec, side, self.buf[(k, side)][1])

    def _colours(self, k):
        return 2 if k == self.top else 4

    def _relax(self, k, nu, reverse):
        order = list(range(self._colours(k)))
        if reverse:
            order.reverse()
        for _ in range(nu):
            for c in order:
                self.halo(k, VX)
                self.part.relax_colour(k, c)

    def _gather_solve_scatter(self):
        """gather_rhs, the coarse cycle on rank 0, scatter_sol (Algorithm 2)."""
        lay, part = self.layout, self.part
        bl = part.get_block(0, VB)
        if self.rank != 0:
            self.comm.exchange([(0, bl)], [])
            (i0, i1), (j0, j1) = lay.block(self.rank, 0)
            xr = part.buffer((j1 - j0 + 3) * (i1 - i0 + 3)).view(j1 - j0 + 3, i1 - i0 + 3)
            self.comm.exchange([], [(0, xr)])
            part.put_block(0, VX, xr, ring=True)
            return
        torch = part.torch
        nxg, nyg = lay.shapes[lay.gather]
        bfull = torch.zeros((nyg, nxg), dtype=torch.float64, device=part.device)
        (i0, i1), (j0, j1) = lay.block(0, 0)
        bfull[j0 - 1:j1, i0 - 1:i1] = bl
        for r in range(1, lay.size):
            (i0, i1), (j0, j1) = lay.block(r, 0)
            t = part.buffer((j1 - j0 + 1) * (i1 - i0 + 1)).view(j1 - j0 + 1, i1 - i0 + 1)
            self.comm.exchange([], [(r, t)])
            bfull[j0 - 1:j1, i0 - 1:i1] = t
        xfull = torch.zeros_like(bfull)
        self.coarse.vcycle_from(lay.gather, bfull, xfull)
        xpad = torch.nn.functional.pad(xfull, (1, 1, 1, 1))
        for r in range(1, lay.size):
            (i0, i1), (j0, j1) = lay.block(r, 0)
            self.comm.exchange([(r, xpad[j0 - 1:j1 + 2, i0 - 1:i1 + 2].contiguous())], [])
        (i0, i1), (j0, j1) = lay.block(0, 0)
        part.put_block(0, VX, xpad[j0 - 1:j1 + 2, i0 - 1:i1 + 2].contiguous(), ring=True)

    def vcycle(self):
        """One V(nu1, nu2) cycle of Algorithm 2 on the current iterate."""
        part, top = self.part, self.top
        for k in range(top, 0, -1):
            self._relax(k, self.nu1, reverse=False)
            self.halo(k, VX)
            part.residual(k)
            self.halo(k, VR)
            part.restrict(k)
        self._gather_solve_scatter()
        for k in range(1, top + 1):
            if k > 1:
                self.halo(k - 1, VX)
            part.interp(k)
            self._relax(k, self.nu2, reverse=True)

    def norms(self):
        self.halo(self.top, VX)
        self.part.residual(self.top)
        rr, bb = self.part.norms(self.top)
        return self.comm.allreduce_sum([rr, bb], self.part.device)

    def solve(self, b_block, x_block=None, tol=1e-10, max_cycles=200):
        """Iterate cycles until ||b - A x||_2 / ||b||_2 <= tol (checked before
        the first cycle and after each).  b_block, x_block: this rank's owned
        block of the finest level, (ny, nx) tensors; x_block (initial guess,
        zero if None) is overwritten.  Returns (x_block, DDInfo)."""
        part, top = self.part, self.top
        part.put_block(top, VB, b_block.contiguous())
        if x_block is None:
            x_block = part.torch.zeros_like(b_block)
        part.put_block(top, VX, x_block.contiguous())
        rr, bb = self.norms()
        bn = bb ** 0.5
        if bn == 0.0:
            x_block.zero_()
            return x_block, DDInfo(0, 0.0, [0.0])
        rel = rr ** 0.5 / bn
        hist, cycles = [rel], 0
        while rel > tol and cycles < max_cycles:
            self.vcycle()
            cycles += 1
            rel = self.norms()[0] ** 0.5 / bn
            hist.append(rel)
            if not np.isfinite(rel):
                break
        x_block.copy_(part.get_block(top, VX))
        return x_block, DDInfo(cycles, rel, hist)


def cuda_setup(comm, layout_args, k=None, options=None, device=None):
    """Centralised setup for the CUDA path: rank 0 builds the global
    hierarchy from k ((ny, nx) float64 CUDA tensor on rank 0) and scatters
    every rank its layout and planes.  layout_args: (px, py, dist_levels or
    None for the minimum-local-size rule).  Returns (DDSolver, hierarchy
    on rank 0 or None)."""
    from . import default_options, setup
    h = None
    if comm.rank == 0:
        if options is None:
            options = default_options()
        h = setup(k, options)
        shapes = [h.level_shape(l) for l in range(h.nlevels)]
        px, py, m = layout_args
        if m is None:
            m = choose_dist_levels(shapes, px, py)
        lay = Layout(shapes, px, py, m)
        if lay.size != comm.size:
            raise ValueError(f"processor grid {px} x {py} needs {lay.size} ranks, have {comm.size}")
        msgs = [(shapes, px, py, m, block_payload(h, lay, r), (options.nu1, options.nu2))
                for r in range(comm.size)]
    else:
        msgs = None
    shapes, px, py, m, payload, (nu1, nu2) = comm.scatter_object(msgs)
    lay = Layout(shapes, px, py, m)
    part = CudaPart(payload, device)
    return DDSolver(comm, lay, part, coarse=h, nu1=nu1, nu2=nu2), h
