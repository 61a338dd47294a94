"""Domain-decomposed solve phase (Section 2.1) with coarse-grid
redistribution by agglomeration (Section 2.2, Algorithm 2), along a path
chosen by the performance model (Sections 3-4, ``redist``).

The ranks form a px x py processor grid.  A redistribution plan (`Plan`)
is a path of states (grid, level): the fine grid runs the finest levels,
then the problem of the level where the coarsening limit is reached is
agglomerated onto a coarser grid, which runs the next levels, and so on
down to one rank, which runs the rest of the cycle with the library's
single-GPU schedule.  On each level of its stage a rank owns one
rectangular block of points and keeps it, with a one-point ring of its
neighbours' values (the width-1 halo), in a part of the CUDA library
(``bmg_dd_*``).  One V-cycle is Algorithm 2 with p_l decreasing stage by
stage:

* relax: one halo exchange of x before every colour, then the colour;
* residual: a halo exchange of x, r = b - A x;
* restriction: a halo exchange of r, b_{l-1} = P^T r (local otherwise);
* gather_rhs where p_l > p_{l-1}: the processor block of each coarse task
  sends its blocks of the restricted right-hand side to the block's first
  member, which runs the coarse task; or, redundant, every member
  allgathers them and runs it as a replica;
* scatter_sol: the coarse task sends every member its block of the coarse
  solution, ring included (none when redundant); then interpolation and
  post-smoothing climb back, with a halo exchange of the coarser x before
  each interpolation;
* the stop test adds the ranks' partial sums of r^2 and b^2 (allreduce).

A halo exchange runs in two phases, west/east (owned rows) and then
south/north (rows including the ring columns, which carry the corners).

Setup is centralised: rank 0 builds the global hierarchy (assembly,
operator-induced interpolation, Galerkin operators, coarsest factor) and
scatters to every rank the planes of its blocks, ring included.  A stage's
blocks start at 0-based indices that are multiples of 2^(levels it
coarsens), so the colours, coarse points and restriction/interpolation
offsets of a block are those of the full level.

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
# Layout: processor grids, blocks and ranks of a redistribution plan
# ---------------------------------------------------------------------------

def coarse_range(lo: int, hi: int):
    """Coarse points of a 1-based fine range: coarse point I is fine point 2I."""
    return (lo + 1) // 2, hi // 2


def split_weighted(lo: int, hi: int, weights, align: int):
    """Contiguous 0-based half-open ranges covering [lo, hi), one per weight,
    each starting at a multiple of `align` (lo is one).  The units are the
    whole `align`-point units of the range (the points a coarser level keeps
    after log2(align) coarsenings); the last range also takes the remainder,
    so every range keeps at least one point on that level.  Unit counts
    follow the weights: floors, then the largest remainders (ties to the
    lower index), at least one unit each."""
    units = (hi - lo) // align
    p = len(weights)
    if units < p:
        raise ValueError(f"{hi - lo} points cannot be split into {p} blocks of at least {align}")
    W = sum(weights)
    cnt = [units * w // W for w in weights]
    order = sorted(range(p), key=lambda i: (-(units * weights[i] % W), i))
    for i in order[:units - sum(cnt)]:
        cnt[i] += 1
    for i in range(p):
        if cnt[i] == 0:
            big = max(range(p), key=lambda t: cnt[t])
            cnt[big] -= 1
            cnt[i] = 1
    out, u = [], 0
    for c in cnt:
        out.append((lo + u * align, lo + (u + c) * align))
        u += c
    out[-1] = (out[-1][0], hi)
    return out


def split(n: int, p: int, align: int):
    """p contiguous 1-based ranges covering 1..n, each starting at a 0-based
    index that is a multiple of `align`, sizes as equal as alignment allows."""
    return [(a + 1, b) for a, b in split_weighted(0, n, [1] * p, align)]


def groups(p: int, q: int):
    """Processor blocks of an agglomeration by dimension: p indices in q
    contiguous groups of floor or ceil(p / q) members."""
    return [list(range(g * p // q, (g + 1) * p // q)) for g in range(q)]


class Plan:
    """A redistribution path executed on px x py ranks (Section 2.2,
    Algorithm 2): states ((qx, qy), level), the first the fine grid at the
    finest level, the last (1, 1).  Stage s runs its grid from level path[s]
    down to path[s + 1]'s level + 1, restricts onto path[s + 1]'s level on
    its own blocks ("part level 0") and agglomerates that level onto the next
    grid: the processor blocks of each coarse task gather the right-hand side
    to one member (the first) and get the solution back, or, if
    `redundant`, allgather it and every member runs the coarse task as a
    replica (no scatter).  The last state runs the rest of the cycle on one
    rank with the single-GPU schedule.

    Blocks: a stage's blocks start, on its finest level, at 0-based indices
    that are multiples of 2^(levels it coarsens), so colours and
    coarse-point offsets are those of the global level; a coarse task's block
    is the union of its members' blocks.  The ranges are built from the
    coarsest stage down, each split in proportion to the fine-grid ranks a
    task stands for.

    Ranks: rank r is fine-grid task (r % px, r // px).  A coarse task is run
    by its group's first member; replicas (redundant) form copies of the
    coarser grids, one per position in the processor block."""

    def __init__(self, shapes, path, redundant=False):
        self.shapes = [tuple(int(v) for v in s) for s in shapes]
        self.path = [((int(q[0]), int(q[1])), int(l)) for q, l in path]
        self.redundant = bool(redundant)
        L = len(self.shapes)
        P, top = self.path[0]
        if top != L - 1 or self.path[-1][0] != (1, 1) or len(self.path) < 2:
            raise ValueError("a path runs from the fine grid at the finest level to 1 x 1")
        for (q, j), (q2, j2) in zip(self.path, self.path[1:]):
            if not 0 <= j2 < j:
                raise ValueError("levels must decrease along a path")
            if q2[0] > q[0] or q2[1] > q[1] or q2[0] * q2[1] >= q[0] * q[1] or min(q2) < 1:
                raise ValueError(f"{q} -> {q2} is not an agglomeration")
            if self.redundant and (q[0] % q2[0] or q[1] % q2[1]):
                raise ValueError(f"redundant agglomeration {q} -> {q2} needs equal processor blocks")
        self.px, self.py = P
        self.size = P[0] * P[1]
        S = self.nstage = len(self.path) - 1
        grids = [q for q, _ in self.path]
        lev = [j for _, j in self.path]
        self.grp = [[groups(grids[s][d], grids[s + 1][d]) for d in range(2)] for s in range(S)]
        # fine-grid ranks per task, by dimension
        w = [[[1] * P[d] for d in range(2)]]
        for s in range(S - 1):
            w.append([[sum(w[s][d][a] for a in g) for g in self.grp[s][d]] for d in range(2)])
        # 0-based ranges per stage on its finest level, coarsest stage first
        cuts = [[None, None] for _ in range(S)]
        for d in range(2):
            Nd = [self.shapes[l][d] for l in range(L)]
            cuts[S - 1][d] = split_weighted(0, Nd[lev[S - 1]], w[S - 1][d], 2 ** (lev[S - 1] - lev[S]))
            for s in range(S - 2, -1, -1):
                m = lev[s] - lev[s + 1]
                rng = []
                for g, (c0, c1) in enumerate(cuts[s + 1][d]):
                    hi = c1 << m if c1 < Nd[lev[s + 1]] else Nd[lev[s]]
                    rng += split_weighted(c0 << m, hi, [w[s][d][a] for a in self.grp[s][d][g]],
                                          2 ** (lev[s] - lev[s + 1]))
                cuts[s][d] = rng
        self.stages = [StageLayout(self, s, cuts[s]) for s in range(S)]
        # ranks of the tasks, per copy
        ranks = [{(): [[b * P[0] + a for a in range(P[0])] for b in range(P[1])]}]
        for s in range(S - 1):
            gx, gy = self.grp[s]
            new = {}
            for c, arr in ranks[s].items():
                if not self.redundant:
                    new[c] = [[arr[gy[b][0]][gx[a][0]] for a in range(len(gx))] for b in range(len(gy))]
                    continue
                for ry in range(len(gy[0])):
                    for rx in range(len(gx[0])):
                        new[c + ((rx, ry),)] = [[arr[gy[b][ry]][gx[a][rx]] for a in range(len(gx))]
                                                for b in range(len(gy))]
            ranks.append(new)
        self.ranks = ranks
        self.final = {}
        qx, qy = grids[S - 1]
        for c, arr in ranks[S - 1].items():
            if not self.redundant:
                self.final[c] = arr[0][0]
            else:
                for ry in range(qy):
                    for rx in range(qx):
                        self.final[c + ((rx, ry),)] = arr[ry][rx]
        self.roles = [[] for _ in range(self.size)]
        for s in range(S):
            for c, arr in ranks[s].items():
                for b, row in enumerate(arr):
                    for a, r in enumerate(row):
                        self.roles[r].append((s, c, a, b))
        for r in range(self.size):
            if [t[0] for t in self.roles[r]] != list(range(len(self.roles[r]))):
                raise AssertionError("a rank must run a prefix of the stages, one task each")

    @property
    def final_level(self):
        return self.path[-1][1]

    def coarse_ranks(self):
        """Ranks that run the one-rank coarse cycle."""
        return sorted(set(self.final.values()))

    def group_of(self, s, a, b):
        """Index of the stage-(s + 1) task (or None for the one-rank coarse
        task) whose processor block holds stage-s task (a, b), and its
        members."""
        if s == self.nstage - 1:
            q = self.path[s][0]
            return None, [(x, y) for y in range(q[1]) for x in range(q[0])]
        gx, gy = self.grp[s]
        ga = next(g for g, mem in enumerate(gx) if a in mem)
        gb = next(g for g, mem in enumerate(gy) if b in mem)
        return (ga, gb), [(x, y) for y in gy[gb] for x in gx[ga]]

    def position(self, s, a, b):
        """(rx, ry): position of stage-s task (a, b) in its processor block."""
        if s == self.nstage - 1:
            return (a, b)
        gx, gy = self.grp[s]
        ga = next(g for g, mem in enumerate(gx) if a in mem)
        gb = next(g for g, mem in enumerate(gy) if b in mem)
        return (gx[ga].index(a), gy[gb].index(b))


class StageLayout:
    """Blocks of one stage: grid qx x qy over the levels lo..hi of the
    global hierarchy; part level k is level lo + k (k = 0 the level the
    stage restricts onto and agglomerates)."""

    def __init__(self, plan: Plan, s: int, cuts):
        self.plan, self.s = plan, s
        (self.qx, self.qy), self.hi = plan.path[s]
        self.lo = plan.path[s + 1][1]
        self.nlev = self.hi - self.lo + 1
        self.fine = self.hi == len(plan.shapes) - 1
        self.xr, self.yr = [], []
        for d, out in ((0, self.xr), (1, self.yr)):
            rs = [(c0 + 1, c1) for c0, c1 in cuts[d]]
            per = [rs]
            for _ in range(self.nlev - 1):
                per.append([coarse_range(*r) for r in per[-1]])
            per.reverse()
            out.extend(per)
        for k in range(self.nlev):
            for lo, hi in self.xr[k] + self.yr[k]:
                if hi < lo:
                    raise ValueError("a block is empty on a distributed level; use fewer ranks or levels")

    def block(self, a, b, k):
        """((i0, i1), (j0, j1)) 1-based owned ranges of task (a, b) on part level k."""
        return self.xr[k][a], self.yr[k][b]

    def neighbours(self, a, b):
        """Neighbouring tasks by side."""
        nb = {}
        if a > 0:
            nb[WEST] = (a - 1, b)
        if a < self.qx - 1:
            nb[EAST] = (a + 1, b)
        if b > 0:
            nb[SOUTH] = (a, b - 1)
        if b < self.qy - 1:
            nb[NORTH] = (a, b + 1)
        return nb

    def nine(self):
        """Per part level: 9-point (four colours) or, on the finest level,
        5-point (red-black)."""
        return [0 if (self.fine and k == self.nlev - 1) else 1 for k in range(self.nlev)]


class Layout:
    """One-stage plan: the px x py grid on the finest `dist_levels` levels,
    level L - 1 - dist_levels (the gather level) agglomerated to one rank."""

    def __init__(self, shapes, px, py, dist_levels, redundant=False):
        L = len(shapes)
        if not 1 <= dist_levels <= L - 1:
            raise ValueError(f"dist_levels must be in 1..{L - 1}")
        self.shapes, self.px, self.py, self.dist_levels = shapes, px, py, dist_levels
        self.gather = L - 1 - dist_levels
        if (px, py) == (1, 1):
            raise ValueError("a 1 x 1 grid has nothing to distribute")
        self.plan = Plan(shapes, [((px, py), L - 1), ((1, 1), self.gather)], redundant)
        self.stage = self.plan.stages[0]
        self.xr, self.yr = self.stage.xr, self.stage.yr

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
        return self.stage.block(*self.coords(rank), k)

    def neighbours(self, rank):
        return {side: b * self.px + a for side, (a, b) in self.stage.neighbours(*self.coords(rank)).items()}


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


def search_plan(shapes, P, machine=None, min_local=1024, redundant=False, cycle=None):
    """The cheapest redistribution path of the V-cycle model (Sections 3-4,
    A* search) for a hierarchy of `shapes` on the grid P, as a Plan, with
    the search result.  Grids whose processor blocks are unequal are left
    out of a redundant search."""
    from . import redist as R
    space = R.Space(shapes, P, machine or R.BLUE_WATERS, cycle or R.Cycle(), min_local, redundant)
    res = R.search_astar(space)
    return Plan(shapes, res.path, redundant), res


def stage_payload(source, st: StageLayout, a: int, b: int):
    """The planes task (a, b) of a stage needs: per part level k >= 1 the
    stencil of its block with ring (5, ny + 2, nx + 2) and the interpolation
    planes on the coarser block with ring (8, nyc + 2, nxc + 2); part level
    0 has none."""
    stencils, interps, dims = [None], [None], []
    for k in range(st.nlev):
        (i0, i1), (j0, j1) = st.block(a, b, k)
        dims.append((i1 - i0 + 1, j1 - j0 + 1))
        if k == 0:
            continue
        lvl = st.lo + k
        s = source.level_stencil(lvl)
        pl = np.stack([np.pad(s[key], 1) for key in STENCIL_KEYS])
        stencils.append(np.ascontiguousarray(pl[:, j0 - 1:j1 + 2, i0 - 1:i1 + 2]))
        (I0, I1), (J0, J1) = st.block(a, b, k - 1)
        pi = source.level_interp(lvl)             # (ncy + 1, ncx + 1), index 0 = ring
        pp = np.stack([np.pad(pi[key], ((0, 1), (0, 1))) for key in INTERP_KEYS])
        interps.append(np.ascontiguousarray(pp[:, J0 - 1:J1 + 2, I0 - 1:I1 + 2]))
    return {"dims": dims, "stencils": stencils, "interps": interps, "nine": st.nine()}


def plan_payloads(source, plan: Plan, rank: int):
    """Per stage this rank runs, the planes of its task."""
    return [stage_payload(source, plan.stages[s], a, b) for s, _, a, b in plan.roles[rank]]


def block_payload(source, layout: Layout, rank: int):
    """The planes rank needs on a one-stage layout."""
    return stage_payload(source, layout.stage, *layout.coords(rank))


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


class _Task:
    """This rank's task in one stage: its part, neighbours and halo buffers."""

    def __init__(self, plan: Plan, s, copy, a, b, part):
        self.s, self.copy, self.a, self.b = s, copy, a, b
        self.lay = plan.stages[s]
        self.part = part
        self.top = self.lay.nlev - 1
        self.nine = self.lay.nine()
        ranks = plan.ranks[s][copy]
        self.nb = {side: ranks[bb][aa] for side, (aa, bb) in self.lay.neighbours(a, b).items()}
        self.buf = {}
        for k in range(self.lay.nlev):
            for side in self.nb:
                n = part.strip_len(k, side)
                self.buf[(k, side)] = (part.buffer(n), part.buffer(n))
        self.zero_top = None


class DDSolver:
    """One rank of the distributed solve along a redistribution plan.
    `parts` holds the rank's blocks per stage it runs (CudaPart, or any
    object with the same methods; a single part for a one-stage plan);
    `coarse` (on the ranks that run the one-rank coarse task) runs the cycle
    below the plan's last level: coarse.vcycle_from(level, b, x) with
    full-level (ny, nx) tensors."""

    def __init__(self, comm, plan, parts, coarse=None, nu1=2, nu2=1):
        self.layout = plan if isinstance(plan, Layout) else None
        plan = plan.plan if isinstance(plan, Layout) else plan
        if not isinstance(parts, (list, tuple)):
            parts = [parts]
        self.comm, self.plan, self.coarse = comm, plan, coarse
        self.nu1, self.nu2 = nu1, nu2
        self.rank = comm.rank
        roles = plan.roles[self.rank]
        if len(parts) != len(roles):
            raise ValueError(f"rank {self.rank} runs {len(roles)} stages, got {len(parts)} parts")
        self.tasks = [_Task(plan, s, c, a, b, p) for (s, c, a, b), p in zip(roles, parts)]
        self.part = parts[0]
        if self.rank in plan.coarse_ranks() and coarse is None:
            raise ValueError(f"rank {self.rank} runs the coarse cycle and needs the coarse-level solver")

    def block(self):
        """((i0, i1), (j0, j1)) 1-based ranges of this rank's finest block."""
        t = self.tasks[0]
        return t.lay.block(t.a, t.b, t.top)

    def destroy(self):
        for t in self.tasks:
            if hasattr(t.part, "destroy"):
                t.part.destroy()

    def halo(self, t: _Task, k, vec):
        """Width-1 halo exchange of a vector on part level k (Section 2.1):
        west/east strips of the owned rows, then south/north rows including
        the ring columns (the corners)."""
        for sides in ((WEST, EAST), (SOUTH, NORTH)):
            sends, recvs = [], []
            for side in sides:
                if side in t.nb:
                    sb, rb = t.buf[(k, side)]
                    t.part.get_strip(k, vec, side, sb)
                    sends.append((t.nb[side], sb))
                    recvs.append((t.nb[side], rb))
            self.comm.exchange(sends, recvs)
            for side in sides:
                if side in t.nb:
                    t.part.put_strip(k, vec, side, t.buf[(k, side)][1])

    def _relax(self, t: _Task, k, nu, reverse):
        order = list(range(4 if t.nine[k] else 2))
        if reverse:
            order.reverse()
        for _ in range(nu):
            for c in order:
                self.halo(t, k, VX)
                t.part.relax_colour(k, c)

    def _cycle(self, s):
        """Stage s of one V(nu1, nu2) cycle, with everything below it."""
        t = self.tasks[s]
        part = t.part
        for k in range(t.top, 0, -1):
            self._relax(t, k, self.nu1, reverse=False)
            self.halo(t, k, VX)
            part.residual(k)
            self.halo(t, k, VR)
            part.restrict(k)
        self._agglomerate(s)
        for k in range(1, t.top + 1):
            if k > 1:
                self.halo(t, k - 1, VX)
            part.interp(k)
            self._relax(t, k, self.nu2, reverse=True)

    def _agglomerate(self, s):
        """gather_rhs, the coarser cycle, scatter_sol (Algorithm 2) of stage
        s's last level: the processor block gathers (or, redundant,
        allgathers) the right-hand side, the coarse task cycles, the solution
        with its ring comes back to every member."""
        plan, t = self.plan, self.tasks[s]
        part, torch = t.part, t.part.torch
        g, members = plan.group_of(s, t.a, t.b)
        ranks = plan.ranks[s][t.copy]
        mem = [(ranks[bb][aa], aa, bb) for aa, bb in members]
        final = s == plan.nstage - 1
        bl = part.get_block(0, VB)
        if plan.redundant:
            ry = plan.position(s, t.a, t.b)
            copy = t.copy + (ry,)
            root = self.rank
        else:
            copy = t.copy
            root = plan.final[copy] if final else plan.ranks[s + 1][copy][g[1]][g[0]]
        if root != self.rank:
            (i0, i1), (j0, j1) = t.lay.block(t.a, t.b, 0)
            self.comm.exchange([(root, bl)], [])
            xr = part.buffer((j1 - j0 + 3) * (i1 - i0 + 3)).view(j1 - j0 + 3, i1 - i0 + 3)
            self.comm.exchange([], [(root, xr)])
            part.put_block(0, VX, xr, ring=True)
            return
        # the coarse task's block on this level
        if final:
            nx, ny = plan.shapes[t.lay.lo]
            (U0, U1), (V0, V1) = (1, nx), (1, ny)
        else:
            t2 = self.tasks[s + 1]
            assert (t2.a, t2.b) == g and t2.copy == copy
            (U0, U1), (V0, V1) = t2.lay.block(t2.a, t2.b, t2.top)
        bu = torch.zeros((V1 - V0 + 1, U1 - U0 + 1), dtype=torch.float64, device=part.device)
        others = [(r, aa, bb) for r, aa, bb in mem if r != self.rank]
        recvs = []
        for r, aa, bb in others:
            (i0, i1), (j0, j1) = t.lay.block(aa, bb, 0)
            recvs.append((r, part.buffer((j1 - j0 + 1) * (i1 - i0 + 1)).view(j1 - j0 + 1, i1 - i0 + 1)))
        sends = [(r, bl) for r, _, _ in others] if plan.redundant else []
        self.comm.exchange(sends, recvs)
        for (r, aa, bb), (_, blk) in zip(others, recvs):
            (i0, i1), (j0, j1) = t.lay.block(aa, bb, 0)
            bu[j0 - V0:j1 - V0 + 1, i0 - U0:i1 - U0 + 1] = blk
        (i0, i1), (j0, j1) = t.lay.block(t.a, t.b, 0)
        bu[j0 - V0:j1 - V0 + 1, i0 - U0:i1 - U0 + 1] = bl
        if final:
            xu = torch.zeros_like(bu)
            self.coarse.vcycle_from(t.lay.lo, bu, xu)
            xring = torch.nn.functional.pad(xu, (1, 1, 1, 1))
        else:
            p2 = t2.part
            if t2.zero_top is None:
                t2.zero_top = torch.zeros_like(bu)
            p2.put_block(t2.top, VB, bu)
            p2.put_block(t2.top, VX, t2.zero_top)
            self._cycle(s + 1)
            self.halo(t2, t2.top, VX)
            xring = p2.get_block(t2.top, VX, ring=True)
        if not plan.redundant:
            for r, aa, bb in others:
                (i0, i1), (j0, j1) = t.lay.block(aa, bb, 0)
                self.comm.exchange([(r, xring[j0 - V0:j1 - V0 + 3, i0 - U0:i1 - U0 + 3].contiguous())], [])
        (i0, i1), (j0, j1) = t.lay.block(t.a, t.b, 0)
        part.put_block(0, VX, xring[j0 - V0:j1 - V0 + 3, i0 - U0:i1 - U0 + 3].contiguous(), ring=True)

    def vcycle(self):
        """One V(nu1, nu2) cycle of Algorithm 2 on the current iterate."""
        self._cycle(0)

    def norms(self):
        t = self.tasks[0]
        self.halo(t, t.top, VX)
        t.part.residual(t.top)
        rr, bb = t.part.norms(t.top)
        return self.comm.allreduce_sum([rr, bb], t.part.device)

    def solve(self, b_block, x_block=None, tol=1e-10, max_cycles=200):
        """Iterate cycles until ||b - A x||_2 / ||b||_2 <= tol (checked before
        the first cycle and after each).  b_block, x_block: this rank's owned
        block of the finest level, (ny, nx) tensors; x_block (initial guess,
        zero if None) is overwritten.  Returns (x_block, DDInfo)."""
        t = self.tasks[0]
        part, top = t.part, t.top
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


_SETUP_LOCK = threading.Lock()


def make_plan(shapes, px, py, dist_levels=None, path=None, redundant=False, machine=None, min_local=1024):
    """The plan of a px x py grid: one stage (path None; dist_levels or the
    minimum-local-size rule), the model's cheapest path (path "search"), a
    list of grids (fine grid first, 1 x 1 last; each agglomeration at the
    coarsening limit) or a list of states ((qx, qy), level)."""
    L = len(shapes)
    if path is None:
        m = choose_dist_levels(shapes, px, py, min_local) if dist_levels is None else dist_levels
        return Plan(shapes, [((px, py), L - 1), ((1, 1), L - 1 - m)], redundant)
    if isinstance(path, str):
        if path != "search":
            raise ValueError(f"unknown path {path!r}")
        return search_plan(shapes, (px, py), machine, min_local, redundant)[0]
    path = list(path)
    if path and isinstance(path[0][0], (tuple, list)):
        return Plan(shapes, path, redundant)
    from . import redist as R
    space = R.Space(shapes, (px, py), machine or R.BLUE_WATERS, R.Cycle(), min_local, redundant)
    return Plan(shapes, space.states_of_grids(path, enumerated=False), redundant)


def cuda_setup(comm, layout_args, k=None, options=None, device=None, path=None, redundant=False,
               machine=None, min_local=1024):
    """Centralised setup for the CUDA path: rank 0 builds the global
    hierarchy from k ((ny, nx) float64 CUDA tensor on rank 0), makes the plan
    (`make_plan`; layout_args = (px, py) or (px, py, dist_levels or None))
    and scatters every rank its plan and planes; every other rank that runs
    the one-rank coarse task (redundant plans) builds the same hierarchy
    from a copy of k.  Returns (DDSolver, hierarchy or None)."""
    import torch

    from . import Options, default_options, setup
    h = None
    if comm.rank == 0:
        if options is None:
            options = default_options()
        with _SETUP_LOCK:
            h = setup(k, options)
        shapes = [h.level_shape(l) for l in range(h.nlevels)]
        px, py = layout_args[:2]
        m = layout_args[2] if len(layout_args) > 2 else None
        plan = make_plan(shapes, px, py, m, path, redundant, machine, min_local)
        if plan.size != comm.size:
            raise ValueError(f"processor grid {px} x {py} needs {plan.size} ranks, have {comm.size}")
        kc = k.cpu().numpy() if len(plan.coarse_ranks()) > 1 else None
        msgs = [(shapes, plan.path, plan.redundant, plan_payloads(h, plan, r), bytes(options),
                 kc if (r != 0 and r in plan.coarse_ranks()) else None) for r in range(comm.size)]
    else:
        msgs = None
    shapes, states, red, payloads, opt, kc = comm.scatter_object(msgs)
    plan = Plan(shapes, states, red)
    options = Options.from_buffer_copy(opt)
    parts = [CudaPart(p, device) for p in payloads]
    if kc is not None:
        with _SETUP_LOCK:
            h = setup(torch.from_numpy(kc).to(parts[0].device), options)
    return DDSolver(comm, plan, parts, coarse=h, nu1=options.nu1, nu2=options.nu2), h
