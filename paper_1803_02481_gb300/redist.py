"""Model-guided coarse-grid redistribution: the postal performance model of
one V-cycle (Section 3), the enumeration of coarse processor grids (Section
4.1) and the search for the cheapest redistribution path (Section 4.2:
brute force over every path, and A* with f = g + h).

A path is a list of states (grid, level): the processor grid ((qx, qy) in
2D, (qx, qy, qz) in 3D) that runs the cycle from `level` down, until the
next state's level, whose problem is agglomerated onto the next (coarser)
grid.  The first state is the fine grid at the finest level; the last has
the grid of one processor.  Levels are numbered as in the library, 0 =
coarsest, with `shapes[l]` the global size of level l ((Nx, Ny) or
(Nx, Ny, Nz)); the dimension is that of the shapes.

Readings of the model (the paper leaves these open):

* local size on grid q: n_d = ceil(N_d / q_d);
* a halo exchange is charged only across the dimensions in which the grid
  has more than one processor, 2 alpha + 2 * face * 8 beta each with face
  the block's cross-section normal to that dimension (n_other in 2D, the
  product of the other two extents in 3D), so one processor exchanges
  nothing (in 2D the paper's formula, 2 D alpha + 2 sum_d n_d 8 beta, is the
  interior processor of a grid that is split in every dimension; its 3D form
  would charge edge lengths for faces, read here as face areas);
* interpolation costs the paper's counts: in 2D n^l + 20 n^{l-1} +
  6 sum_d n_d^{l-1} flops, in 3D n^l + 60 n^{l-1} + 15 n_0 n_2 + 6 n_1 n_2 +
  n_2 (level l - 1 extents), plus one halo exchange;
* stencils and colours: 5-point red-black finest and 9-point four-colour
  Galerkin levels in 2D; 7-point red-black finest and 27-point eight-colour
  Galerkin levels in 3D;
* interpolation into level l runs on level l's grid, and its coarse-side
  counts use level l - 1's local size on that grid;
* the agglomeration of level j from grid q to grid q' costs one gather of
  the right-hand side plus one scatter of the solution (none when
  redundant), p_block = prod_d ceil(q_d / q'_d) and n_block the local size
  of level j on q'; the coarsest solve adds the agglomeration of level 0 to
  one processor when a path reaches level 0 on a larger grid, plus
  (prod_d N_d^0)^2 gamma for the stored Cholesky factor's solve;
* coarsening continues on a grid while the local problem keeps at least
  `min_local` points; the first level below that is redistributed, and the
  level a state starts at always runs on its grid; level 0 only ever goes to
  one processor (it holds the coarsest solve), and a path whose grid keeps
  the limit down to level 1 ends with the agglomeration of level 0 to one
  processor, so every path ends at a one-processor state; a grid must hold
  every level it runs and its hand-off level with at least one point per
  processor in each dimension (the model's ceil-local sizes would hide
  processors without points): the hand-off moves up to the coarsest level
  the grid holds, and a grid that cannot run a level of its own is not
  entered;
* the enumeration refines, from 1 x 1, the dimension with the largest
  agglomerated local extent by a factor 2 (capped at the current grid);
  ties go to the dimension with fewer processors, then to y;
* the A* heuristic h is the remaining levels' computation at the current
  grid's local sizes without ceilings, plus the coarsest solve, plus one
  latency alpha while the grid has more than one processor: a lower bound
  of every completion (every later grid is coarser, every agglomeration
  costs at least alpha), so A* returns the brute-force optimum.
"""
from __future__ import annotations

import heapq
import math
from dataclasses import dataclass

Grid = tuple  # (qx, qy)


@dataclass(frozen=True)
class Machine:
    """Postal model parameters (Section 3): latency alpha [s], inverse
    bandwidth beta [s/B], inverse effective flop rate gamma [s/flop]."""
    alpha: float
    beta: float
    gamma: float


# Section 3, Table "Model parameters on Blue Waters" (9-point 2D stencil).
BLUE_WATERS = Machine(alpha=0.65e-6, beta=5.65e-9, gamma=0.44e-9)


@dataclass(frozen=True)
class Cycle:
    """V(nu1, nu2) with n_s stencil points and n_c colours on the finest and
    on the Galerkin levels; None: the method's (2D: 5-point red-black
    finest, 9-point four-colour Galerkin levels; 3D: 7-point red-black,
    27-point eight-colour)."""
    nu1: int = 2
    nu2: int = 1
    ns_fine: int | None = None
    nc_fine: int | None = None
    ns: int | None = None
    nc: int | None = None

    def stencils(self, dims):
        """(ns_fine, nc_fine, ns, nc) for a problem of `dims` dimensions."""
        d = {2: (5, 2, 9, 4), 3: (7, 2, 27, 8)}[dims]
        return tuple(v if v is not None else dv
                     for v, dv in zip((self.ns_fine, self.nc_fine, self.ns, self.nc), d))


def local(N, q):
    """Local extents of a global level of size N on grid q."""
    return tuple(-(-N[d] // q[d]) for d in range(len(N)))


def nprocs(q):
    return math.prod(q)


def t_exchange(n, q, m: Machine):
    """Width-1 halo exchange of a local block of extents n (Section 3)."""
    t = 0.0
    for d in range(len(n)):
        if q[d] > 1:
            face = math.prod(n[e] for e in range(len(n)) if e != d)
            t += 2 * m.alpha + 2 * face * 8 * m.beta
    return t


def t_smooth(n, q, m: Machine, ns, nc, nu):
    return 2 * ns * math.prod(n) * nu * m.gamma + nc * nu * t_exchange(n, q, m)


def t_residual(n, q, m: Machine, ns):
    return 2 * ns * math.prod(n) * m.gamma + t_exchange(n, q, m)


def t_restrict(n, m: Machine, ns):
    return 2 * ns * math.prod(n) * m.gamma


def interp_flops(n, nc_):
    """Flops of interpolation and correction (Section 3): 2D, fine points,
    20 per coarse point and 6 per coarse line point; 3D, fine points, 60 per
    coarse point, 15 n_0 n_2 + 6 n_1 n_2 + n_2 (coarse extents)."""
    if len(n) == 2:
        return n[0] * n[1] + 20 * nc_[0] * nc_[1] + 6 * (nc_[0] + nc_[1])
    return (n[0] * n[1] * n[2] + 60 * nc_[0] * nc_[1] * nc_[2] + 15 * nc_[0] * nc_[2]
            + 6 * nc_[1] * nc_[2] + nc_[2])


def t_interp(n, nc_, q, m: Machine):
    """Interpolation and correction plus one halo exchange."""
    return interp_flops(n, nc_) * m.gamma + t_exchange(n, q, m)


def t_gather(p_block, n_block, m: Machine):
    """Gather of n_block values over a processor block of p_block ranks."""
    if p_block <= 1:
        return 0.0
    return math.ceil(math.log2(p_block)) * m.alpha + n_block * (p_block - 1) / p_block * 8 * m.beta


def t_agglomerate(N, q, q2, m: Machine, redundant=False):
    """Level of global size N moved from grid q to the coarser grid q2:
    gather of the right-hand side plus scatter of the solution (no scatter
    when the coarse cycle runs redundantly in every processor block)."""
    p_block = math.prod(math.ceil(q[d] / q2[d]) for d in range(len(q)))
    g = t_gather(p_block, math.prod(local(N, q2)), m)
    return g if redundant else 2 * g


def level_time(shapes, l, q, m: Machine, cyc: Cycle):
    """Smoothing, residual, restriction and interpolation of level l >= 1 on
    grid q: one level's share of the V-cycle model."""
    fine = l == len(shapes) - 1
    ns_f, nc_f, ns_c, nc_c = cyc.stencils(len(q))
    ns, nc = (ns_f, nc_f) if fine else (ns_c, nc_c)
    n = local(shapes[l], q)
    nc_ = local(shapes[l - 1], q)
    return (t_smooth(n, q, m, ns, nc, cyc.nu1 + cyc.nu2) + t_residual(n, q, m, ns)
            + t_restrict(n, m, ns) + t_interp(n, nc_, q, m))


def t_cgsolve_factor(shapes, m: Machine):
    return math.prod(shapes[0]) ** 2 * m.gamma


# ---------------------------------------------------------------------------
# Coarse processor grid enumeration (Section 4.1)
# ---------------------------------------------------------------------------

def enumerate_grids(N, q):
    """Coarse processor grids for a global problem N on grid q: from one
    processor, refine by 2 the dimension with the largest agglomerated local
    extent (capped at q; ties to the dimension with fewer processors, then
    to the later dimension), until q itself is reached.  Returns the grids
    coarser than q, one processor first (log2 of q's processor count of
    them on a power-of-two grid)."""
    p = [1] * len(q)
    out = []
    while tuple(p) != tuple(q):
        out.append(tuple(p))
        n = local(N, p)
        cand = [d for d in range(len(q)) if p[d] < q[d]]
        d = max(cand, key=lambda d: (n[d], -p[d], d))
        p[d] = min(2 * p[d], q[d])
    return out


# ---------------------------------------------------------------------------
# Search (Section 4.2)
# ---------------------------------------------------------------------------

@dataclass
class SearchResult:
    path: list          # [(grid, level), ...], the last grid one processor
    cost: float         # modelled V-cycle time [s]
    expanded: int       # states expanded (A*) or visited (brute force)


class Space:
    """The redistribution search space of a hierarchy on a fine grid P:
    states (grid, level), edges to the agglomerations the coarsening limit
    allows, costs from the V-cycle model."""

    def __init__(self, shapes, P, machine: Machine = BLUE_WATERS, cycle: Cycle = Cycle(),
                 min_local=1024, redundant=False):
        self.shapes = [tuple(s) for s in shapes]
        self.P = tuple(P)
        self.m, self.cyc = machine, cycle
        self.min_local, self.redundant = min_local, redundant
        self.L = len(shapes)
        self.D = len(self.P)
        self.one = (1,) * self.D
        if any(len(s) != self.D for s in self.shapes):
            raise ValueError("shapes and the processor grid must have the same dimension")

    @property
    def start(self):
        return (self.P, self.L - 1)

    def limit_level(self, q, j):
        """First level below j whose local problem on q is under the
        coarsening limit, or None if every level down to 0 keeps it."""
        for l in range(j - 1, -1, -1):
            if math.prod(local(self.shapes[l], q)) < self.min_local:
                return l
        return None

    def run_time(self, q, j, l):
        """Levels j down to l + 1 on grid q."""
        return sum(level_time(self.shapes, i, q, self.m, self.cyc) for i in range(j, l, -1))

    def successors(self, N, q):
        """Enumerated grids for level size N on q; a redundant search keeps
        those whose processor blocks are all the same size."""
        out = enumerate_grids(N, q)
        if self.redundant:
            out = [g for g in out if all(q[d] % g[d] == 0 for d in range(self.D))]
        return out

    def fits(self, l, q):
        """Grid q can hold level l: at least one point per processor in every
        dimension (monotone: every finer level fits too)."""
        return all(self.shapes[l][d] >= q[d] for d in range(self.D))

    def handoff(self, q, j):
        """Level a state (q, j) agglomerates: the coarsening limit (level 0
        when every level keeps it), raised to the coarsest level q can hold.
        At least j when q cannot run a level of its own (a dead end)."""
        l = self.limit_level(q, j)
        h = 0 if l is None else l
        while h < j and not self.fits(h, q):
            h += 1
        return h

    def edges(self, state):
        """(next state or None for the goal, edge cost) of a state."""
        q, j = state
        if q == self.one:
            yield None, self.run_time(q, j, 0) + t_cgsolve_factor(self.shapes, self.m)
            return
        h = self.handoff(q, j)
        if h >= j:
            return
        base = self.run_time(q, j, h)
        # level 0 holds only the coarsest solve: it goes to one processor
        grids = self.successors(self.shapes[h], q) if h > 0 else [self.one]
        for q2 in grids:
            if q2 != self.one and self.handoff(q2, h) >= h:
                continue
            yield (q2, h), base + t_agglomerate(self.shapes[h], q, q2, self.m, self.redundant)

    def heuristic(self, state):
        """Lower bound of the cost from state to the goal."""
        q, j = state
        g = self.m.gamma
        c = self.cyc
        ns_f, _, ns_c, _ = c.stencils(self.D)
        h = t_cgsolve_factor(self.shapes, self.m) + (self.m.alpha if q != self.one else 0.0)
        for l in range(j, 0, -1):
            ns = ns_f if l == self.L - 1 else ns_c
            n = tuple(self.shapes[l][d] / q[d] for d in range(self.D))
            nc_ = tuple(self.shapes[l - 1][d] / q[d] for d in range(self.D))
            h += (2 * ns * math.prod(n) * (c.nu1 + c.nu2 + 2) + interp_flops(n, nc_)) * g
        return h

    def path_cost(self, path):
        """Model time of one V-cycle along a path of states."""
        cost, state = 0.0, tuple(path[0])
        if state != self.start:
            raise ValueError(f"a path starts at {self.start}")
        for nxt in list(path[1:]) + [None]:
            nxt = None if nxt is None else (tuple(nxt[0]), nxt[1])
            for s2, c in self.edges(state):
                if s2 == nxt:
                    cost += c
                    break
            else:
                raise ValueError(f"no edge {state} -> {nxt}")
            state = nxt
        return cost

    def states_of_grids(self, grids, enumerated=True):
        """The path of states that visits the given grids in order (fine grid
        first, 1 x 1 last), each agglomeration at the coarsening limit; with
        `enumerated`, every grid must be one the enumeration offers."""
        grids = [tuple(g) for g in grids]
        if grids[0] != self.P or grids[-1] != self.one:
            raise ValueError("a path runs from the fine grid to one processor")
        path = [self.start]
        for q2 in grids[1:]:
            q, j = path[-1]
            h = self.handoff(q, j)
            if h >= j:
                raise ValueError(f"{q} cannot run a level below {j}")
            if enumerated and q2 not in (self.successors(self.shapes[h], q) if h > 0 else [self.one]):
                raise ValueError(f"{q} -> {q2} is not a redistribution of the search space")
            path.append((q2, h))
        return path


def search_brute_force(space: Space) -> SearchResult:
    """Every path, depth first; visits are counted per state reached."""
    best = [math.inf, None]
    visits = [0]

    def dfs(state, g, path):
        visits[0] += 1
        for s2, c in space.edges(state):
            if s2 is None:
                if g + c < best[0]:
                    best[0], best[1] = g + c, list(path)
            else:
                dfs(s2, g + c, path + [s2])

    dfs(space.start, 0.0, [space.start])
    return SearchResult(best[1], best[0], visits[0])


def search_astar(space: Space) -> SearchResult:
    """A* over the states with f = g + h (h a consistent lower bound)."""
    start = space.start
    GOAL = ("goal",)
    tie = 0
    heap = [(space.heuristic(start), tie, 0.0, start)]
    g_best = {start: 0.0}
    parent = {start: None}
    closed = set()
    expanded = 0
    while heap:
        f, _, g, s = heapq.heappop(heap)
        if s in closed or g > g_best.get(s, math.inf):
            continue
        if s == GOAL:
            path, t = [], parent[GOAL]
            while t is not None:
                path.append(t)
                t = parent[t]
            return SearchResult(path[::-1], g, expanded)
        closed.add(s)
        expanded += 1
        for s2, c in space.edges(s):
            key = GOAL if s2 is None else s2
            g2 = g + c
            if key in closed or g2 >= g_best.get(key, math.inf):
                continue
            g_best[key] = g2
            parent[key] = s
            tie += 1
            heapq.heappush(heap, (g2 + (0.0 if s2 is None else space.heuristic(s2)), tie, g2, key))
    raise RuntimeError("the goal is unreachable")


def halving_shapes(N, coarsest=3):
    """Global sizes of a hierarchy coarsened by 2 in each dimension (ceil),
    finest N, until a side would drop below `coarsest`; coarsest first."""
    out = [tuple(N)]
    while min(out[-1]) // 2 >= coarsest:
        out.append(tuple(-(-n // 2) for n in out[-1]))
    return out[::-1]
