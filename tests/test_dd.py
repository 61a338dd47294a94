"""Domain-decomposed solve (Section 2.1) with agglomeration to one rank
(Section 2.2, Algorithm 2), on CPU ranks.

The ranks run the SPMD driver of paper_1803_02481_gb300.dd with the CPU
stand-in for their parts (the oracle's per-point arithmetic on blocks with a
one-point ring) and the oracle's hierarchy as the global source.  The
distributed V-cycle must reproduce the oracle's single-domain solve: the
same cycle count and the same iterate up to the rounding of the different
summation orders, on 1 x 2, 2 x 1, 2 x 2 and 3 x 2 processor grids, with the
gather level near the top and near the bottom of the hierarchy, over real
`gloo` process groups and over the in-process thread communicator.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from oracle import boxmg_oracle as O  # noqa: E402
from paper_1803_02481_gb300 import dd, inputs  # noqa: E402
from tests.dd_cpu_part import CpuPart, OracleSource  # noqa: E402

TOL = 1e-10


def _problem(n, seed):
    return inputs.block_problem(n, seed=seed, block=8, lo=-2, hi=2)


def _solve_ranks(comm, pr, px, py, m):
    """SPMD body: centralised setup on rank 0 from the oracle hierarchy,
    scatter of the layout and the block planes, distributed solve; returns
    this rank's block of x and the info."""
    if comm.rank == 0:
        h = O.setup(pr["k"])
        src = OracleSource(h)
        shapes = [src.level_shape(l) for l in range(src.nlevels)]
        lay = dd.Layout(shapes, px, py, m)
        msgs = [(shapes, dd.block_payload(src, lay, r)) for r in range(comm.size)]
    else:
        src = None
        msgs = None
    shapes, payload = comm.scatter_object(msgs)
    lay = dd.Layout(shapes, px, py, m)
    solver = dd.DDSolver(comm, lay, CpuPart(payload), coarse=src)
    (i0, i1), (j0, j1) = lay.block(comm.rank, lay.nlev - 1)
    b = torch.from_numpy(np.ascontiguousarray(pr["b"][j0 - 1:j1, i0 - 1:i1]))
    x, info = solver.solve(b, tol=TOL, max_cycles=100)
    return (i0, i1, j0, j1), x.numpy().copy(), info


def _check(pr, results):
    ref = O.solve(O.setup(pr["k"]), pr["b"], tol=TOL, max_cycles=100)
    x = np.zeros_like(pr["b"])
    for (i0, i1, j0, j1), xb, info in results:
        x[j0 - 1:j1, i0 - 1:i1] = xb
        assert info.cycles == ref.cycles, (info.cycles, ref.cycles)
        assert abs(info.rel_resid - ref.rel_resid) <= 1e-13
        np.testing.assert_allclose(info.history, ref.history, rtol=1e-9, atol=1e-13)
    assert np.abs(x - ref.x).max() <= 1e-10 * np.abs(ref.x).max()


@pytest.mark.parametrize("px,py,m", [(2, 1, 2), (1, 2, 3), (2, 2, 1), (2, 2, 4), (3, 2, 2)])
def test_thread_ranks_reproduce_the_single_domain_solve(px, py, m):
    pr = _problem(63, seed=21)
    res = dd.run_threads(px * py, lambda comm: _solve_ranks(comm, pr, px, py, m))
    _check(pr, res)


def test_rectangular_grid_and_uneven_blocks():
    pr = inputs.block_problem(seed=22, block=8, lo=-2, hi=2, nx=127, ny=31)
    res = dd.run_threads(6, lambda comm: _solve_ranks(comm, pr, 3, 2, 2))
    _check(pr, res)


def test_layout_alignment_and_rules():
    shapes = [(3, 3), (7, 7), (15, 15), (31, 31), (63, 63)]
    lay = dd.Layout(shapes, 2, 2, 3)
    # fine blocks start at 0-based multiples of 2^3
    assert lay.xr[-1] == [(1, 32), (33, 63)]
    assert lay.xr[0] == [(1, 4), (5, 7)]            # gather level 7 x 7
    # every coarse range is the coarse points of its fine range
    for k in range(lay.nlev - 1):
        for (lo, hi), (clo, chi) in zip(lay.xr[k + 1], lay.xr[k]):
            assert (clo, chi) == ((lo + 1) // 2, hi // 2)
    with pytest.raises(ValueError):
        dd.Layout(shapes, 4, 1, 4)                  # 16-aligned blocks: only 4 units of 63 -> empty
    # whole 64-point units (the 3 points 255 keeps after six coarsenings);
    # the last block takes the remainder, and four blocks do not fit
    assert dd.split(255, 3, 64) == [(1, 64), (65, 128), (129, 255)]
    with pytest.raises(ValueError):
        dd.split(255, 4, 64)
    # 255^2 on 2 x 2: the smallest blocks of the 127^2 level hold 63^2 = 3969
    # points, of the 63^2 level 31^2 = 961, of the 31^2 level 15^2 = 225
    big = [(3, 3), (7, 7), (15, 15), (31, 31), (63, 63), (127, 127), (255, 255)]
    assert dd.choose_dist_levels(big, 2, 2, min_local=1024) == 2
    assert dd.choose_dist_levels(big, 2, 2, min_local=200) == 4
    nb = lay.neighbours(0)
    assert nb == {dd.EAST: 1, dd.NORTH: 2}
    assert lay.neighbours(3) == {dd.WEST: 2, dd.SOUTH: 1}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_worker(rank, world, port, px, py, m, n, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pr = _problem(n, seed=23)
        out[rank] = _solve_ranks(dd.TorchComm(), pr, px, py, m)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("px,py,m", [(2, 1, 3), (2, 2, 2)])
def test_gloo_ranks_reproduce_the_single_domain_solve(px, py, m):
    world = px * py
    n = 63
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_gloo_worker, args=(world, _free_port(), px, py, m, n, out), nprocs=world,
                           start_method="spawn", join=True)
        res = [out[r] for r in range(world)]
    _check(_problem(n, seed=23), res)


def test_a_failed_rank_surfaces_instead_of_hanging():
    """A rank that raises before the first exchange ends the run with its
    error (the other ranks' waits are bounded), and no rank blocks forever."""
    pr = _problem(63, seed=24)

    def body(comm):
        if comm.rank == 1:
            raise RuntimeError("rank 1 failed")
        return _solve_ranks(comm, pr, 2, 1, 2)

    with pytest.raises(RuntimeError, match="rank 1 failed"):
        dd.run_threads(2, body)


class _DyingComm(dd.TorchComm):
    """TorchComm whose rank `victim` dies (the process exits at once, as a
    crashed rank would) at its `after`-th exchange."""

    def __init__(self, victim, after):
        super().__init__()
        self.victim, self.after, self.n = victim, after, 0

    def exchange(self, sends, recvs):
        self.n += 1
        if self.rank == self.victim and self.n == self.after:
            os._exit(3)
        return super().exchange(sends, recvs)


def _gloo_dying_worker(rank, world, port, out):
    import datetime
    import time
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.set_num_threads(1)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    pr = _problem(31, seed=25)
    comm = _DyingComm(victim=1, after=40)
    t0 = time.monotonic()
    try:
        _solve_ranks(comm, pr, 2, 1, 2)
        out[rank] = ("finished", time.monotonic() - t0)
    except Exception as e:  # noqa: BLE001 - the error is the result
        out[rank] = ("error: " + type(e).__name__ + ": " + str(e)[:200], time.monotonic() - t0)
    os._exit(0)


def test_a_dead_gloo_rank_ends_the_others_solve_with_an_error():
    """Failure detection across processes: rank 1 dies in the middle of a
    V-cycle (between two halo exchanges); rank 0's next exchange with it
    fails within the process group's timeout instead of blocking forever."""
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        pc = mp.start_processes(_gloo_dying_worker, args=(world, _free_port(), out), nprocs=world,
                                start_method="spawn", join=False)
        codes = {}
        deadline = 120.0
        import time
        t0 = time.monotonic()
        while len(codes) < world and time.monotonic() - t0 < deadline:
            for r, proc in enumerate(pc.processes):
                if r not in codes and not proc.is_alive():
                    codes[r] = proc.exitcode
            time.sleep(0.2)
        for proc in pc.processes:
            if proc.is_alive():
                proc.kill()
        res = dict(out)
    assert codes == {0: 0, 1: 3}, codes
    status, seconds = res[0]
    assert status.startswith("error"), status
    assert seconds < 60.0


# ---------------------------------------------------------------------------
# Multi-stage redistribution plans (Section 2.2, Algorithm 2; Section 4)
# ---------------------------------------------------------------------------

def _coarsen(r, m):
    for _ in range(m):
        r = dd.coarse_range(*r)
    return r


def _check_plan(plan):
    """Blocks tile every level, start on the stage's alignment, and a coarse
    task's block is the union of its processor block's blocks; every rank
    runs a prefix of the stages; the coarse task runs on rank 0."""
    for s, st in enumerate(plan.stages):
        for k in range(st.nlev):
            nx, ny = plan.shapes[st.lo + k]
            for rng, n in ((st.xr[k], nx), (st.yr[k], ny)):
                assert rng[0][0] == 1 and rng[-1][1] == n
                assert all(b[0] == a[1] + 1 for a, b in zip(rng, rng[1:]))
        for lo, _ in st.xr[-1] + st.yr[-1]:
            assert (lo - 1) % 2 ** (st.nlev - 1) == 0
        if s + 1 < plan.nstage:
            nxt = plan.stages[s + 1]
            for d, (mine, theirs) in enumerate(((st.xr[0], nxt.xr[-1]), (st.yr[0], nxt.yr[-1]))):
                for g, members in enumerate(plan.grp[s][d]):
                    assert (mine[members[0]][0], mine[members[-1]][1]) == theirs[g]
    for r in range(plan.size):
        assert [t[0] for t in plan.roles[r]] == list(range(len(plan.roles[r])))
    assert 0 in plan.coarse_ranks()


def test_plan_layouts_tile_nest_and_balance():
    shapes = [(7, 3), (15, 7), (31, 15), (63, 31), (127, 63), (255, 127)]
    for path, red in [([((4, 2), 5), ((2, 1), 3), ((1, 1), 1)], False),
                      ([((4, 2), 5), ((2, 2), 4), ((2, 1), 2), ((1, 1), 0)], False),
                      ([((3, 2), 5), ((2, 1), 3), ((1, 1), 2)], False),
                      ([((4, 2), 5), ((2, 1), 3), ((1, 1), 1)], True),
                      ([((4, 4), 5), ((2, 2), 3), ((1, 1), 2)], True)]:
        plan = dd.Plan(shapes, path, red)
        _check_plan(plan)
        if red:
            # every fine rank runs the coarse task of one copy
            assert plan.coarse_ranks() == list(range(plan.size))
        else:
            assert plan.coarse_ranks() == [0]
    # 3 ranks agglomerated into groups of 1 and 2: the coarse split follows the
    # rank counts, so the finest blocks stay balanced (85 = 255 / 3 points each,
    # within the coarse stage's alignment of 2 points on level 3, 8 on level 5)
    plan = dd.Plan(shapes, [((3, 2), 5), ((2, 1), 3), ((1, 1), 2)])
    widths = [hi - lo + 1 for lo, hi in plan.stages[0].xr[-1]]
    assert max(widths) - min(widths) <= 8 and sum(widths) == 255
    assert plan.grp[0][0] == [[0], [1, 2]]
    with pytest.raises(ValueError):
        dd.Plan(shapes, [((3, 2), 5), ((2, 1), 3), ((1, 1), 2)], redundant=True)
    with pytest.raises(ValueError):
        dd.Plan(shapes, [((4, 2), 5), ((4, 2), 3), ((1, 1), 2)])
    with pytest.raises(ValueError):
        dd.Plan(shapes, [((4, 2), 5), ((2, 1), 3)])


def test_search_plan_on_the_minimum_local_size_rule():
    shapes = [(3, 3), (7, 7), (15, 15), (31, 31), (63, 63), (127, 127), (255, 255), (511, 511)]
    plan, res = dd.search_plan(shapes, (8, 8), min_local=256)
    _check_plan(plan)
    assert plan.path == res.path and plan.path[0] == ((8, 8), 7) and plan.path[-1][0] == (1, 1)


def _solve_plan(comm, pr, P, path, redundant, cycles, min_local=64):
    h = O.setup(pr["k"])
    src = OracleSource(h)
    shapes = [src.level_shape(l) for l in range(src.nlevels)]
    plan = dd.make_plan(shapes, P[0], P[1], path=path, redundant=redundant, min_local=min_local)
    parts = [CpuPart(p) for p in dd.plan_payloads(src, plan, comm.rank)]
    coarse = src if comm.rank in plan.coarse_ranks() else None
    solver = dd.DDSolver(comm, plan, parts, coarse=coarse)
    (i0, i1), (j0, j1) = solver.block()
    b = torch.from_numpy(np.ascontiguousarray(pr["b"][j0 - 1:j1, i0 - 1:i1]))
    x, info = solver.solve(b, tol=1e-300, max_cycles=cycles)
    return (i0, i1, j0, j1), x.numpy().copy(), info


def _check_cycles(pr, results, cycles):
    ref = O.solve(O.setup(pr["k"]), pr["b"], tol=1e-300, max_cycles=cycles)
    x = np.zeros_like(pr["b"])
    for (i0, i1, j0, j1), xb, info in results:
        x[j0 - 1:j1, i0 - 1:i1] = xb
        assert info.cycles == cycles
        np.testing.assert_allclose(info.history, ref.history, rtol=1e-9, atol=1e-15)
    assert np.abs(x - ref.x).max() <= 1e-12 * np.abs(ref.x).max()


@pytest.mark.parametrize("P,path,red", [
    ((4, 2), [(4, 2), (2, 1), (1, 1)], False),
    ((4, 2), [(4, 2), (2, 1), (1, 1)], True),
    ((3, 2), [(3, 2), (2, 1), (1, 1)], False),
    ((4, 2), [((4, 2), 4), ((2, 2), 2), ((2, 1), 1), ((1, 1), 0)], False),
    ((4, 4), "search", False),
    ((4, 4), [(4, 4), (2, 2), (1, 1)], True),
])
def test_thread_ranks_on_a_redistribution_path_reproduce_the_single_domain_cycles(P, path, red):
    pr = inputs.block_problem(seed=31, block=8, lo=-2, hi=2, nx=127, ny=63)
    res = dd.run_threads(P[0] * P[1], lambda comm: _solve_plan(comm, pr, P, path, red, 3), timeout=120.0)
    _check_cycles(pr, res, 3)


def _gloo_plan_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.set_num_threads(1)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pr = inputs.block_problem(seed=32, block=8, lo=-2, hi=2, nx=127, ny=63)
        out[rank] = _solve_plan(dd.TorchComm(), pr, (2, 2), [(2, 2), (2, 1), (1, 1)], False, 3)
    finally:
        dist.destroy_process_group()


def test_gloo_ranks_on_a_two_stage_path():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_gloo_plan_worker, args=(4, _free_port(), out), nprocs=4,
                           start_method="spawn", join=True)
        res = [out[r] for r in range(4)]
    _check_cycles(inputs.block_problem(seed=32, block=8, lo=-2, hi=2, nx=127, ny=63), res, 3)
