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
    assert dd.split(255, 4, 64) == [(1, 64), (65, 128), (129, 192), (193, 255)]
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
