"""Domain-decomposed solve on the GPU: several blocks of one GPU, driven in
lockstep by thread ranks (Section 2.1 halo exchange per colour, residual and
restriction; Algorithm 2 gather to rank 0, which runs the coarse levels with
the single-GPU schedule, and scatter back).  Every block operation runs the
same per-point kernels as the single-domain solve, and the coarse cycle on
rank 0 is the single-domain cycle's lower part, so the iterate must equal the
single-domain solve's bit for bit; only the stop test's partial sums are
added in another order."""
import numpy as np
import pytest

from paper_1803_02481_gb300 import inputs

torch = pytest.importorskip("torch")
import paper_1803_02481_gb300 as bm  # noqa: E402
from paper_1803_02481_gb300 import dd  # noqa: E402

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _dd_solve(pr, px, py, m, tol=1e-10):
    k = dev(pr["k"])

    def body(comm):
        solver, _ = dd.cuda_setup(comm, (px, py, m), k if comm.rank == 0 else None)
        (i0, i1), (j0, j1) = solver.block()
        x, info = solver.solve(dev(pr["b"][j0 - 1:j1, i0 - 1:i1]), tol=tol, max_cycles=300)
        solver.destroy()
        return (i0, i1, j0, j1), x.cpu().numpy(), info, solver.plan.path[1][1]

    res = dd.run_threads(px * py, body, timeout=300.0)
    x = np.zeros_like(pr["b"])
    for (i0, i1, j0, j1), xb, _, _ in res:
        x[j0 - 1:j1, i0 - 1:i1] = xb
    return x, [r[2] for r in res], res[0][3]


@pytest.mark.parametrize("px,py,m", [(2, 2, 2), (2, 2, 4), (3, 1, 3), (1, 2, 1)])
def test_dd_blocks_reproduce_the_single_domain_solve(px, py, m):
    pr = inputs.block_problem(255, seed=1, block=64, lo=-4, hi=4)
    h = bm.setup(dev(pr["k"]))
    xg, ig = h.solve(dev(pr["b"]), tol=1e-10)
    h.destroy()
    x, infos, gather = _dd_solve(pr, px, py, m)
    for info in infos:
        assert info.cycles == ig.cycles, (info.cycles, ig.cycles)
        assert abs(info.rel_resid - ig.rel_resid) <= 1e-13
    assert np.array_equal(x, xg.cpu().numpy())


def test_dd_on_a_rectangular_grid_with_the_minimum_local_size_rule():
    pr = inputs.block_problem(seed=6, block=64, lo=-2, hi=2, nx=1023, ny=255)
    h = bm.setup(dev(pr["k"]))
    xg, ig = h.solve(dev(pr["b"]), tol=1e-10)
    h.destroy()
    x, infos, gather = _dd_solve(pr, 4, 1, None)
    assert infos[0].cycles == ig.cycles
    assert np.array_equal(x, xg.cpu().numpy())


def test_dd_at_four_million_unknowns_reproduces_the_single_domain_solve():
    """1023 x 2047 block field (4.2 M unknowns, 11 levels) on 2 x 2 blocks
    with the gather level chosen by the minimum-local-size rule: the same
    bits as the single-domain solve."""
    pr = inputs.block_problem(seed=8, block=32, lo=-2, hi=2, nx=1023, ny=2047)
    h = bm.setup(dev(pr["k"]))
    xg, ig = h.solve(dev(pr["b"]), tol=1e-10)
    h.destroy()
    x, infos, gather = _dd_solve(pr, 2, 2, None)
    assert infos[0].cycles == ig.cycles, (infos[0].cycles, ig.cycles)
    assert np.array_equal(x, xg.cpu().numpy())


def test_vcycle_from_the_top_is_one_solve_cycle():
    """bmg_op_vcycle_from at the finest level from x = 0 is the first cycle
    of bmg_solve."""
    pr = inputs.block_problem(127, seed=3, block=16, lo=-2, hi=2)
    h = bm.setup(dev(pr["k"]), bm.default_options(max_cycles=1))
    x1, _ = h.solve(dev(pr["b"]), tol=1e-300, allow_noconv=True)
    xv = torch.zeros_like(x1)
    h.vcycle_from(h.nlevels - 1, dev(pr["b"]), xv)
    h.destroy()
    assert torch.equal(x1, xv)


def _plan_solve(pr, P, path, redundant=False, min_local=1024, tol=1e-10):
    k = dev(pr["k"])

    def body(comm):
        solver, _ = dd.cuda_setup(comm, P, k if comm.rank == 0 else None, path=path, redundant=redundant,
                                  min_local=min_local)
        (i0, i1), (j0, j1) = solver.block()
        x, info = solver.solve(dev(pr["b"][j0 - 1:j1, i0 - 1:i1]), tol=tol, max_cycles=300)
        solver.destroy()
        return (i0, i1, j0, j1), x.cpu().numpy(), info, solver.plan.path

    res = dd.run_threads(P[0] * P[1], body, timeout=600.0)
    x = np.zeros_like(pr["b"])
    for (i0, i1, j0, j1), xb, _, _ in res:
        x[j0 - 1:j1, i0 - 1:i1] = xb
    return x, [r[2] for r in res], res[0][3]


@pytest.mark.parametrize("P,path,red", [
    ((4, 2), [(4, 2), (2, 1), (1, 1)], False),
    ((4, 2), [(4, 2), (2, 1), (1, 1)], True),
    ((4, 4), [(4, 4), (2, 2), (1, 1)], True),
    ((3, 2), [(3, 2), (2, 1), (1, 1)], False),
    ((4, 2), [((4, 2), 6), ((2, 2), 4), ((2, 1), 2), ((1, 1), 0)], False),
    ((4, 4), "search", False),
])
def test_dd_redistribution_paths_reproduce_the_single_domain_solve(P, path, red):
    """Multi-stage agglomeration (Algorithm 2 with p_l decreasing in several
    steps, Section 2.2's gather/scatter and redundant forms): the same bits
    as the single-domain solve on every path."""
    pr = inputs.block_problem(255, seed=4, block=64, lo=-4, hi=4)
    h = bm.setup(dev(pr["k"]))
    xg, ig = h.solve(dev(pr["b"]), tol=1e-10)
    h.destroy()
    x, infos, states = _plan_solve(pr, P, path, red, min_local=256)
    assert len(states) >= 2
    for info in infos:
        assert info.cycles == ig.cycles, (info.cycles, ig.cycles)
    assert np.array_equal(x, xg.cpu().numpy())


def test_dd_model_guided_path_at_four_million_unknowns():
    """1023 x 2047 block field on 4 x 4 blocks along the model's cheapest
    redistribution path (A* search, minimum local size 1024): the same bits
    as the single-domain solve."""
    pr = inputs.block_problem(seed=9, block=32, lo=-2, hi=2, nx=1023, ny=2047)
    h = bm.setup(dev(pr["k"]))
    xg, ig = h.solve(dev(pr["b"]), tol=1e-10)
    h.destroy()
    x, infos, states = _plan_solve(pr, (4, 4), "search")
    assert len(states) >= 3, states
    assert infos[0].cycles == ig.cycles, (infos[0].cycles, ig.cycles)
    assert np.array_equal(x, xg.cpu().numpy())
