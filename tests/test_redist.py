"""Model-guided redistribution (Sections 3-4): the V-cycle performance model,
the coarse processor grid enumeration and the path search, pinned by the
paper's printed examples and by the mathematics of the search.

* the enumeration reproduces the paper's worked example (the 9088 x 568
  problem on 16 x 8 processors) and offers log2(n_p) grids on a
  power-of-two processor grid;
* the nine paths the paper prints for a 64 x 32 grid with 568 x 71 local
  problems are paths of the search space, and the model ranks the paper's
  selected path (Path 1) cheapest of them, far below all-to-one (Path 0);
* brute force visits 2^h states when every state can reach every coarser
  grid of an h-grid enumeration (the paper's recurrence T(h) = 2^h);
* A* with its heuristic returns the brute-force optimum on random spaces and
  expands far fewer states; the heuristic never exceeds the optimal cost to
  the goal;
* the model's terms agree with their definitions on hand-counted cases, in
  2D and in 3D (the paper's 3D interpolation count); the 3D search space
  has the same properties.
"""
import math
import os
import random

import pytest

from paper_1803_02481_gb300 import redist as R

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def _paper_space(min_local=1024, cycle=R.Cycle()):
    # 568 x 71 local problems on 64 x 32 processors, coarsened by 2 (ceil)
    return R.Space(R.halving_shapes((568 * 64, 71 * 32)), (64, 32), R.BLUE_WATERS, cycle, min_local)


def _paper_paths():
    out = {}
    for row in _rows("redistribution_paths_64x32.txt"):
        grids = [tuple(int(v) for v in g.split("x")) for g in row[1:]]
        if grids[-1] != (1, 1):
            grids.append((1, 1))        # Path 2 continues to one processor
        out[int(row[0])] = grids
    return out


def test_blue_waters_parameters_match_the_table():
    (a, b, g), = [[float(v) for v in r] for r in _rows("model_parameters_blue_waters.txt")]
    bw = R.BLUE_WATERS
    assert (bw.alpha, bw.beta, bw.gamma) == pytest.approx((a * 1e-6, b * 1e-9, g * 1e-9), rel=1e-12)


def test_enumeration_reproduces_the_worked_example():
    want = [tuple(int(v) for v in r) for r in _rows("redistribution_enumeration_1136x71_on_16x8.txt")]
    got = R.enumerate_grids((1136, 71), (16, 8))
    assert got == [w[:2] for w in want]
    assert [R.local((1136, 71), g) for g in got] == [w[2:] for w in want]


@pytest.mark.parametrize("seed", range(20))
def test_enumeration_is_a_chain_of_log2_np_grids(seed):
    rng = random.Random(seed)
    q = (rng.randint(1, 70), rng.randint(1, 70)) if seed % 2 else (2 ** rng.randint(0, 7), 2 ** rng.randint(0, 7))
    if q == (1, 1):
        q = (2, 1)
    N = (rng.randint(q[0], 5000), rng.randint(q[1], 5000))
    grids = R.enumerate_grids(N, q)
    assert grids[0] == (1, 1)
    # log2(n_p) grids for power-of-two grids; a capped factor adds a step per dimension
    assert len(grids) == sum(math.ceil(math.log2(v)) for v in q)
    if all(v & (v - 1) == 0 for v in q):
        assert len(grids) == math.log2(q[0] * q[1])
    for g, g2 in zip(grids, grids[1:] + [q]):
        # each step doubles one dimension (or caps it at q) and keeps the other
        d = 0 if g2[0] != g[0] else 1
        assert g2[1 - d] == g[1 - d] and g2[d] == min(2 * g[d], q[d])


def test_the_papers_paths_are_paths_of_the_search_space_and_path_1_is_cheapest():
    sp = _paper_space()
    cost = {k: sp.path_cost(sp.states_of_grids(g)) for k, g in _paper_paths().items()}
    assert min(cost, key=cost.get) == 1
    # all-to-one is over an order of magnitude slower (measured: 40x)
    assert 20 < cost[0] / cost[1] < 100
    best = R.search_astar(sp)
    assert best.cost <= cost[1] * (1 + 1e-12)
    # the optimum shares Path 1's first four grids and ends in 16 x 1 -> 1 x 1
    grids = [q for q, _ in best.path]
    assert grids[:4] == _paper_paths()[1][:4] and grids[-2:] == [(16, 1), (1, 1)]


def test_brute_force_visits_two_to_the_h_states():
    # a 1-D grid of 2^h processors: the enumeration is 1, 2, ..., 2^(h-1);
    # a coarsening limit on every level lets each state reach every coarser grid
    for h in range(1, 7):
        P = (2 ** h, 1)
        shapes = R.halving_shapes((2 ** 14, 2 ** 14))
        sp = R.Space(shapes, P, min_local=10 ** 18)
        res = R.search_brute_force(sp)
        assert res.expanded == 2 ** h == P[0] * P[1]


def _random_space(rng):
    P = (2 ** rng.randint(0, 4) * rng.choice([1, 1, 3]), 2 ** rng.randint(0, 4))
    if P == (1, 1):
        P = (4, 2)
    n = (rng.randint(60, 4000), rng.randint(60, 4000))
    machine = R.Machine(alpha=10 ** rng.uniform(-7, -4), beta=10 ** rng.uniform(-11, -8),
                        gamma=10 ** rng.uniform(-11, -9))
    return R.Space(R.halving_shapes((n[0] * P[0] // 4 + 7, n[1] * P[1] // 4 + 7)), P, machine,
                   R.Cycle(), min_local=rng.choice([16, 64, 256, 1024, 4096]),
                   redundant=rng.random() < 0.3)


@pytest.mark.parametrize("seed", range(25))
def test_astar_returns_the_brute_force_optimum(seed):
    sp = _random_space(random.Random(seed))
    a, b = R.search_astar(sp), R.search_brute_force(sp)
    assert a.cost == pytest.approx(b.cost, rel=1e-12)
    assert sp.path_cost(a.path) == pytest.approx(a.cost, rel=1e-12)
    assert a.expanded <= b.expanded


def test_astar_expands_far_fewer_states_on_the_papers_example():
    sp = _paper_space()
    a, b = R.search_astar(sp), R.search_brute_force(sp)
    assert a.cost == pytest.approx(b.cost, rel=1e-12)
    assert a.expanded * 20 < b.expanded


@pytest.mark.parametrize("seed", range(6))
def test_heuristic_never_exceeds_the_optimal_cost_to_go(seed):
    sp = _random_space(random.Random(100 + seed))
    memo = {}

    def opt(state):                      # exact cost to the goal, by recursion
        if state not in memo:
            memo[state] = min(c + (0.0 if s2 is None else opt(s2)) for s2, c in sp.edges(state))
        return memo[state]

    seen, stack = set(), [sp.start]
    while stack:
        s = stack.pop()
        if s in seen:
            continue
        seen.add(s)
        assert sp.heuristic(s) <= opt(s) * (1 + 1e-12)
        stack += [s2 for s2, _ in sp.edges(s) if s2 is not None]


def test_model_terms_on_hand_counted_cases():
    m = R.Machine(alpha=1.0, beta=1e-3, gamma=1e-6)
    # halo of a 10 x 20 block on a 2 x 2 grid: 4 messages, 2 * (10 + 20) values
    assert R.t_exchange((10, 20), (2, 2), m) == pytest.approx(4 + 2 * 30 * 8e-3)
    # split in x only: the west and east strips of 20 values
    assert R.t_exchange((10, 20), (2, 1), m) == pytest.approx(2 + 2 * 20 * 8e-3)
    assert R.t_exchange((10, 20), (1, 1), m) == 0.0
    # gather over 4 ranks: 2 latency steps, 3/4 of the block through the root
    assert R.t_gather(4, 100, m) == pytest.approx(2 + 100 * 0.75 * 8e-3)
    assert R.t_gather(5, 100, m) == pytest.approx(3 + 100 * 0.8 * 8e-3)
    # 8 x 4 -> 2 x 1: processor blocks of 4 x 4, the 15 x 7 level on 2 x 1 is 8 x 7 per rank
    assert R.t_agglomerate((15, 7), (8, 4), (2, 1), m) == pytest.approx(2 * (4 + 56 * 15 / 16 * 8e-3))
    assert R.t_agglomerate((15, 7), (8, 4), (2, 1), m, redundant=True) == pytest.approx(
        4 + 56 * 15 / 16 * 8e-3)
    # level 1 (7 x 7, 9-point, 4 colours) of a 3-level hierarchy on 1 x 1, V(2,1):
    # smoothing 2*9*49*3, residual and restriction 2*9*49 each, interpolation
    # 49 + 20*9 + 6*6 flops (coarse 3 x 3)
    shapes = [(3, 3), (7, 7), (15, 15)]
    want = (2 * 9 * 49 * 3 + 2 * 2 * 9 * 49 + 49 + 20 * 9 + 36) * 1e-6
    assert R.level_time(shapes, 1, (1, 1), m, R.Cycle()) == pytest.approx(want)
    # the finest level uses the 5-point stencil and two colours
    want = (2 * 5 * 225 * 3 + 2 * 2 * 5 * 225 + 225 + 20 * 49 + 6 * 14) * 1e-6
    assert R.level_time(shapes, 2, (1, 1), m, R.Cycle()) == pytest.approx(want)
    assert R.t_cgsolve_factor(shapes, m) == pytest.approx(81 * 1e-6)


# ---------------------------------------------------------------------------
# 3D: the paper's 3D interpolation count, and the search over 3D grids
# ---------------------------------------------------------------------------

def test_3d_model_terms_on_hand_counted_cases():
    m = R.Machine(alpha=1.0, beta=1e-3, gamma=1e-6)
    # a 10 x 20 x 30 block split in every dimension: faces 600, 300, 200
    assert R.t_exchange((10, 20, 30), (2, 2, 2), m) == pytest.approx(6 + 2 * 1100 * 8e-3)
    assert R.t_exchange((10, 20, 30), (1, 1, 2), m) == pytest.approx(2 + 2 * 200 * 8e-3)
    # 3D interpolation onto a 5^3 block from a 2^3 coarse block:
    # 125 + 60 * 8 + 15 * 2 * 2 + 6 * 2 * 2 + 2 flops
    assert R.interp_flops((5, 5, 5), (2, 2, 2)) == 125 + 480 + 60 + 24 + 2
    # level 1 (7^3, 27-point, 8 colours) of a 3-level hierarchy on one
    # processor, V(2,1): smoothing 2*27*343*3, residual and restriction
    # 2*27*343 each, interpolation 343 + 60*27 + 15*9 + 6*9 + 3
    shapes = [(3, 3, 3), (7, 7, 7), (15, 15, 15)]
    want = (2 * 27 * 343 * 3 + 2 * 2 * 27 * 343 + 343 + 60 * 27 + 15 * 9 + 6 * 9 + 3) * 1e-6
    assert R.level_time(shapes, 1, (1, 1, 1), m, R.Cycle()) == pytest.approx(want)
    # the finest level: 7-point, red-black
    want = (2 * 7 * 3375 * 3 + 2 * 2 * 7 * 3375 + 3375 + 60 * 343 + 15 * 49 + 6 * 49 + 7) * 1e-6
    assert R.level_time(shapes, 2, (1, 1, 1), m, R.Cycle()) == pytest.approx(want)
    # gather over 2 x 2 x 2 -> 1: three latency steps
    assert R.t_agglomerate((7, 7, 7), (2, 2, 2), (1, 1, 1), m, redundant=True) == pytest.approx(
        3 + 343 * 7 / 8 * 8e-3)
    assert R.t_cgsolve_factor(shapes, m) == pytest.approx(27 ** 2 * 1e-6)


@pytest.mark.parametrize("seed", range(10))
def test_3d_enumeration_is_a_chain(seed):
    rng = random.Random(200 + seed)
    q = tuple(2 ** rng.randint(0, 4) for _ in range(3))
    if q == (1, 1, 1):
        q = (2, 2, 1)
    N = tuple(rng.randint(q[d], 3000) for d in range(3))
    grids = R.enumerate_grids(N, q)
    assert grids[0] == (1, 1, 1)
    assert len(grids) == math.log2(q[0] * q[1] * q[2])
    for g, g2 in zip(grids, grids[1:] + [q]):
        changed = [d for d in range(3) if g2[d] != g[d]]
        assert len(changed) == 1 and g2[changed[0]] == 2 * g[changed[0]]


@pytest.mark.parametrize("seed", range(10))
def test_3d_astar_returns_the_brute_force_optimum(seed):
    rng = random.Random(300 + seed)
    P = tuple(2 ** rng.randint(0, 3) for _ in range(3))
    if P == (1, 1, 1):
        P = (2, 2, 2)
    machine = R.Machine(alpha=10 ** rng.uniform(-7, -4), beta=10 ** rng.uniform(-11, -8),
                        gamma=10 ** rng.uniform(-11, -9))
    N = tuple(rng.randint(40, 160) * P[d] for d in range(3))
    sp = R.Space(R.halving_shapes(N), P, machine, R.Cycle(), min_local=rng.choice([64, 512, 4096]),
                 redundant=rng.random() < 0.3)
    a, b = R.search_astar(sp), R.search_brute_force(sp)
    assert a.cost == pytest.approx(b.cost, rel=1e-12)
    assert sp.path_cost(a.path) == pytest.approx(a.cost, rel=1e-12)
    assert a.path[0] == (P, len(sp.shapes) - 1) and a.path[-1][0] == (1, 1, 1)


def test_paths_always_end_on_one_processor_and_execute_as_plans():
    """A grid that keeps the coarsening limit down to level 1 hands level 0
    to one processor as an explicit last state, so every searched path is a
    runnable redistribution plan."""
    from paper_1803_02481_gb300 import dd
    shapes = [(3, 3), (7, 7), (15, 15), (31, 31), (63, 63)]
    sp = R.Space(shapes, (2, 2), min_local=4)          # 2 x 2 keeps >= 4 points to level 1
    res = R.search_astar(sp)
    assert res.path[-1] == ((1, 1), 0)
    assert sp.states_of_grids([(2, 2), (1, 1)]) == [((2, 2), 4), ((1, 1), 0)]
    dd.Plan(shapes, res.path)
    for seed in range(5):
        sp = _random_space(random.Random(500 + seed))
        if sp.redundant:
            continue
        path = R.search_astar(sp).path
        assert path[-1][0] == sp.one
        dd.Plan(sp.shapes, path)
