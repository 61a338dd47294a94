"""Batched solves (many uneven problems, FP32 V-cycles inside FP64
refinement, one graph launch) against individual solves and the oracle."""
import numpy as np
import pytest

from oracle import boxmg_oracle as O
from paper_1803_02481_gb300 import inputs

torch = pytest.importorskip("torch")
import paper_1803_02481_gb300 as bm  # noqa: E402

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel_resid(k, x, b):
    st = O.assemble_fv5(k)
    return np.linalg.norm(O.residual(st, x, b)) / np.linalg.norm(b)


def test_small_mixed_batch_matches_individual_solves_and_oracle():
    probs = inputs.batch_problems(count=11, seed=4, sides=(63, 127, 255), weights=(4, 2, 1))
    probs.append({"n": 63, "k": np.ones((63, 63)), "b": np.zeros((63, 63))})   # zero RHS
    ks = [dev(p["k"]) for p in probs]
    bs = [dev(p["b"]) for p in probs]
    xs = [torch.zeros_like(b) for b in bs]
    batch = bm.Batch(ks)
    infos = batch.solve(bs, xs, tol=1e-8)
    for p, x, info, k, b in zip(probs, xs, infos, ks, bs):
        xn = x.cpu().numpy()
        if not p["b"].any():
            assert info.cycles == 0 and not xn.any()
            continue
        assert info.rel_resid <= 1e-8
        assert rel_resid(p["k"], xn, p["b"]) <= 1.000001e-8
        # the same problem solved on its own with the same method
        h = bm.setup(k, bm.default_options(precision=bm.BMG_FP32_REFINE))
        xi, ii = h.solve(b, tol=1e-8)
        h.destroy()
        assert abs(ii.cycles - info.cycles) <= 1
        xo = O.direct_solve(p["k"], p["b"])
        scale = np.abs(xo).max()
        assert np.abs(xn - xo).max() <= 1e-5 * scale
        assert np.abs(xn - xi.cpu().numpy()).max() <= 1e-5 * scale
    batch.destroy()


def test_full_batch_every_problem_meets_tolerance():
    """All 512 problems of the batched workload (sides 63..1023, 10^[-3,3]
    blocks): every returned x satisfies ||b - A x|| / ||b|| <= 1e-8 with the
    oracle's operator; a sample agrees with its individual solve."""
    probs = inputs.batch_problems(count=512, seed=4)
    ks = [dev(p["k"]) for p in probs]
    bs = [dev(p["b"]) for p in probs]
    xs = [torch.zeros_like(b) for b in bs]
    # the slowest 1023^2 problems need about 2300 refinement steps (their
    # 16-cell blocks are narrower than a coarse cell on the 63^2 level)
    batch = bm.Batch(ks, bm.default_options(max_cycles=3000))
    infos = batch.solve(bs, xs, tol=1e-8)
    for p, x, info in zip(probs, xs, infos):
        assert info.rel_resid <= 1e-8
        assert rel_resid(p["k"], x.cpu().numpy(), p["b"]) <= 1.000001e-8
    for q in (0, 17, 100, 311):
        h = bm.setup(ks[q], bm.default_options(precision=bm.BMG_FP32_REFINE, max_cycles=3000))
        xi, ii = h.solve(bs[q], tol=1e-8)
        h.destroy()
        assert abs(ii.cycles - infos[q].cycles) <= 1
        scale = xi.abs().max().item()
        assert (xi - xs[q]).abs().max().item() <= 1e-5 * scale
    batch.destroy()


def _pcg_options(**kw):
    return bm.default_options(nu1=1, nu2=1, solver=bm.BMG_SOLVER_PCG, **kw)


def test_batched_pcg_matches_individual_solves_and_oracle():
    """Batched CG preconditioned by the symmetric FP32 V(1,1) cycle: every
    problem meets the FP64 stop test against the oracle's operator, within
    a few iterations of the same problem's own PCG solve with FP32 cycles
    and close to its iterate; a zero right-hand side runs no iteration."""
    probs = inputs.batch_problems(count=11, seed=5, sides=(63, 127, 255), weights=(4, 2, 1))
    probs.append({"n": 127, "k": np.ones((127, 127)), "b": np.zeros((127, 127))})   # zero RHS
    ks = [dev(p["k"]) for p in probs]
    bs = [dev(p["b"]) for p in probs]
    xs = [torch.zeros_like(b) for b in bs]
    batch = bm.Batch(ks, _pcg_options(max_cycles=500))
    infos = batch.solve(bs, xs, tol=1e-10)
    for p, x, info, k, b in zip(probs, xs, infos, ks, bs):
        xn = x.cpu().numpy()
        if not p["b"].any():
            assert info.cycles == 0 and not xn.any()
            continue
        assert info.rel_resid <= 1e-10
        assert rel_resid(p["k"], xn, p["b"]) <= 2e-10
        h = bm.setup(k, _pcg_options(precision=bm.BMG_FP32_REFINE, max_cycles=500))
        xi, ii = h.solve(b, tol=1e-10)
        h.destroy()
        assert abs(ii.cycles - info.cycles) <= 2, (ii.cycles, info.cycles)
        xo = O.direct_solve(p["k"], p["b"])
        scale = np.abs(xo).max()
        assert np.abs(xn - xo).max() <= 1e-7 * scale
        assert np.abs(xn - xi.cpu().numpy()).max() <= 1e-7 * scale
    batch.destroy()
    with pytest.raises(bm.BoxMGError):
        bm.Batch(ks[:2], bm.default_options(solver=bm.BMG_SOLVER_PCG))     # V(2,1): not symmetric


def test_full_batch_pcg_every_problem_meets_tolerance():
    """All 512 problems of the batched workload with batched PCG (FP32 V(1,1)
    cycles): every returned x satisfies the stop test with the oracle's
    operator, in a few dozen iterations where the V-cycle refinement needs
    up to about 2300 steps."""
    probs = inputs.batch_problems(count=512, seed=4)
    ks = [dev(p["k"]) for p in probs]
    bs = [dev(p["b"]) for p in probs]
    xs = [torch.zeros_like(b) for b in bs]
    batch = bm.Batch(ks, _pcg_options(max_cycles=500))
    infos = batch.solve(bs, xs, tol=1e-8)
    for p, x, info in zip(probs, xs, infos):
        assert info.rel_resid <= 1e-8
        assert rel_resid(p["k"], x.cpu().numpy(), p["b"]) <= 2e-8
    assert max(i.cycles for i in infos) < 150
    batch.destroy()
