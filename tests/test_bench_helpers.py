"""Host-side helpers of bench.py checked on CPU.

The extended-precision residual the benchmark reports for its headline solve
evaluates b - A x from the library's stored planes (C, W, S, with the east
and north couplings read from the neighbours' W and S) in long double.  On a
small heterogeneous problem it must agree with the oracle's own FP64
residual to FP64 rounding, and a plane read in the wrong place (a dropped or
shifted coupling) must change it."""
import numpy as np
import pytest

from oracle import boxmg_oracle as O
from paper_1803_02481_gb300 import inputs

bench = pytest.importorskip("bench")


def _problem():
    pr = inputs.block_problem(63, seed=1, block=8, lo=-3, hi=3)
    st = O.assemble_fv5(pr["k"])
    x = np.random.default_rng(0).uniform(-1, 1, pr["b"].shape)
    return pr, st, x


def test_extended_residual_matches_the_oracle_residual():
    pr, st, x = _problem()
    ext = bench.extended_residual(st, x, pr["b"])
    ref = np.linalg.norm(O.residual(st, x, pr["b"])) / np.linalg.norm(pr["b"])
    assert abs(ext - ref) <= 1e-13 * ref


def test_extended_residual_sees_every_coupling():
    pr, st, x = _problem()
    ext = bench.extended_residual(st, x, pr["b"])
    for plane in ("W", "S"):
        bad = dict(st)
        bad[plane] = np.roll(st[plane], 1, axis=1 if plane == "W" else 0)
        assert abs(bench.extended_residual(bad, x, pr["b"]) - ext) > 1e-6 * ext, plane


def test_extended_residual_of_the_exact_solution_is_at_rounding_level():
    # x solving A x = b to FP64 (a sparse direct solve): the residual in long
    # double is at the size the FP64 rounding of x allows
    import scipy.sparse.linalg as spla
    pr, st, _ = _problem()
    a = O.stencil_to_csr(st)
    x = spla.spsolve(a.tocsc(), pr["b"].ravel()).reshape(pr["b"].shape)
    assert bench.extended_residual(st, x, pr["b"]) < 1e-12
