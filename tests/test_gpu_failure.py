"""Failure detection without a GPU fault.

The TMA-staged sweeps wait for their bulk copies on mbarriers, and every
such wait is bounded: after about one second it records DEV_TIMEOUT in the
device error word and the kernel returns.  The self-test entry point runs
that wait on a barrier phase that expects bytes no copy delivers (a flag
nothing sets); the call must come back with BMG_ETIMEOUT after about a
second, and the context must stay usable for a solve afterwards.
"""
import time

import numpy as np
import pytest

from oracle import boxmg_oracle as O
from paper_1803_02481_gb300 import inputs

torch = pytest.importorskip("torch")
import paper_1803_02481_gb300 as bm  # noqa: E402

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_context_stays_usable():
    t0 = time.perf_counter()
    rc = bm.selftest_bounded_wait()
    dt = time.perf_counter() - t0
    assert rc == bm.BMG_ETIMEOUT
    assert 0.5 <= dt <= 30.0, dt
    # the context still works: a small solve matches the oracle
    pr = inputs.block_problem(seed=5, block=8, lo=-3, hi=3, nx=127, ny=31)
    h = bm.setup(torch.from_numpy(pr["k"]).cuda())
    x, info = h.solve(torch.from_numpy(pr["b"]).cuda(), tol=1e-10)
    h.destroy()
    ro = O.solve(O.setup(pr["k"]), pr["b"], tol=1e-10, max_cycles=400)
    assert info.cycles == ro.cycles
    assert np.abs(x.cpu().numpy() - ro.x).max() <= 1e-9 * np.abs(ro.x).max()
