"""Every measured sweep shape (and the fused or separate residual and
restriction) gives the same bits.

The TMA-staged sweeps have tables of tile shapes (tile sides, threads,
blocks per SM, stages) selected once per process by environment variables:
BMG_TMA9_CFG (9-point levels, FP64 and FP32), BMG_TMA_PRE_CFG (the
prescaled FP64 finest level), BMG_TMA_CFG (5-point levels: FP32, and FP64
with BMG_RB_PRESCALE=0); BMG_RR_FUSED picks the levels whose residual and
restriction run as one kernel; BMG_ZERO_START=0 sweeps zero iterates (each
coarse level's, the FP32 finest level's in refinement) in the plain form.  The defaults are covered by the oracle parity
tests; here each other entry runs in a subprocess on a grid that puts every
level through the full-grid kernels (threshold 1), with ragged tiles on every
level, and its iterates must equal the default's bit for bit, in FP64, in
FP32 refinement and in PCG with the V(1,1) cycle (and its stop-test residuals too, except where the prescaled
sweep sums them: there another tile shape changes only the order of the sum).
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from tests.parity_helpers import problem

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
import torch
import paper_1803_02481_gb300 as bm
src, dst = sys.argv[1], sys.argv[2]
d = np.load(src)
dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
out, meta = {}, {}
for tag, prec, kw in (("fp64", bm.BMG_FP64, {}), ("fp32", bm.BMG_FP32_REFINE, {}),
                      ("pcg", bm.BMG_FP64, dict(nu1=1, nu2=1, solver=bm.BMG_SOLVER_PCG))):
    h = bm.setup(dev(d["k"]), bm.default_options(coarse_threshold=1, precision=prec, **kw))
    x, info = h.solve(dev(d["b"]), tol=1e-10)
    out[tag] = x.cpu().numpy()
    meta[tag] = [info.cycles, info.rel_resid]
    h.destroy()
np.savez(dst, **out)
print(json.dumps(meta))
"""


def run_child(tmp_path, name, env_extra):
    env = {k: v for k, v in os.environ.items() if not k.startswith("BMG")}
    env.update(env_extra)
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    src = tmp_path / "in.npz"
    if not src.exists():
        pr = problem("wide2047x127")
        np.savez(src, k=pr["k"], b=pr["b"])
    dst = tmp_path / f"{name}.npz"
    res = subprocess.run([sys.executable, "-c", CHILD, str(src), str(dst)], env=env, cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    meta = json.loads(res.stdout.strip().splitlines()[-1])
    with np.load(dst) as z:
        return {k: z[k] for k in z.files}, meta


SETTINGS = ([("nine%d" % k, {"BMG_TMA9_CFG": str(k)}) for k in range(1, 6)] +
            [("pre%d" % k, {"BMG_TMA_PRE_CFG": str(k)}) for k in range(1, 6)] +
            [("rb%d" % k, {"BMG_TMA_CFG": str(k)}) for k in range(1, 3)] +
            # residual and restriction fused into one kernel on every level, or on none
            [("rr%d" % k, {"BMG_RR_FUSED": str(k)}) for k in range(2)] +
            # first pre-sweeps of zero iterates in the plain form
            [("zero_start_off", {"BMG_ZERO_START": "0"})])


def test_every_sweep_shape_gives_identical_iterates(tmp_path):
    ref, ref_meta = run_child(tmp_path, "default", {})
    std, std_meta = run_child(tmp_path, "standard", {"BMG_RB_PRESCALE": "0"})
    assert ref_meta["fp64"][1] <= 1e-10 and std_meta["fp64"][1] <= 1e-10
    # the standard operator is the same step with different rounding; FP32
    # refinement never uses the prescaled level
    assert np.array_equal(std["fp32"], ref["fp32"])
    for name, env in SETTINGS:
        got, meta = run_child(tmp_path, name, env)
        for tag in ("fp64", "fp32", "pcg"):
            if name.startswith("pre") and tag == "fp64":
                # the stop test is summed inside the prescaled sweep, per tile
                # and block: another tile shape adds the same squares in
                # another order
                assert meta[tag][0] == ref_meta[tag][0], (name, meta[tag], ref_meta[tag])
                assert abs(meta[tag][1] - ref_meta[tag][1]) <= 1e-13 * ref_meta[tag][1]
            else:
                assert meta[tag] == ref_meta[tag], (name, tag, meta[tag], ref_meta[tag])
            assert np.array_equal(got[tag], ref[tag]), (name, tag)
    # the standard FP64 operator through the other 5-point shapes
    for k in (1, 2):
        got, meta = run_child(tmp_path, "std_rb%d" % k, {"BMG_RB_PRESCALE": "0",
                                                         "BMG_TMA_CFG": str(k)})
        assert meta["fp64"] == std_meta["fp64"], k
        assert np.array_equal(got["fp64"], std["fp64"]), k
