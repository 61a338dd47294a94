"""The allocation-free residual check (bmg_residual_norm_noalloc).

Some callers cannot let a library allocate device memory: programs whose
device memory is all served by their own pool, and latency-critical loops
where a cudaMalloc/cudaFree pair may synchronise the whole device.  For them
the library offers one entry point that keeps its reduction scratch in a
static device array.  These tests call it through the C ABI and compare it
with the existing entry points (bmg_op_residual, and the residual bmg_solve
reports), twice in a row, so a stale scratch array would show.  This file is
collected last so that a stop-at-first-failure run has run everything else.
"""
import ctypes

import numpy as np
import pytest

from paper_1803_02481_gb300 import inputs

torch = pytest.importorskip("torch")
import paper_1803_02481_gb300 as bm  # noqa: E402

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_norm_matches_existing_entry_points_twice():
    pr = inputs.block_problem(255, seed=1, block=64, lo=-4, hi=4)
    k = torch.from_numpy(pr["k"]).cuda()
    b = torch.from_numpy(pr["b"]).cuda()
    h = bm.setup(k)
    x, info = h.solve(b, tol=1e-10)
    ny, nx = pr["k"].shape
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    bnorm = np.linalg.norm(pr["b"])
    for call, xx in enumerate((x, 0.5 * x)):        # two calls in a row, different inputs
        rc = bm.lib().bmg_residual_norm_noalloc(_ptr(k), _ptr(xx), _ptr(b), nx, ny, _ptr(norms), stream)
        assert rc == bm.BMG_OK
        got = norms.cpu().numpy()
        r = h.op_residual(h.nlevels - 1, xx.contiguous(), b, torch.zeros_like(b)).cpu().numpy()
        rnorm = np.linalg.norm(r)
        # same tolerance as the solve parity tests: relative residuals agree
        # to 1e-13 (rounding of b - A x near convergence), ||b|| to 1e-13
        assert abs(got[0] - rnorm) / bnorm <= 1e-13
        assert abs(got[1] - bnorm) <= 1e-13 * bnorm
        if call == 0:
            # the residual bmg_solve reported for the same x
            assert abs(got[0] / got[1] - info.rel_resid) <= 1e-13
    h.destroy()


def test_noalloc_allocates_no_device_memory():
    """The point of the entry point: repeated calls leave the device's free
    memory unchanged.  The first call resolves the scratch array's address
    (with lazy module loading that may load the library's device code), so
    it comes before the first reading."""
    pr = inputs.block_problem(127, seed=1, block=16, lo=-2, hi=2)
    k = torch.from_numpy(pr["k"]).cuda()
    b = torch.from_numpy(pr["b"]).cuda()
    x = torch.zeros_like(b)
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    ny, nx = pr["k"].shape
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert bm.lib().bmg_residual_norm_noalloc(_ptr(k), _ptr(x), _ptr(b), nx, ny, _ptr(norms), stream) == bm.BMG_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(50):
        assert bm.lib().bmg_residual_norm_noalloc(_ptr(k), _ptr(x), _ptr(b), nx, ny, _ptr(norms),
                                                  stream) == bm.BMG_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    # with x = 0 the residual is b itself
    got = norms.cpu().numpy()
    bnorm = np.linalg.norm(pr["b"])
    assert abs(got[0] - bnorm) <= 1e-13 * bnorm and abs(got[1] - bnorm) <= 1e-13 * bnorm


def test_noalloc_python_wrapper_checks_shapes():
    """bm.residual_norm_noalloc passes k's sizes to the kernels, so it must
    refuse x, b or norms that are smaller than those sizes imply."""
    pr = inputs.block_problem(63, seed=1, block=16, lo=-2, hi=2)
    k = torch.from_numpy(pr["k"]).cuda()
    b = torch.from_numpy(pr["b"]).cuda()
    x = torch.zeros_like(b)
    norms = bm.residual_norm_noalloc(k, x, b)
    bnorm = np.linalg.norm(pr["b"])
    assert abs(norms[0].item() - bnorm) <= 1e-13 * bnorm
    small = torch.zeros((62, 63), dtype=torch.float64, device="cuda")
    with pytest.raises(TypeError):
        bm.residual_norm_noalloc(k, small, b)
    with pytest.raises(TypeError):
        bm.residual_norm_noalloc(k, x, small)
    with pytest.raises(TypeError):
        bm.residual_norm_noalloc(k, x, b, norms=torch.zeros(1, dtype=torch.float64, device="cuda"))
    with pytest.raises(TypeError):
        bm.residual_norm_noalloc(k.reshape(-1), x, b)


def test_noalloc_rejects_grids_beyond_its_scratch():
    t = torch.zeros((3, 3), dtype=torch.float64, device="cuda")
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    rc = bm.lib().bmg_residual_norm_noalloc(_ptr(t), _ptr(t), _ptr(t), 3, 16385, _ptr(norms), None)
    assert rc == bm.BMG_EINVAL
    assert b"16384" in bm.lib().bmg_last_error()
