"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (FP64):
* coarse stencil entries: |gpu - oracle| <= 1e-12 * max(|a|, C_row), the
  row diagonal as scale because off-diagonals can be tiny under 10^8
  contrast; the finest level is assembled with the same operation order as
  the oracle and must match exactly;
* interpolation weights (in [0, 1]): 1e-12 absolute;
* solves: identical V-cycle counts; final relative residuals within 1e-10 of
  each other (both are below tol = 1e-10) and, tighter, within 1e-13: the
  relative residual of an iterate is evaluated in FP64 with rounding of order
  eps * ||(|A| |x|)|| / ||b||, a few hundred ulp here, and the GPU (FMA)
  and the oracle (no FMA) round differently; iterates within 1e-9 of max|x|.
"""
import functools

import numpy as np
import pytest

from oracle import boxmg_oracle as O
from paper_1803_02481_gb300 import inputs
from tests.parity_helpers import (PROBLEMS, interp_planes, nine_from_five, oracle_hierarchy,
                                  oracle_solve, problem)

torch = pytest.importorskip("torch")
import paper_1803_02481_gb300 as bm  # noqa: E402

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def gpu_setup(name, **opts):
    return bm.setup(dev(problem(name)["k"]), bm.default_options(**opts))


SETUP_CASES = ["poisson255", "blocks255", "blocks511_c2", "lognormal255", "random63",
               "rect127x31", "tiny3"]


def rel_stencil_err(sg, so):
    """max over entries of |gpu - oracle| / max(|a|, C_row)."""
    scale = np.maximum(np.abs(so["C"]), 1e-300)
    return max(float((np.abs(sg[d] - so[d]) / np.maximum(np.abs(so[d]), scale)).max())
               for d in ("C", "W", "S", "SW", "NW"))


def p_err(hg, l, st_fine):
    """max |gpu weight - oracle weight| of P_l, the oracle's P built from
    the given fine stencil."""
    ny, nx = st_fine["C"].shape
    planes, valid = interp_planes(O.interpolation(st_fine), nx, ny)
    pg = hg.level_interp(l)
    return max(float(np.abs(pg[key] - planes[k])[valid[k]].max(initial=0.0))
               for k, key in enumerate(("XW", "XE", "YS", "YN", "CSW", "CSE", "CNW", "CNE")))


@pytest.mark.parametrize("name", SETUP_CASES)
def test_setup_each_step_matches_oracle(name):
    """Each setup step on the GPU's own input: the finest level is assembled
    bit-identically; P_l from A_l and A_{l-1} = P_l^T A_l P_l agree with the
    oracle's operations applied to the GPU's A_l (1e-12 per entry, relative
    to the row diagonal; 1e-12 absolute for weights); the coarsest factor
    with the oracle's Cholesky of the GPU's A_0."""
    ho = oracle_hierarchy(name)
    hg = gpu_setup(name)
    L = ho.nlevels
    assert hg.nlevels == L
    sg = hg.level_stencil(L - 1)
    so = ho.levels[L - 1].st
    for d in ("C", "W", "S"):
        assert np.array_equal(sg[d], so[d]), d
    assert not sg["SW"].any() and not sg["NW"].any()
    for l in range(L - 1, 0, -1):
        st_g = nine_from_five(hg.level_stencil(l))
        assert p_err(hg, l, st_g) <= 1e-12, l
        coarse_o = O.galerkin(st_g, O.interpolation(st_g))
        assert rel_stencil_err(hg.level_stencil(l - 1), coarse_o) <= 1e-12, l
    a0 = O.stencil_to_csr(nine_from_five(hg.level_stencil(0))).toarray()
    lo = O.cholesky(a0)
    assert np.abs(hg.coarse_factor() - lo).max() <= 1e-12 * np.abs(lo).max()
    hg.destroy()


@pytest.mark.parametrize("name", SETUP_CASES)
def test_setup_hierarchy_matches_oracle_end_to_end(name):
    """The whole GPU hierarchy against the oracle's own hierarchy.  Rounding
    differences of one Galerkin product (~1e-15 of the row scale) are
    amplified by cancellation in the coarser products, so level l is allowed
    1e-12 per Galerkin product between it and the finest level."""
    ho = oracle_hierarchy(name)
    hg = gpu_setup(name)
    L = ho.nlevels
    for l in range(L - 1):
        depth = L - 1 - l
        err = rel_stencil_err(hg.level_stencil(l), ho.levels[l].st)
        assert err <= 1e-12 * depth, (l, err)
    for l in range(1, L):
        depth = L - l
        assert p_err(hg, l, ho.levels[l].st) <= 1e-12 * depth, l
    hg.destroy()


@pytest.mark.parametrize("name", ["blocks255", "rect127x31", "wide2047x127"])
def test_single_operations_match_oracle(name):
    ho = oracle_hierarchy(name)
    hg = gpu_setup(name)
    rng = np.random.default_rng(3)
    L = ho.nlevels
    for l in (L - 1, L - 2, 1):
        st = ho.levels[l].st
        ny, nx = st["C"].shape
        x = rng.uniform(-1, 1, (ny, nx))
        b = rng.uniform(-1, 1, (ny, nx))
        scale = np.abs(st["C"]).max()
        # residual
        r_g = hg.op_residual(l, dev(x), dev(b), torch.zeros((ny, nx), dtype=torch.float64, device="cuda"))
        r_o = O.residual(st, x, b)
        assert np.abs(r_g.cpu().numpy() - r_o).max() <= 1e-13 * scale * 4
        # relaxation, forward and reverse, two sweeps
        for rev in (False, True):
            xg = hg.op_relax(l, dev(x), dev(b), nu=2, reverse=rev).cpu().numpy()
            xo = x.copy()
            O.relax(st, xo, b, 2, O.colour_order(st), reverse=rev)
            assert np.abs(xg - xo).max() <= 1e-11 * max(1.0, np.abs(xo).max()), (l, rev)
        if l >= 1:
            p = ho.levels[l].p
            nyc, nxc = ho.levels[l - 1].shape
            bc_g = hg.op_restrict(l, dev(r_o), torch.zeros((nyc, nxc), dtype=torch.float64, device="cuda"))
            bc_o = (p.T @ r_o.ravel()).reshape(nyc, nxc)
            assert np.abs(bc_g.cpu().numpy() - bc_o).max() <= 1e-12 * max(1.0, np.abs(bc_o).max())
            xc = rng.uniform(-1, 1, (nyc, nxc))
            xi_g = hg.op_interp(l, dev(xc), dev(x)).cpu().numpy()
            xi_o = x + (p @ xc.ravel()).reshape(ny, nx)
            assert np.abs(xi_g - xi_o).max() <= 1e-13 * 4
    hg.destroy()


SOLVE_CASES = ["poisson255", "blocks255", "lognormal255", "random63", "rect127x31", "tiny3",
               "wide2047x127"]


@pytest.mark.parametrize("name", SOLVE_CASES)
def test_solve_matches_oracle(name):
    pr = problem(name)
    ro = oracle_solve(name)
    hg = gpu_setup(name)
    x, info = hg.solve(dev(pr["b"]), tol=1e-10)
    xg = x.cpu().numpy()
    assert info.cycles == ro.cycles, (info.cycles, ro.cycles, ro.history[-3:])
    assert info.rel_resid <= 1e-10 and ro.rel_resid <= 1e-10
    assert abs(info.rel_resid - ro.rel_resid) <= 1e-10
    assert abs(info.rel_resid - ro.rel_resid) <= 1e-13
    assert np.abs(xg - ro.x).max() <= 1e-9 * np.abs(ro.x).max()
    # the returned x satisfies the stop test with the oracle's own operator
    st = oracle_hierarchy(name).levels[-1].st
    rel = np.linalg.norm(O.residual(st, xg, pr["b"])) / np.linalg.norm(pr["b"])
    assert rel <= 1.0000001e-10
    hg.destroy()


def test_solve_slow_contrast_case_matches_oracle():
    """511^2, 64-cell blocks, contrast 10^4: several hundred thousand
    unknowns, 8 full tiles and ragged tails on every coarse level."""
    test_solve_matches_oracle("blocks511_c2")


def cluster_sizes(precision=bm.BMG_FP64):
    cmax = bm.max_coarse_ctas(precision)
    return sorted({1, min(2, cmax), cmax})


@pytest.mark.parametrize("name", ["blocks255", "rect127x31"])
def test_every_threshold_gives_identical_iterates(name):
    """The level schedule moves levels between full-grid launches and the
    persistent kernel, run by one block or by a thread-block cluster;
    per-point arithmetic is shared and the points of a colour are
    independent, so results are bit-identical for every threshold and every
    number of blocks.  While the finest level is swept outside the
    persistent kernel the stop test runs inside its next sweep (the same bits
    for every such threshold); with the finest level inside the kernel it is
    the separate norm pass, equal to rounding."""
    pr = problem(name)
    L = oracle_hierarchy(name).nlevels
    ref = None
    for ctas in cluster_sizes():
        for thr in range(1, L + 1):
            hg = gpu_setup(name, coarse_threshold=thr, coarse_ctas=ctas)
            x, info = hg.solve(dev(pr["b"]), tol=1e-10)
            assert info.threshold == thr and info.coarse_ctas == ctas
            xn = x.cpu().numpy()
            if ref is None:
                ref = (xn, info.cycles, info.rel_resid)
            else:
                assert np.array_equal(xn, ref[0]), (ctas, thr)
                assert info.cycles == ref[1]
                if thr < L:
                    assert info.rel_resid == ref[2]
                else:
                    assert abs(info.rel_resid - ref[2]) <= 1e-6 * ref[2] + 2e-15
            hg.destroy()


def test_cluster_coarse_kernel_fp32_and_rc_identical_to_one_block():
    """FP32 refinement and the r/C variant through the cluster kernel: the
    same bits as the one-block kernel at every threshold."""
    name = "lognormal255"
    pr = problem(name)
    L = oracle_hierarchy(name).nlevels
    for prec, kw in ((bm.BMG_FP32_REFINE, {}), (bm.BMG_FP64, dict(interp_residual_term=1))):
        cmax = bm.max_coarse_ctas(prec)
        for thr in (2, L - 2, L):
            out = []
            for ctas in (1, cmax):
                hg = gpu_setup(name, precision=prec, coarse_threshold=thr, coarse_ctas=ctas, **kw)
                x, info = hg.solve(dev(pr["b"]), tol=1e-10)
                hg.destroy()
                out.append((x.cpu().numpy(), info.cycles, info.rel_resid))
            assert np.array_equal(out[0][0], out[1][0]), (prec, thr)
            assert out[0][1:] == out[1][1:]


def test_schedule_options_are_checked():
    k = dev(np.ones((31, 31)))
    cmax = bm.max_coarse_ctas()
    for kw in (dict(coarse_ctas=0), dict(coarse_ctas=17), dict(coarse_ctas=cmax + 1),
               dict(coarse_ctas=2, smoother=bm.BMG_SMOOTH_XLINE), dict(coarse_threshold=0)):
        if kw.get("coarse_ctas") == 2 and cmax < 2:
            continue
        with pytest.raises(bm.BoxMGError) as e:
            bm.setup(k, bm.default_options(**kw))
        assert e.value.code == bm.BMG_EINVAL, kw
    h = bm.setup(k)                     # the model's choice is reported
    _, info = h.solve(dev(np.ones((31, 31))))
    assert 1 <= info.coarse_ctas <= cmax and 1 <= info.threshold <= h.nlevels
    h.destroy()


def test_prescaled_fine_level_identical_in_every_kernel():
    """A fine level wide enough for the TMA sweep runs on the prescaled
    operator; the persistent kernel applies the same prescaled update when
    the threshold hands it the finest level, so the iterates stay
    bit-identical across thresholds; FP32 refinement is never prescaled.
    While the finest level is swept outside the persistent kernel the stop
    test runs inside its next sweep (prescaled evaluation, the same bits for
    every threshold); with the finest level inside the kernel it is the
    separate norm pass, equal to rounding."""
    name = "wide2047x127"
    pr = problem(name)
    L = oracle_hierarchy(name).nlevels
    ref = None
    for thr, ctas in ((1, 1), (L - 1, 1), (L, 1), (L, bm.max_coarse_ctas())):
        hg = gpu_setup(name, coarse_threshold=thr, coarse_ctas=ctas)
        assert hg.level_prescaled(L - 1) and not hg.level_prescaled(L - 2)
        x, info = hg.solve(dev(pr["b"]), tol=1e-10)
        hg.destroy()
        xn = x.cpu().numpy()
        if ref is None:
            ref = (xn, info.cycles, info.rel_resid)
        else:
            assert np.array_equal(xn, ref[0]), (thr, ctas)
            assert info.cycles == ref[1]
            if thr < L:
                assert info.rel_resid == ref[2]
            else:
                assert abs(info.rel_resid - ref[2]) <= 1e-6 * ref[2] + 2e-15
    hf = gpu_setup(name, precision=bm.BMG_FP32_REFINE)
    assert not hf.level_prescaled(L - 1)
    hf.destroy()


def test_interp_residual_term_variant_matches_oracle():
    name = "random63"
    pr = problem(name)
    ho = O.setup(pr["k"], interp_residual_term=True)
    ro = O.solve(ho, pr["b"], tol=1e-10)
    hg = gpu_setup(name, interp_residual_term=1)
    x, info = hg.solve(dev(pr["b"]), tol=1e-10)
    assert info.cycles == ro.cycles
    assert np.abs(x.cpu().numpy() - ro.x).max() <= 1e-9 * np.abs(ro.x).max()
    hg.destroy()


@pytest.mark.parametrize("name", ["poisson255", "lognormal255", "blocks255"])
def test_interp_residual_term_on_the_gpu_is_the_post_smoothing_residual_over_c(name):
    """The property that pins the oracle's r/C term, checked on the GPU's own
    cycle: with nu2 = 0, one cycle's update minus r_pre/C at non-coarse points
    (r_pre the residual after pre-smoothing, C the fine diagonal) is P times
    the coarse correction, i.e. interpolated exactly from its values at the
    coarse points.  Then the same cycle against the oracle's."""
    pr = problem(name)
    ny, nx = pr["k"].shape
    rng = np.random.default_rng(17)
    x0 = rng.uniform(-1, 1, (ny, nx))
    hg = bm.setup(dev(pr["k"]), bm.default_options(nu1=1, nu2=0, interp_residual_term=1, max_cycles=1))
    x1, info = hg.solve(dev(pr["b"]), dev(x0), tol=1e-300, allow_noconv=True)
    assert info.cycles == 1
    x1 = x1.cpu().numpy()
    hg.destroy()
    ho = O.setup(pr["k"], nu1=1, nu2=0, interp_residual_term=True)
    st = ho.levels[-1].st
    x_pre = x0.copy()
    O.relax(st, x_pre, pr["b"], 1, O.colour_order(st))
    r_pre = O.residual(st, x_pre, pr["b"])
    cm = np.zeros((ny, nx), dtype=bool)
    cm[1::2, 1::2] = True
    y = x1 - x_pre - np.where(cm, 0.0, r_pre / st["C"])
    # P from the oracle (the GPU's weights equal it to 1e-12, tested above)
    py = (ho.levels[-1].p @ y[1::2, 1::2].ravel()).reshape(ny, nx)
    scale = np.abs(y).max()
    assert scale > 1e-3
    assert np.abs(y - py).max() <= 1e-11 * scale
    xo = x0.copy()
    O.vcycle(ho, xo, pr["b"])
    assert np.abs(x1 - xo).max() <= 1e-10 * np.abs(xo).max()


@pytest.mark.parametrize("name", ["poisson255", "blocks255", "lognormal255", "wide2047x127"])
def test_fp32_refinement_reaches_fp64_tolerance(name):
    pr = problem(name)
    ro = oracle_solve(name)
    hg = gpu_setup(name, precision=bm.BMG_FP32_REFINE)
    x, info = hg.solve(dev(pr["b"]), tol=1e-10)
    xg = x.cpu().numpy()
    st = oracle_hierarchy(name).levels[-1].st
    rel = np.linalg.norm(O.residual(st, xg, pr["b"])) / np.linalg.norm(pr["b"])
    assert rel <= 1.0000001e-10 and info.rel_resid <= 1e-10
    # error against the FP64 oracle solution, bounded by what 1e-10 allows
    err = np.abs(xg - ro.x).max() / np.abs(ro.x).max()
    assert err <= 1e-7
    # FP32 coarse hierarchy is the FP32 Galerkin product of the FP32 fine operator
    so = O.galerkin({k: v.astype(np.float32).astype(np.float64) for k, v in st.items()},
                    O.interpolation({k: v.astype(np.float32).astype(np.float64) for k, v in st.items()}))
    sg = hg.level_stencil(hg.nlevels - 2)
    assert np.abs(sg["C"] - so["C"]).max() <= 1e-5 * np.abs(so["C"]).max()
    hg.destroy()


def test_assembly_backward_matches_oracle():
    rng = np.random.default_rng(31)
    n = 127
    theta = rng.normal(0, 1, (n, n))
    k = np.exp(theta)
    u = rng.uniform(-1, 1, (n, n))
    lam = rng.uniform(-1, 1, (n, n))
    hg = bm.setup(dev(k))
    g = hg.assemble_backward(dev(u), dev(lam), torch.zeros((n, n), dtype=torch.float64, device="cuda"))
    go = O.assembly_vjp(k, u, lam)
    assert np.abs(g.cpu().numpy() - go).max() <= 1e-13 * np.abs(go).max()
    hg.destroy()


def test_zero_rhs_and_error_codes():
    k = dev(np.ones((31, 31)))
    hg = bm.setup(k)
    x, info = hg.solve(dev(np.zeros((31, 31))), x=dev(np.ones((31, 31))))
    assert info.cycles == 0 and not x.any()
    hg.destroy()
    bad = np.ones((31, 31))
    bad[4, 5] = np.nan
    with pytest.raises(bm.BoxMGError) as e:
        bm.setup(dev(bad))
    assert e.value.code == bm.BMG_EINVAL
    bad[4, 5] = -1.0
    with pytest.raises(bm.BoxMGError) as e:
        bm.setup(dev(bad))
    assert e.value.code == bm.BMG_EINVAL
    with pytest.raises(bm.BoxMGError) as e:          # a side needs at least 2 cells
        bm.setup(dev(np.ones((1, 31))))
    assert e.value.code == bm.BMG_EINVAL
    with pytest.raises(bm.BoxMGError) as e:          # coarsest level above 1024 unknowns
        bm.setup(dev(np.ones((3, 400))))
    assert e.value.code == bm.BMG_EINVAL
    # the cycle cap returns ENOCONV with the last iterate
    pr = problem("blocks255")
    hg = bm.setup(dev(pr["k"]), bm.default_options(max_cycles=3))
    with pytest.raises(bm.BoxMGError) as e:
        hg.solve(dev(pr["b"]), tol=1e-10)
    assert e.value.code == bm.BMG_ENOCONV
    x, info = hg.solve(dev(pr["b"]), tol=1e-10, allow_noconv=True)
    assert info.cycles == 3 and info.rel_resid > 1e-10
    ro = O.setup(pr["k"])
    xo = np.zeros_like(pr["b"])
    for _ in range(3):
        O.vcycle(ro, xo, pr["b"])
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-12 * np.abs(xo).max()
    hg.destroy()


def test_solve_host_end_to_end():
    pr = problem("poisson255")
    ro = oracle_solve("poisson255")
    x = np.zeros_like(pr["b"])
    info = bm.solve_host(np.ascontiguousarray(pr["k"]), np.ascontiguousarray(pr["b"]), x)
    assert info.cycles == ro.cycles
    assert np.abs(x - ro.x).max() <= 1e-9 * np.abs(ro.x).max()


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine", "pcg"])
def test_graph_and_stream_paths_agree(precision):
    """The solve loop recorded as one CUDA graph (default) and launched op by
    op on the stream (used while kernel classes are being timed) run the
    same kernels in the same order: identical results."""
    pr = problem("blocks255")
    if precision == "pcg":
        hg = gpu_setup("blocks255", nu1=1, nu2=1, solver=bm.BMG_SOLVER_PCG)
    else:
        prec = bm.BMG_FP64 if precision == "fp64" else bm.BMG_FP32_REFINE
        hg = gpu_setup("blocks255", precision=prec)
    x1, i1 = hg.solve(dev(pr["b"]), tol=1e-10)
    bm.profile_set(("norm",))
    try:
        x2, i2 = hg.solve(dev(pr["b"]), tol=1e-10)
    finally:
        bm.profile_set(())
    assert i1.cycles == i2.cycles and i1.rel_resid == i2.rel_resid
    assert torch.equal(x1, x2)
    hg.destroy()


# ---------------------------------------------------------------------------
# Conjugate gradients preconditioned by one symmetric V(1,1) cycle
# ---------------------------------------------------------------------------

PCG_CASES = ["poisson255", "blocks255", "blocks511_c2", "lognormal255", "random63", "rect127x31",
             "wide2047x127", "tiny3"]


@functools.lru_cache(maxsize=None)
def oracle_pcg(name, tol=1e-10):
    pr = problem(name)
    return O.pcg(O.setup(pr["k"], nu1=1, nu2=1), pr["b"], tol=tol, max_iter=400)


@pytest.mark.parametrize("name", PCG_CASES)
def test_pcg_matches_oracle(name):
    pr = problem(name)
    ro = oracle_pcg(name)
    hg = gpu_setup(name, nu1=1, nu2=1, solver=bm.BMG_SOLVER_PCG, max_cycles=400)
    x, info = hg.solve(dev(pr["b"]), tol=1e-10)
    xg = x.cpu().numpy()
    hist = hg.residual_history()
    hg.destroy()
    assert ro.converged and info.cycles == ro.cycles, (info.cycles, ro.cycles)
    # the recurrences agree to rounding: dot products summed in another order
    h_o = np.array(ro.history)
    assert np.all(np.abs(hist - h_o) <= 1e-7 * h_o + 1e-14)
    assert info.rel_resid <= 1e-10
    assert np.abs(xg - ro.x).max() <= 1e-9 * np.abs(ro.x).max()
    # the true residual of the returned x (the stop test uses the updated one)
    st = oracle_hierarchy(name).levels[-1].st
    rel = np.linalg.norm(O.residual(st, xg, pr["b"])) / np.linalg.norm(pr["b"])
    assert rel <= 2e-10


def test_pcg_with_fp32_cycles_reaches_fp64_tolerance():
    """PCG whose V(1,1) preconditioner runs on the FP32 hierarchy (r / ||r||
    cast down, ||r|| e cast back): the FP64 recurrences reach 1e-10 against
    the oracle's operator, within a few iterations of the FP64-cycle PCG."""
    for name in ("blocks255", "rect127x31", "lognormal255"):
        pr = problem(name)
        ro = oracle_pcg(name)
        hg = gpu_setup(name, nu1=1, nu2=1, solver=bm.BMG_SOLVER_PCG, max_cycles=400,
                       precision=bm.BMG_FP32_REFINE)
        x, info = hg.solve(dev(pr["b"]), tol=1e-10)
        hg.destroy()
        xg = x.cpu().numpy()
        st = oracle_hierarchy(name).levels[-1].st
        rel = np.linalg.norm(O.residual(st, xg, pr["b"])) / np.linalg.norm(pr["b"])
        assert info.rel_resid <= 1e-10 and rel <= 2e-10, (name, rel)
        assert np.abs(xg - ro.x).max() <= 1e-7 * np.abs(ro.x).max()
        assert info.cycles <= ro.cycles + 3, (name, info.cycles, ro.cycles)


def test_pcg_needs_a_symmetric_cycle():
    k = dev(problem("blocks255")["k"])
    for opts in (dict(solver=bm.BMG_SOLVER_PCG),                       # V(2,1)
                 dict(solver=bm.BMG_SOLVER_PCG, nu1=1, nu2=1, interp_residual_term=1)):
        with pytest.raises(bm.BoxMGError) as e:
            bm.setup(k, bm.default_options(**opts))
        assert e.value.code == bm.BMG_EINVAL


# ---------------------------------------------------------------------------
# The paper's workload: D = diag(k/r, k r) on stretched cells (Section 5)
# ---------------------------------------------------------------------------

ANISO_CASES = {
    # nx x ny cells of the unit square (cell aspect nx / ny), r = 16
    "paper1023x63": lambda: {"k": np.ones((63, 1023)),
                             "b": np.random.default_rng(41).uniform(-1, 1, (63, 1023)),
                             "r": 16.0, "aspect": 1023 / 63},
    # the same with a block field k (10^[-1, 1], 8-cell blocks) and r = 4
    "blocks511x31": lambda: dict(inputs.block_problem(seed=42, block=8, lo=-1, hi=1, nx=511, ny=31),
                                 r=4.0, aspect=511 / 31),
    # uncompensated: isotropic k on stretched cells, V(2,1) slow but correct
    "stretched255x63": lambda: {"k": np.ones((63, 255)),
                                "b": np.random.default_rng(43).uniform(-1, 1, (63, 255)),
                                "r": 1.0, "aspect": 255 / 63},
}


@functools.lru_cache(maxsize=None)
def aniso_case(name):
    return ANISO_CASES[name]()


@pytest.mark.parametrize("name", list(ANISO_CASES))
def test_anisotropic_stretched_workload_matches_oracle(name):
    pr = aniso_case(name)
    ho = O.setup(pr["k"], r=pr["r"], aspect=pr["aspect"])
    hg = bm.setup(dev(pr["k"]), bm.default_options(aniso_r=pr["r"], cell_aspect=pr["aspect"],
                                                   max_cycles=400))
    L = ho.nlevels
    sg = hg.level_stencil(L - 1)
    so = ho.levels[L - 1].st
    for d in ("C", "W", "S"):
        assert np.array_equal(sg[d], so[d]), d
    for l in range(L - 1):
        assert rel_stencil_err(hg.level_stencil(l), ho.levels[l].st) <= 1e-12 * (L - 1 - l), l
    ro = O.solve(ho, pr["b"], tol=1e-10, max_cycles=400)
    x, info = hg.solve(dev(pr["b"]), tol=1e-10)
    hg.destroy()
    assert ro.converged and info.cycles == ro.cycles, (info.cycles, ro.cycles)
    assert abs(info.rel_resid - ro.rel_resid) <= 1e-13
    assert np.abs(x.cpu().numpy() - ro.x).max() <= 1e-9 * np.abs(ro.x).max()


def test_anisotropic_options_are_checked():
    k = dev(np.ones((31, 63)))
    for opts in (dict(aniso_r=0.0), dict(cell_aspect=-1.0), dict(aniso_r=float("inf"))):
        with pytest.raises(bm.BoxMGError) as e:
            bm.setup(k, bm.default_options(**opts))
        assert e.value.code == bm.BMG_EINVAL
    h = bm.setup(k, bm.default_options(aniso_r=4.0))
    u = dev(np.ones((31, 63)))
    with pytest.raises(bm.BoxMGError):
        h.assemble_backward(u, u, torch.zeros_like(u))
    h.destroy()


def test_binding_rejects_tensors_of_the_wrong_shape():
    """The kernels index b, x and the level arrays by the hierarchy's sizes,
    so the binding refuses any tensor whose shape differs from them."""
    k = dev(np.ones((31, 63)))
    h = bm.setup(k)
    good = torch.zeros((31, 63), dtype=torch.float64, device="cuda")
    small = torch.zeros((30, 63), dtype=torch.float64, device="cuda")
    for args in ((small, None), (good, small), (small.t().contiguous(), None)):
        with pytest.raises(TypeError):
            h.solve(args[0], args[1])
    L = h.nlevels
    nxc, nyc = h.level_shape(L - 2)
    coarse = torch.zeros((nyc, nxc), dtype=torch.float64, device="cuda")
    with pytest.raises(TypeError):
        h.op_relax(L - 1, small, good)
    with pytest.raises(TypeError):
        h.op_residual(L - 1, good, good, small)
    with pytest.raises(TypeError):
        h.op_restrict(L - 1, good, small)
    with pytest.raises(TypeError):
        h.op_interp(L - 1, good, good)      # xc must have the coarse shape
    with pytest.raises(TypeError):
        h.assemble_backward(good, good, small)
    h.op_restrict(L - 1, good, coarse)      # the right shapes still pass
    x, info = h.solve(good.clone().fill_(1.0))
    assert info.rel_resid <= 1e-10
    h.destroy()


# ---------------------------------------------------------------------------
# General grid sides (other than 2^m - 1)
# ---------------------------------------------------------------------------

GENERAL_CASES = {
    "even100x60": lambda: dict(inputs.block_problem(seed=51, block=8, lo=-2, hi=2, nx=100, ny=60),
                               r=1.0, aspect=1.0),
    "mixed131x46": lambda: dict(inputs.block_problem(seed=52, block=16, lo=-3, hi=3, nx=131, ny=46),
                                r=1.0, aspect=1.0),
    "pow2_256x256": lambda: dict(inputs.block_problem(seed=53, block=32, lo=-2, hi=2, nx=256, ny=256),
                                 r=1.0, aspect=1.0),
    # the paper's local problem: 568 x 71 cells (8:1) with compensating r = 8
    "paper568x71": lambda: {"k": np.ones((71, 568)),
                            "b": np.random.default_rng(54).uniform(-1, 1, (71, 568)),
                            "r": 8.0, "aspect": 8.0},
    # wide enough for the TMA-staged sweeps on the finest and first coarse level
    "even2100x40": lambda: dict(inputs.block_problem(seed=55, block=32, lo=-1, hi=1, nx=2100, ny=40),
                                r=1.0, aspect=1.0),
    "tiny2x5": lambda: {"k": np.array([[1.0, 2.0], [3.0, 4.0], [5.0, 6.0], [7.0, 8.0], [9.0, 1.0]]),
                        "b": np.arange(10.0).reshape(5, 2) - 4.5, "r": 1.0, "aspect": 1.0},
}


@functools.lru_cache(maxsize=None)
def general_case(name):
    return GENERAL_CASES[name]()


@pytest.mark.parametrize("name", list(GENERAL_CASES))
def test_general_sides_match_oracle(name):
    pr = general_case(name)
    ho = O.setup(pr["k"], r=pr["r"], aspect=pr["aspect"])
    hg = bm.setup(dev(pr["k"]), bm.default_options(aniso_r=pr["r"], cell_aspect=pr["aspect"],
                                                   max_cycles=400))
    L = ho.nlevels
    assert hg.nlevels == L
    for l in range(L):
        assert hg.level_shape(l) == ho.levels[l].shape[::-1], l
    sg = hg.level_stencil(L - 1)
    so = ho.levels[L - 1].st
    for d in ("C", "W", "S"):
        assert np.array_equal(sg[d], so[d]), d
    # each setup step on the GPU's own input
    for l in range(L - 1, 0, -1):
        st_g = nine_from_five(hg.level_stencil(l))
        assert p_err(hg, l, st_g) <= 1e-12, l
        coarse_o = O.galerkin(st_g, O.interpolation(st_g))
        assert rel_stencil_err(hg.level_stencil(l - 1), coarse_o) <= 1e-12, l
    ro = O.solve(ho, pr["b"], tol=1e-10, max_cycles=400)
    x, info = hg.solve(dev(pr["b"]), tol=1e-10)
    hg.destroy()
    assert ro.converged and info.cycles == ro.cycles, (info.cycles, ro.cycles)
    assert abs(info.rel_resid - ro.rel_resid) <= 1e-13
    assert np.abs(x.cpu().numpy() - ro.x).max() <= 1e-9 * np.abs(ro.x).max()


# ---------------------------------------------------------------------------
# Neumann and Robin walls
# ---------------------------------------------------------------------------

BC_CASES = {
    "blocks127x63_nnd_robin": (lambda: inputs.block_problem(seed=71, block=8, lo=-2, hi=2, nx=127, ny=63),
                               (0.0, 0.0, None, 0.5)),
    "even100x60_one_dirichlet": (lambda: inputs.block_problem(seed=72, block=8, lo=-1, hi=1, nx=100,
                                                              ny=60),
                                 (None, 0.0, 0.0, 0.0)),
    "lognormal255_robin": (lambda: problem("lognormal255"), (0.1, 2.0, 0.0, None)),
}


@pytest.mark.parametrize("name", list(BC_CASES))
def test_neumann_robin_walls_match_oracle(name):
    make, bc = BC_CASES[name]
    pr = make()
    ho = O.setup(pr["k"], bc=bc)
    hg = bm.setup(dev(pr["k"]), bm.default_options(bc_beta=bc, max_cycles=400))
    L = ho.nlevels
    sg = hg.level_stencil(L - 1)
    so = ho.levels[L - 1].st
    for d in ("C", "W", "S"):
        assert np.array_equal(sg[d], so[d]), d
    for l in range(L - 1):
        assert rel_stencil_err(hg.level_stencil(l), ho.levels[l].st) <= 1e-12 * (L - 1 - l), l
    ro = O.solve(ho, pr["b"], tol=1e-10, max_cycles=400)
    x, info = hg.solve(dev(pr["b"]), tol=1e-10)
    hg.destroy()
    assert ro.converged and info.cycles == ro.cycles, (info.cycles, ro.cycles)
    assert abs(info.rel_resid - ro.rel_resid) <= 1e-13
    assert np.abs(x.cpu().numpy() - ro.x).max() <= 1e-9 * np.abs(ro.x).max()


def test_all_neumann_walls_are_rejected():
    with pytest.raises(bm.BoxMGError) as e:
        bm.setup(dev(np.ones((31, 31))), bm.default_options(bc_beta=(0.0, 0.0, 0.0, 0.0)))
    assert e.value.code == bm.BMG_EINVAL


# ---------------------------------------------------------------------------
# Zebra line Gauss-Seidel smoothers (x-lines, y-lines, alternating)
# ---------------------------------------------------------------------------

SMOOTHER_CODES = {"x": bm.BMG_SMOOTH_XLINE, "y": bm.BMG_SMOOTH_YLINE, "xy": bm.BMG_SMOOTH_ALTLINE}

LINE_RELAX_CASES = {
    # 2^m - 1 sides: 255-point lines, 15 full blocks and a ragged 16th
    "blocks255": lambda: dict(problem("blocks255"), r=1.0, aspect=1.0),
    # sides that are multiples of 16 (a separator ends every line) down to 16
    "pow2_256x256": lambda: dict(general_case("pow2_256x256")),
    # even, ragged sides on stretched anisotropic cells
    "even100x60_r4": lambda: dict(inputs.block_problem(seed=81, block=8, lo=-2, hi=2, nx=100, ny=60),
                                  r=4.0, aspect=0.5),
}


@pytest.mark.parametrize("smoother", list(SMOOTHER_CODES))
@pytest.mark.parametrize("name", list(LINE_RELAX_CASES))
def test_line_relaxation_matches_oracle(name, smoother):
    """Two line sweeps forward and two reversed, on the 5-point finest level
    and on 9-point levels with and without separators, against the oracle's
    banded solves.  Each line is solved exactly by both sides (different
    elimination orders), so the iterates agree to rounding: 1e-11 of max|x|."""
    pr = LINE_RELAX_CASES[name]()
    ho = O.setup(pr["k"], r=pr["r"], aspect=pr["aspect"], smoother=smoother)
    hg = bm.setup(dev(pr["k"]), bm.default_options(aniso_r=pr["r"], cell_aspect=pr["aspect"],
                                                   smoother=SMOOTHER_CODES[smoother]))
    rng = np.random.default_rng(82)
    L = ho.nlevels
    for l in sorted({L - 1, L - 2, L - 3, 1}):
        st = nine_from_five(hg.level_stencil(l)) if l < L - 1 else ho.levels[l].st
        ny, nx = st["C"].shape
        x = rng.uniform(-1, 1, (ny, nx))
        b = rng.uniform(-1, 1, (ny, nx))
        for rev in (False, True):
            xg = hg.op_relax(l, dev(x), dev(b), nu=2, reverse=rev).cpu().numpy()
            xo = x.copy()
            O.relax_lines(st, xo, b, 2, smoother, reverse=rev)
            assert np.abs(xg - xo).max() <= 1e-11 * max(1.0, np.abs(xo).max()), (l, rev)
    hg.destroy()


LINE_SOLVE_CASES = {
    # D = diag(1/r, r) on square cells: r = 0.01 couples x 10^4 times more
    # strongly than y, r = 100 the reverse; point smoothing stalls on both
    "strong_x127": (lambda: {"k": np.ones((127, 127)),
                             "b": np.random.default_rng(83).uniform(-1, 1, (127, 127)),
                             "r": 0.01, "aspect": 1.0}, "x"),
    "strong_y127_alt": (lambda: {"k": np.ones((127, 127)),
                                 "b": np.random.default_rng(84).uniform(-1, 1, (127, 127)),
                                 "r": 100.0, "aspect": 1.0}, "xy"),
    "strong_y127": (lambda: {"k": np.ones((127, 127)),
                             "b": np.random.default_rng(84).uniform(-1, 1, (127, 127)),
                             "r": 100.0, "aspect": 1.0}, "y"),
    # a heterogeneous block field with anisotropy, alternating lines
    "blocks255_r8_alt": (lambda: dict(problem("blocks255"), r=8.0, aspect=1.0), "xy"),
    # the paper's workload (compensated anisotropy on 16:1 cells), long lines
    "paper1023x63_alt": (lambda: dict(aniso_case("paper1023x63")), "xy"),
    # general sides, lines ending on separators
    "pow2_256_alt": (lambda: dict(general_case("pow2_256x256")), "xy"),
    # Neumann and Robin walls on even sides, stretched anisotropic cells
    "robin100x60_alt": (lambda: dict(inputs.block_problem(seed=85, block=8, lo=-1, hi=1, nx=100, ny=60),
                                     r=0.2, aspect=2.0, bc=(0.0, 2.0, None, 0.5)), "xy"),
    # the r/C interpolation variant with x-lines
    "rc_blocks127_x": (lambda: dict(inputs.block_problem(seed=86, block=8, lo=-2, hi=2, nx=127, ny=127),
                                    r=0.05, aspect=1.0, rc=True), "x"),
}


@pytest.mark.parametrize("name", list(LINE_SOLVE_CASES))
def test_line_smoothed_solve_matches_oracle(name):
    """Identical cycle counts and iterates within 1e-9 of max|x|.  The final
    relative residuals differ by at most ||A (x_gpu - x_oracle)|| / ||b||
    (triangle inequality) plus the rounding of their evaluation, and by at
    most 1e-11: unlike the point smoother, the two sides eliminate each
    line in a different order (blocks and separators against a banded LU),
    so the iterates carry rounding differences of order eps times the line
    systems' condition, which a 10^4-contrast field amplifies in the
    residual of a slowly converging solve (a CPU run of the oracle with the
    block/separator elimination moves the final residual of blocks255 with
    r = 8 by 5e-13)."""
    make, smoother = LINE_SOLVE_CASES[name]
    pr = make()
    bc = pr.get("bc")
    rc = bool(pr.get("rc", False))
    ho = O.setup(pr["k"], r=pr["r"], aspect=pr["aspect"], smoother=smoother, bc=bc,
                 interp_residual_term=rc)
    extra = {} if bc is None else {"bc_beta": bc}
    hg = bm.setup(dev(pr["k"]), bm.default_options(aniso_r=pr["r"], cell_aspect=pr["aspect"],
                                                   smoother=SMOOTHER_CODES[smoother],
                                                   interp_residual_term=int(rc), max_cycles=200,
                                                   **extra))
    ro = O.solve(ho, pr["b"], tol=1e-10, max_cycles=200)
    x, info = hg.solve(dev(pr["b"]), tol=1e-10)
    hg.destroy()
    xg = x.cpu().numpy()
    assert ro.converged and info.cycles == ro.cycles, (info.cycles, ro.cycles)
    assert info.rel_resid <= 1e-10
    st = ho.levels[-1].st
    dres = np.linalg.norm(O.apply(st, xg - ro.x)) / np.linalg.norm(pr["b"])
    assert abs(info.rel_resid - ro.rel_resid) <= dres + 1e-13
    assert abs(info.rel_resid - ro.rel_resid) <= 1e-11
    assert np.abs(xg - ro.x).max() <= 1e-9 * np.abs(ro.x).max()


def test_line_smoothing_restores_convergence_on_the_gpu():
    """Strong x coupling on square cells: point smoothing does not reach
    1e-10 in 100 cycles, x-line smoothing needs a handful."""
    pr = LINE_SOLVE_CASES["strong_x127"][0]()
    hp = bm.setup(dev(pr["k"]), bm.default_options(aniso_r=pr["r"], max_cycles=100))
    with pytest.raises(bm.BoxMGError) as e:
        hp.solve(dev(pr["b"]), tol=1e-10)
    assert e.value.code == bm.BMG_ENOCONV
    hp.destroy()
    hl = bm.setup(dev(pr["k"]), bm.default_options(aniso_r=pr["r"], smoother=bm.BMG_SMOOTH_XLINE))
    _, info = hl.solve(dev(pr["b"]), tol=1e-10)
    hl.destroy()
    assert info.cycles <= 8


@pytest.mark.parametrize("name", ["blocks255_r8_alt", "paper1023x63_alt"])
def test_line_smoother_every_threshold_gives_identical_iterates(name):
    """The persistent coarse kernel smooths its levels with the same per-line
    arithmetic as the full-grid kernels: bit-identical for every threshold."""
    make, smoother = LINE_SOLVE_CASES[name]
    pr = make()
    ref = None
    hg0 = bm.setup(dev(pr["k"]), bm.default_options(aniso_r=pr["r"], cell_aspect=pr["aspect"],
                                                    smoother=SMOOTHER_CODES[smoother]))
    L = hg0.nlevels
    hg0.destroy()
    for thr in range(1, L + 1):
        hg = bm.setup(dev(pr["k"]), bm.default_options(aniso_r=pr["r"], cell_aspect=pr["aspect"],
                                                       smoother=SMOOTHER_CODES[smoother],
                                                       coarse_threshold=thr))
        x, info = hg.solve(dev(pr["b"]), tol=1e-10)
        hg.destroy()
        assert info.threshold == thr
        xn = x.cpu().numpy()
        if ref is None:
            ref = (xn, info.cycles, info.rel_resid)
        else:
            assert np.array_equal(xn, ref[0]), thr
            assert info.cycles == ref[1] and info.rel_resid == ref[2]


def test_line_smoothed_pcg_and_fp32_refinement():
    """PCG with the symmetric alternating-line V(1,1) cycle matches the
    oracle's PCG; FP32 refinement with line smoothing reaches the FP64
    tolerance."""
    pr = dict(problem("blocks255"), r=8.0, aspect=1.0)
    ho = O.setup(pr["k"], nu1=1, nu2=1, r=8.0, smoother="xy")
    ro = O.pcg(ho, pr["b"], tol=1e-10)
    hg = bm.setup(dev(pr["k"]), bm.default_options(nu1=1, nu2=1, aniso_r=8.0,
                                                   smoother=bm.BMG_SMOOTH_ALTLINE,
                                                   solver=bm.BMG_SOLVER_PCG))
    x, info = hg.solve(dev(pr["b"]), tol=1e-10)
    hg.destroy()
    assert ro.converged and info.cycles == ro.cycles, (info.cycles, ro.cycles)
    assert np.abs(x.cpu().numpy() - ro.x).max() <= 1e-9 * np.abs(ro.x).max()
    hf = bm.setup(dev(pr["k"]), bm.default_options(aniso_r=8.0, smoother=bm.BMG_SMOOTH_ALTLINE,
                                                   precision=bm.BMG_FP32_REFINE))
    xf, infof = hf.solve(dev(pr["b"]), tol=1e-10)
    hf.destroy()
    st = O.assemble_fv5(pr["k"], r=8.0)
    rel = np.linalg.norm(O.residual(st, xf.cpu().numpy(), pr["b"])) / np.linalg.norm(pr["b"])
    assert infof.rel_resid <= 1e-10 and rel <= 1.0000001e-10


def test_smoother_option_is_checked():
    k = dev(np.ones((31, 31)))
    for bad in (-1, 4):
        with pytest.raises(bm.BoxMGError) as e:
            bm.setup(k, bm.default_options(smoother=bad))
        assert e.value.code == bm.BMG_EINVAL
    with pytest.raises(bm.BoxMGError) as e:
        bm.Batch([dev(np.ones((31, 31)))], bm.default_options(smoother=bm.BMG_SMOOTH_ALTLINE))
    assert e.value.code == bm.BMG_EINVAL


@pytest.mark.parametrize("name", ["wide2047x127", "blocks255"])
@pytest.mark.parametrize("stream_launched,nu", [(False, (2, 1)), (True, (2, 1)), (False, (1, 1)),
                                                (True, (3, 2)), (False, (0, 1)), (False, (1, 0))])
def test_stop_test_fused_into_the_next_fine_sweep(monkeypatch, name, stream_launched, nu):
    """On a prescaled finest level (nx >= 1024: the TMA sweep) and on a
    narrower one (the small tiled sweep) the residual after a cycle is
    summed inside the next cycle's first fine sweep (after the reverse-order
    post-smoothing sweep one colour satisfies its equation exactly), and that
    sweep's output is dropped when the loop stops.  The iterate must be the
    same bits as with the separate norm pass, cycle count and residual
    history equal to rounding, and the reported residual that of the
    oracle's operator on the returned iterate.  Cycles V(nu1, nu2) with
    nu1 = 1 (the sweep with the residual is the only pre-sweep), more sweeps,
    and nu1 or nu2 = 0 (no fusion: the separate pass)."""
    pr = problem(name)
    b = dev(pr["b"])
    fused = nu[0] >= 1 and nu[1] >= 1
    out = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("BMG_FUSED_NORM", mode)
        for cap, tol in ((5, 1e-300), (400, 1e-10)):
            hg = gpu_setup(name, max_cycles=cap, nu1=nu[0], nu2=nu[1])
            if stream_launched:
                bm.profile_set(("norm", "fine_smooth"))
            try:
                x, info = hg.solve(b, tol=tol, allow_noconv=True)
                if stream_launched:
                    # fused: the prologue's sweep and nu1 - 1 + nu2 sweeps per
                    # cycle are plain; the norm class holds the fused sweeps
                    # (one per cycle) and the passes for ||b|| and r(x0)
                    c, per = info.cycles, nu[0] + nu[1]
                    want = 1 + (per - 1) * c if mode == "1" and fused else per * c
                    assert bm.profile_read("fine_smooth")[0] == want
                    assert bm.profile_read("norm")[0] == c + 2
            finally:
                bm.profile_set(())
            out[mode, cap] = (x, info, hg.residual_history())
            hg.destroy()
    st = oracle_hierarchy(name).levels[-1].st
    st_abs = dict(st)
    for d in O.DIRS:
        st_abs[d] = -st[d]                       # |A| |x| = C |x| + sum_X a_X |x_X|
    for cap in (5, 400):
        (x0, i0, h0), (x1, i1, h1) = out["0", cap], out["1", cap]
        assert i0.cycles == i1.cycles and len(h0) == len(h1) == i1.cycles + 1
        assert torch.equal(x0, x1)
        # two evaluations of ||b - A x|| / ||b|| of the same iterate differ by
        # rounding: a few eps ||A| |x|| / ||b|| (x: the final iterate)
        xn = x1.cpu().numpy()
        floor = np.finfo(np.float64).eps * np.linalg.norm(O.apply(st_abs, np.abs(xn))) / np.linalg.norm(pr["b"])
        assert np.all(np.abs(h1 - h0) <= 1e-6 * h0 + 10 * floor), (np.abs(h1 - h0).max(), floor)
        rel = np.linalg.norm(O.residual(st, xn, pr["b"])) / np.linalg.norm(pr["b"])
        assert abs(i1.rel_resid - rel) <= 1e-6 * rel + 10 * floor, (i1.rel_resid, rel, floor)
    assert out["1", 5][1].cycles == 5
    assert out["1", 400][1].rel_resid <= 1e-10 or nu == (1, 0)
