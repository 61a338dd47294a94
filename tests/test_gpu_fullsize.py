"""GPU parity at the benchmark sizes, in the configuration bench.py times.

The oracle cannot run these problems whole, so the tests check
* sampled outputs: interpolation weights, Galerkin entries and one
  Gauss-Seidel sweep depend only on a small neighbourhood, so the oracle
  applied to a window cut from the GPU's own full-size level gives the exact
  result at the window's central points (those at least a dependency radius
  from the window's edge);
* a property that holds at any size: the returned iterate satisfies the stop
  test against the oracle's own assembly of the same problem.

Tolerances as in test_gpu_parity.py: weights 1e-12 absolute, coarse entries
1e-12 of the row diagonal, one sweep 1e-12 of max|x| (the same Gauss-Seidel
step in a different rounding order).  Residuals: the oracle's FP64
evaluation of ||b - A x|| / ||b|| and the GPU's (with fused multiply-adds)
are two roundings of the same quantity, apart by about eps ||(|A| |x|)|| /
||b||, which on these grids reaches ~1e-10 (the C2 field's residual floor is
6e-10): the oracle's value may exceed tol, and differ from the reported
one, by at most 0.2 tol.  For the C2 solve the residual is also evaluated in
extended precision (long double), which decides whether the iterate meets
the tolerance.
"""
import numpy as np
import pytest

from oracle import boxmg_oracle as O
from paper_1803_02481_gb300 import inputs
from tests.parity_helpers import interp_planes, nine_from_five

torch = pytest.importorskip("torch")
import paper_1803_02481_gb300 as bm  # noqa: E402

pytestmark = pytest.mark.gpu

C2_SIDE = 4095


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.fixture(scope="module")
def c2():
    """The C2 problem (4095^2 block field, 64-cell blocks, 10^[-4, 4]) and
    its GPU hierarchy in the benchmark's options."""
    pr = inputs.block_problem(C2_SIDE, seed=1, block=64, lo=-4, hi=4)
    h = bm.setup(dev(pr["k"]), bm.default_options(max_cycles=4000))
    yield pr, h
    h.destroy()


def crop(st, s, t, nw):
    """Window of nw x nw fine points starting at 1-based (s, t)."""
    return {d: np.ascontiguousarray(a[t - 1:t - 1 + nw, s - 1:s - 1 + nw]) for d, a in st.items()}


# window origins (1-based, odd) spread over the grid, away from and at walls
WINDOWS = [(1, 1), (1001, 2047), (2049, 65), (4063, 4063), (129, 3969), (3201, 1537)]
NW = 33                      # window side (odd): 16 coarse points per side


def test_c2_setup_sampled_against_oracle_windows(c2):
    """P_L and A_{L-1} = P^T A P of the finest level, and the next coarse
    step, on windows of the full-size hierarchy."""
    pr, h = c2
    L = h.nlevels
    fine = {d: np.asarray(v) for d, v in h.level_stencil(L - 1).items()}
    st_f = nine_from_five(fine)
    # the assembled finest level is the oracle's assembly bit for bit
    st_o = O.assemble_fv5(pr["k"])
    for d in ("C", "W", "S"):
        assert np.array_equal(st_f[d], st_o[d]), d
    del st_o
    for lvl, st_full in ((L - 1, st_f), (L - 2, nine_from_five(h.level_stencil(L - 2)))):
        pg = h.level_interp(lvl)
        coarse = nine_from_five(h.level_stencil(lvl - 1))
        ny, nx = st_full["C"].shape
        for (s, t) in WINDOWS:
            s, t = min(s, nx - NW + 1) | 1, min(t, ny - NW + 1) | 1
            st_w = crop(st_full, s, t, NW)
            p_w = O.interpolation(st_w)
            planes, valid = interp_planes(p_w, NW, NW)
            ncw = NW // 2
            I0, J0 = (s - 1) // 2, (t - 1) // 2
            keys = ("XW", "XE", "YS", "YN", "CSW", "CSE", "CNW", "CNE")
            # coarse points whose fine neighbourhood lies inside the window
            # (and the wall side where the window touches the grid's wall)
            i_lo = 1 if s == 1 else 2
            j_lo = 1 if t == 1 else 2
            i_hi = ncw if s + NW - 1 == nx else ncw - 2
            j_hi = ncw if t + NW - 1 == ny else ncw - 2
            for k, key in enumerate(keys):
                sub = np.s_[j_lo:j_hi + 1, i_lo:i_hi + 1]
                gsub = np.s_[J0 + j_lo:J0 + j_hi + 1, I0 + i_lo:I0 + i_hi + 1]
                ok = valid[k][sub]
                diff = np.abs(pg[key][gsub] - planes[k][sub])[ok]
                assert diff.max(initial=0.0) <= 1e-12, (lvl, s, t, key)
            # Galerkin entries of coarse points two coarse cells from the edge
            ac_w = O.galerkin(st_w, p_w)
            ci_lo = 1 if s == 1 else 3
            cj_lo = 1 if t == 1 else 3
            ci_hi = ncw if s + NW - 1 == nx else ncw - 3
            cj_hi = ncw if t + NW - 1 == ny else ncw - 3
            csub = np.s_[cj_lo - 1:cj_hi, ci_lo - 1:ci_hi]
            gcsub = np.s_[J0 + cj_lo - 1:J0 + cj_hi, I0 + ci_lo - 1:I0 + ci_hi]
            scale = np.abs(ac_w["C"][csub])
            for d in ("C", "W", "E", "S", "N", "SW", "SE", "NW", "NE"):
                err = np.abs(coarse[d][gcsub] - ac_w[d][csub]) / scale
                assert err.max() <= 1e-12, (lvl, s, t, d, err.max())


def test_c2_fine_sweep_sampled_against_oracle_windows(c2):
    """One red-black sweep of the 4095^2 finest level by the kernel the bench
    times (TMA-staged, prescaled), forward and reversed, against the oracle's
    sweep on windows: a point two cells from a window's edge depends only on
    values inside it."""
    pr, h = c2
    L = h.nlevels
    assert h.level_prescaled(L - 1)
    st = O.assemble_fv5(pr["k"])
    rng = np.random.default_rng(90)
    x0 = rng.uniform(-1, 1, (C2_SIDE, C2_SIDE))
    b = rng.uniform(-1, 1, (C2_SIDE, C2_SIDE))
    for rev in (False, True):
        xg = h.op_relax(L - 1, dev(x0), dev(b), nu=1, reverse=rev).cpu().numpy()
        for (s, t) in WINDOWS:
            s, t = min(s, C2_SIDE - NW + 1) | 1, min(t, C2_SIDE - NW + 1) | 1
            st_w = crop(st, s, t, NW)
            xw = np.ascontiguousarray(x0[t - 1:t - 1 + NW, s - 1:s - 1 + NW])
            bw = np.ascontiguousarray(b[t - 1:t - 1 + NW, s - 1:s - 1 + NW])
            O.relax(st_w, xw, bw, 1, O.RB_ORDER, reverse=rev)
            lo_i = 0 if s == 1 else 2
            lo_j = 0 if t == 1 else 2
            hi_i = NW if s + NW - 1 == C2_SIDE else NW - 2
            hi_j = NW if t + NW - 1 == C2_SIDE else NW - 2
            got = xg[t - 1 + lo_j:t - 1 + hi_j, s - 1 + lo_i:s - 1 + hi_i]
            ref = xw[lo_j:hi_j, lo_i:hi_i]
            assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max()), (rev, s, t)


def _rel_resid(st, x, b):
    return float(np.linalg.norm(O.residual(st, x, b)) / np.linalg.norm(b))


def test_c2_solve_satisfies_the_stop_test_against_the_oracle_operator(c2):
    """The benchmark's solve (FP64 V(2,1), tol 1e-9): the iterate's residual,
    evaluated with the oracle's assembly, meets the tolerance and matches
    the residual the GPU reports."""
    pr, h = c2
    x, info = h.solve(dev(pr["b"]), tol=1e-9)
    st = O.assemble_fv5(pr["k"])
    xn = x.cpu().numpy()
    rel = _rel_resid(st, xn, pr["b"])
    assert info.rel_resid <= 1e-9 and rel <= 1.2e-9
    assert abs(rel - info.rel_resid) <= 0.2e-9
    # Why this workload is solved to 1e-9 and not 1e-10: rounding the
    # FP64-stored iterate alone moves b - A x by up to eps (|A| |x|) per row,
    # and for this field eps || |A| |x| ||_2 / ||b||_2 lies above 1e-10
    # (high-k blocks at large potential).
    st_abs = dict(st)
    for d in O.DIRS:
        st_abs[d] = -st[d]                       # |A| |x| = C |x| + sum_X a_X |x_X|
    floor = np.finfo(np.float64).eps * np.linalg.norm(O.apply(st_abs, np.abs(xn))) / np.linalg.norm(pr["b"])
    assert floor > 1e-10, floor
    # The same residual in extended precision (the FP64 iterate and FP64
    # operator taken as exact): the solve meets the tolerance exactly, and
    # the stop test's value (summed inside the prescaled fine sweep) is within
    # the FP64 evaluation noise of it
    ld = np.longdouble
    assert np.finfo(ld).eps < 1e-18
    rl = O.residual({d: v.astype(ld) for d, v in st.items()}, xn.astype(ld), pr["b"].astype(ld))
    exact = float(np.sqrt(np.sum(rl * rl)) / ld(np.linalg.norm(pr["b"])))
    assert exact <= 1e-9, exact
    assert abs(info.rel_resid - exact) <= 0.1 * exact, (info.rel_resid, exact, rel)


@pytest.mark.parametrize("nx,ny", [(16383, 1023), (9088, 568)])
def test_paper_workload_solves_satisfy_the_stop_test(nx, ny):
    """D = diag(1/16, 16) on nx x ny cells of the unit square (the paper's
    anisotropy and stretching): FP64 V(2,1), FP32 refinement and PCG to
    1e-10, checked with the oracle's anisotropic assembly."""
    k = np.ones((ny, nx))
    b = np.random.default_rng(91).uniform(-1, 1, (ny, nx))
    st = O.assemble_fv5(k, r=16.0, aspect=nx / ny)
    base = dict(aniso_r=16.0, cell_aspect=nx / ny, max_cycles=500)
    for kw in (dict(), dict(precision=bm.BMG_FP32_REFINE),
               dict(nu1=1, nu2=1, solver=bm.BMG_SOLVER_PCG)):
        h = bm.setup(dev(k), bm.default_options(**base, **kw))
        x, info = h.solve(dev(b), tol=1e-10)
        h.destroy()
        rel = _rel_resid(st, x.cpu().numpy(), b)
        assert info.rel_resid <= 1e-10 and rel <= 1.2e-10, (kw, rel, info.rel_resid)
        assert abs(rel - info.rel_resid) <= 0.2e-10, (kw, rel, info.rel_resid)


def test_c3_fp32_refinement_satisfies_the_fp64_stop_test():
    """8191^2 log-normal field (k = exp(2 g), correlation 32 cells, seed 2,
    as in the benchmark): FP32 V-cycles inside FP64 refinement reach 1e-10
    for the oracle's FP64 operator."""
    pr = inputs.lognormal_problem(8191, seed=2)
    b = pr["b"]
    h = bm.setup(dev(pr["k"]), bm.default_options(precision=bm.BMG_FP32_REFINE, max_cycles=500))
    x, info = h.solve(dev(b), tol=1e-10)
    h.destroy()
    rel = _rel_resid(O.assemble_fv5(pr["k"]), x.cpu().numpy(), b)
    assert info.rel_resid <= 1e-10 and rel <= 1.2e-10, (rel, info.rel_resid)
    assert abs(rel - info.rel_resid) <= 0.2e-10, (rel, info.rel_resid)


def test_line_smoother_solve_at_4095_satisfies_the_stop_test():
    """Alternating line smoothing on D = diag(1/100, 100), 4095^2 square
    cells (the line-smoother benchmark): FP64 V(2,1) to 1e-10."""
    n = 4095
    k = np.ones((n, n))
    b = np.random.default_rng(93).uniform(-1, 1, (n, n))
    h = bm.setup(dev(k), bm.default_options(aniso_r=100.0, smoother=bm.BMG_SMOOTH_ALTLINE))
    x, info = h.solve(dev(b), tol=1e-10)
    h.destroy()
    rel = _rel_resid(O.assemble_fv5(k, r=100.0), x.cpu().numpy(), b)
    assert info.rel_resid <= 1e-10 and rel <= 1.2e-10, (rel, info.rel_resid)
    assert abs(rel - info.rel_resid) <= 0.2e-10, (rel, info.rel_resid)
    assert info.cycles <= 20


def test_3d_solve_at_255_satisfies_the_stop_test():
    """3D block field, 255^3 (the 3D benchmark's size): FP64 V(2,1) to 1e-10
    for the oracle's 7-point assembly."""
    from oracle import boxmg3d_oracle as O3
    n, block = 255, 16
    rng = np.random.default_rng(94)
    nb = -(-n // block)
    kb = 10.0 ** rng.uniform(-2, 2, (nb, nb, nb))
    k = np.repeat(np.repeat(np.repeat(kb, block, 0), block, 1), block, 2)[:n, :n, :n]
    b = rng.uniform(-1, 1, (n, n, n))
    h = bm.setup3(dev(k))
    x, info = h.solve(dev(b), tol=1e-10)
    h.destroy()
    a = O3.assemble_fv7(k)
    r = b.ravel() - a @ x.cpu().numpy().ravel()
    rel = float(np.linalg.norm(r) / np.linalg.norm(b))
    assert info.rel_resid <= 1e-10 and rel <= 1.2e-10, (rel, info.rel_resid)
    assert abs(rel - info.rel_resid) <= 0.2e-10, (rel, info.rel_resid)


def test_3d_setup_sampled_against_oracle_windows():
    """3D at the benchmark size (255^3 block field): interpolation weights
    and Galerkin entries of the GPU hierarchy against the 3D oracle on 17^3
    windows of the GPU's own finest level (interior points: two fine cells,
    or two coarse cells, from a window face that is not a wall)."""
    from oracle import boxmg3d_oracle as O3
    from tests.test_gpu_parity3d import interp_to_csr, stencil_to_csr
    n, block, nw = 255, 16, 17
    rng = np.random.default_rng(95)
    nb = -(-n // block)
    kb = 10.0 ** rng.uniform(-2, 2, (nb, nb, nb))
    k = np.repeat(np.repeat(np.repeat(kb, block, 0), block, 1), block, 2)[:n, :n, :n]
    h = bm.setup3(dev(k))
    L = h.nlevels
    sten = h.level_stencil(L - 1)
    interp = h.level_interp(L - 1)
    coarse = h.level_stencil(L - 2)
    h.destroy()
    nc, cw = n // 2, nw // 2
    for o in [(0, 0, 0), (96, 32, 160), (238, 238, 238), (0, 120, 64)]:   # 0-based, even
        sl = np.s_[:, o[2]:o[2] + nw, o[1]:o[1] + nw, o[0]:o[0] + nw]
        a_w = stencil_to_csr(sten[sl], (nw, nw, nw))
        p_o = O3.interpolation(a_w, (nw, nw, nw))
        p_g = interp_to_csr(np.ascontiguousarray(interp[sl]), (nw, nw, nw))

        lo = [0 if oo == 0 else 2 for oo in o]
        hi = [nw if oo + nw == n else nw - 2 for oo in o]
        kk, jj, ii = np.meshgrid(np.arange(lo[2], hi[2]), np.arange(lo[1], hi[1]),
                                 np.arange(lo[0], hi[0]), indexing="ij")
        rows = ((kk * nw + jj) * nw + ii).ravel()
        assert abs(p_g[rows] - p_o[rows]).max() <= 1e-12, o
        ac_o = O3.galerkin(a_w, p_o, (cw, cw, cw))
        co = tuple(oo // 2 for oo in o)
        cs = np.s_[:, co[2]:co[2] + cw, co[1]:co[1] + cw, co[0]:co[0] + cw]
        ac_g = stencil_to_csr(np.ascontiguousarray(coarse[cs]), (cw, cw, cw))
        clo = [0 if oo == 0 else 2 for oo in o]
        chi = [cw if oo + nw == n else cw - 2 for oo in o]
        kk, jj, ii = np.meshgrid(np.arange(clo[2], chi[2]), np.arange(clo[1], chi[1]),
                                 np.arange(clo[0], chi[0]), indexing="ij")
        crow = ((kk * cw + jj) * cw + ii).ravel()
        diag = np.abs(ac_o.diagonal())[crow]
        err = abs(ac_g[crow] - ac_o[crow]).max(axis=1).toarray().ravel()
        assert (err / diag).max() <= 1e-12, o
