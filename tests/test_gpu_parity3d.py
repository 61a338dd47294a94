"""GPU parity of the 3D BoxMG path (through the C ABI, include/boxmg3d.h)
against the 3D CPU oracle.

Tolerances: the finest level is assembled with the oracle's operation order
and must match exactly; interpolation weights from the GPU's own A_l agree
with the oracle's to 1e-12 (same operation order, unfused); each Galerkin
product from the GPU's own A_l and P_l to 1e-12 of the row diagonal (a
different summation order); solves: identical cycle counts, relative
residuals within 1e-13 (the FP64 rounding of b - Ax near convergence; the
GPU smoother multiplies by 1/C where the oracle divides), iterates within
1e-9 of max|x|.
"""
import functools

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import boxmg3d_oracle as O3

torch = pytest.importorskip("torch")
import paper_1803_02481_gb300 as bm  # noqa: E402

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def block_k(shape, seed, block=4, lo=-2, hi=2):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    nb = [-(-s // block) for s in (nz, ny, nx)]
    kb = 10.0 ** rng.uniform(lo, hi, nb)
    return np.repeat(np.repeat(np.repeat(kb, block, 0), block, 1), block, 2)[:nz, :ny, :nx]


CASES = {
    "blocks15": lambda: (block_k((15, 15, 15), 21), 22),
    "blocks31_c4": lambda: (block_k((31, 31, 31), 23, block=8, lo=-2, hi=2), 24),
    "poisson31": lambda: (np.ones((31, 31, 31)), 25),
    "general12x9x7": lambda: (block_k((12, 9, 7), 26, block=3), 27),
    "general40x24x20": lambda: (block_k((40, 24, 20), 28, block=5), 29),
    "tiny4": lambda: (block_k((4, 4, 4), 30, block=2), 31),
    # a longer general grid (odd and even sides, four levels)
    "general45x20x70": lambda: (block_k((45, 20, 70), 34, block=6), 35),
    "single3": lambda: (block_k((3, 3, 3), 32, block=1), 33),
}


@functools.lru_cache(maxsize=None)
def case(name):
    k, seed = CASES[name]()
    nz, ny, nx = k.shape
    b = np.random.default_rng(seed).uniform(-1, 1, (nz, ny, nx))
    return k, b


@functools.lru_cache(maxsize=None)
def oracle_h(name):
    return O3.setup(case(name)[0])


def stencil_to_csr(planes, shape):
    """GPU stencil planes (14, nz, ny, nx) -> CSR (couplings to +d from the
    neighbour's -d entry)."""
    nx, ny, nz = shape
    n = nx * ny * nz
    idx = np.arange(n).reshape(nz, ny, nx)
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [planes[0].ravel()]
    for m, (di, dj, dk) in enumerate(bm.STENCIL3_OFFSETS):
        a = planes[1 + m]
        k0, k1 = max(0, -dk), nz - max(0, dk)
        j0, j1 = max(0, -dj), ny - max(0, dj)
        i0, i1 = max(0, -di), nx - max(0, di)
        r = idx[k0:k1, j0:j1, i0:i1].ravel()
        c = idx[k0 + dk:k1 + dk, j0 + dj:j1 + dj, i0 + di:i1 + di].ravel()
        v = -a[k0:k1, j0:j1, i0:i1].ravel()
        rows += [r, c]
        cols += [c, r]
        vals += [v, v]
    m = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return m.tocsr()


def interp_to_csr(planes, shape):
    nx, ny, nz = shape
    cx, cy, cz = nx // 2, ny // 2, nz // 2
    rows, cols, vals = [], [], []
    kk, jj, ii = np.meshgrid(np.arange(1, nz + 1), np.arange(1, ny + 1), np.arange(1, nx + 1),
                             indexing="ij")
    f = ((kk - 1) * ny + (jj - 1)) * nx + (ii - 1)
    for m in range(8):
        sx, sy, sz = m & 1, (m >> 1) & 1, m >> 2

        def par(q, s):
            return np.where(q % 2 == 1, (q - 1) // 2 + s, q // 2)

        ok = ~(((ii % 2 == 0) & (sx == 1)) | ((jj % 2 == 0) & (sy == 1)) | ((kk % 2 == 0) & (sz == 1)))
        I, J, K = par(ii, sx), par(jj, sy), par(kk, sz)
        ok &= (I >= 1) & (I <= cx) & (J >= 1) & (J <= cy) & (K >= 1) & (K <= cz)
        w = planes[m]
        ok &= w != 0
        rows.append(f[ok])
        cols.append((((K - 1) * cy + (J - 1)) * cx + (I - 1))[ok])
        vals.append(w[ok])
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(nx * ny * nz, cx * cy * cz)).tocsr()


@pytest.mark.parametrize("name", list(CASES))
def test_3d_setup_each_step_matches_oracle(name):
    k, _ = case(name)
    ho = oracle_h(name)
    hg = bm.setup3(dev(k))
    L = len(ho.levels)
    assert hg.nlevels == L
    for l in range(L):
        assert hg.level_shape(l) == ho.levels[l].shape, l
    fine = stencil_to_csr(hg.level_stencil(L - 1), ho.levels[-1].shape)
    assert abs(fine - ho.levels[-1].a).max() == 0
    for l in range(L - 1, 0, -1):
        shape = ho.levels[l].shape
        a_g = stencil_to_csr(hg.level_stencil(l), shape)
        p_o = O3.interpolation(a_g, shape)
        p_g = interp_to_csr(hg.level_interp(l), shape)
        assert abs(p_g - p_o).max() <= 1e-12, l
        ac_o = O3.galerkin(a_g, p_o, ho.levels[l - 1].shape)
        ac_g = stencil_to_csr(hg.level_stencil(l - 1), ho.levels[l - 1].shape)
        diag = np.abs(ac_o.diagonal())
        err = abs(ac_g - ac_o).tocsr()
        rel = max((err.getrow(r).max() / diag[r]) for r in range(err.shape[0]))
        assert rel <= 1e-12, (l, rel)
    hg.destroy()


@pytest.mark.parametrize("name", list(CASES))
def test_3d_solve_matches_oracle(name):
    k, b = case(name)
    ro = O3.solve(oracle_h(name), b, tol=1e-10)
    hg = bm.setup3(dev(k))
    x, info = hg.solve(dev(b), tol=1e-10)
    hg.destroy()
    xg = x.cpu().numpy()
    assert ro.converged and info.cycles == ro.cycles, (info.cycles, ro.cycles)
    assert info.rel_resid <= 1e-10
    assert abs(info.rel_resid - ro.rel_resid) <= 1e-13
    assert np.abs(xg - ro.x).max() <= 1e-9 * np.abs(ro.x).max()
    a = oracle_h(name).levels[-1].a
    rel = np.linalg.norm(b.ravel() - a @ xg.ravel()) / np.linalg.norm(b)
    assert rel <= 1.0000001e-10


@pytest.mark.parametrize("name", ["blocks15", "blocks31_c4", "poisson31", "general45x20x70",
                                  "general12x9x7", "tiny4", "single3"])
def test_3d_fp32_refinement_reaches_fp64_tolerance(name):
    """FP32 V-cycles inside FP64 refinement: the iterate meets the FP64 stop
    test against the oracle's operator, and its error against the FP64
    oracle solution is what a 1e-10 relative residual allows."""
    k, b = case(name)
    ro = O3.solve(oracle_h(name), b, tol=1e-10)
    hg = bm.setup3(dev(k), bm.default_options(precision=bm.BMG_FP32_REFINE))
    x, info = hg.solve(dev(b), tol=1e-10)
    hg.destroy()
    xg = x.cpu().numpy()
    a = oracle_h(name).levels[-1].a
    rel = np.linalg.norm(b.ravel() - a @ xg.ravel()) / np.linalg.norm(b)
    assert rel <= 1.0000001e-10 and info.rel_resid <= 1e-10
    assert np.abs(xg - ro.x).max() <= 1e-7 * np.abs(ro.x).max()
    # a step contracts the residual about as much as an FP64 cycle
    assert info.cycles <= 2 * ro.cycles + 4, (info.cycles, ro.cycles)


@functools.lru_cache(maxsize=None)
def oracle_pcg(name):
    k, b = case(name)
    return O3.pcg(O3.setup(k, nu1=1, nu2=1), b, tol=1e-10)


PCG_CASES = ["blocks15", "blocks31_c4", "poisson31", "general45x20x70", "general12x9x7", "tiny4"]


@pytest.mark.parametrize("name", PCG_CASES)
def test_3d_pcg_matches_oracle(name):
    """CG preconditioned by one symmetric V(1,1) cycle: the oracle's
    iteration count, its final relative residual to rounding (the dot
    products are summed in another order) and its iterate."""
    k, b = case(name)
    ro = oracle_pcg(name)
    hg = bm.setup3(dev(k), bm.default_options(nu1=1, nu2=1, solver=bm.BMG_SOLVER_PCG, max_cycles=400))
    x, info = hg.solve(dev(b), tol=1e-10)
    hg.destroy()
    xg = x.cpu().numpy()
    assert ro.converged and info.cycles == ro.cycles, (info.cycles, ro.cycles)
    assert abs(info.rel_resid - ro.rel_resid) <= 1e-7 * ro.rel_resid + 1e-14
    assert np.abs(xg - ro.x).max() <= 1e-9 * np.abs(ro.x).max()
    # the true residual of the returned x (the stop test uses the updated one)
    a = oracle_h(name).levels[-1].a
    assert np.linalg.norm(b.ravel() - a @ xg.ravel()) / np.linalg.norm(b) <= 2e-10


@pytest.mark.parametrize("name", PCG_CASES)
def test_3d_pcg_with_fp32_cycles_reaches_fp64_tolerance(name):
    """The same with the V-cycle on the FP32 copies of the levels (r / ||r||
    cast down, ||r|| e cast back): the FP64 recurrences still reach 1e-10."""
    k, b = case(name)
    ro = oracle_pcg(name)
    hg = bm.setup3(dev(k), bm.default_options(nu1=1, nu2=1, solver=bm.BMG_SOLVER_PCG, max_cycles=400,
                                              precision=bm.BMG_FP32_REFINE))
    x, info = hg.solve(dev(b), tol=1e-10)
    hg.destroy()
    xg = x.cpu().numpy()
    a = oracle_h(name).levels[-1].a
    assert info.rel_resid <= 1e-10
    assert np.linalg.norm(b.ravel() - a @ xg.ravel()) / np.linalg.norm(b) <= 2e-10
    assert np.abs(xg - ro.x).max() <= 1e-7 * np.abs(ro.x).max()
    assert info.cycles <= ro.cycles + 3, (info.cycles, ro.cycles)


def test_3d_zero_rhs_and_error_codes():
    k = np.ones((7, 7, 7))
    h = bm.setup3(dev(k))
    x, info = h.solve(dev(np.zeros((7, 7, 7))), tol=1e-10)
    assert info.cycles == 0 and not x.abs().max().item()
    h.destroy()
    for bad in [np.ones((1, 7, 7)), -np.ones((7, 7, 7)), np.full((7, 7, 7), np.nan)]:
        with pytest.raises(bm.BoxMGError) as e:
            bm.setup3(dev(bad))
        assert e.value.code == bm.BMG_EINVAL
    for opts in (dict(smoother=bm.BMG_SMOOTH_ALTLINE), dict(solver=bm.BMG_SOLVER_PCG),
                 dict(aniso_r=2.0)):
        with pytest.raises(bm.BoxMGError) as e:
            bm.setup3(dev(k), bm.default_options(**opts))
        assert e.value.code == bm.BMG_EINVAL
    # the coarsest level would exceed the dense-solve limit
    with pytest.raises(bm.BoxMGError) as e:
        bm.setup3(dev(np.ones((3, 40, 40))))
    assert e.value.code == bm.BMG_EINVAL
    # max_cycles reached
    k, b = case("blocks15")
    h = bm.setup3(dev(k), bm.default_options(max_cycles=2))
    with pytest.raises(bm.BoxMGError) as e:
        h.solve(dev(b), tol=1e-14)
    assert e.value.code == bm.BMG_ENOCONV
    h.destroy()



@pytest.mark.parametrize("name", ["blocks31_c4", "general45x20x70", "general12x9x7"])
@pytest.mark.parametrize("nu", [(2, 1), (1, 1)])
def test_3d_paired_colour_sweeps_are_bit_identical(name, nu, monkeypatch):
    """The 27-point sweeps as four colour-pair launches (one thread block per
    x-row, the two colours of a row separated by a barrier) give the same
    bits as eight colour launches, forward and reversed."""
    k, b = case(name)
    out = []
    for pairs in ("0", "1"):
        monkeypatch.setenv("BMG3_GS27_PAIRS", pairs)
        h = bm.setup3(dev(k), bm.default_options(nu1=nu[0], nu2=nu[1], max_cycles=400))
        x, info = h.solve(dev(b), tol=1e-10)
        h.destroy()
        out.append((x.cpu().numpy(), info.cycles, info.rel_resid))
    assert out[0][1] == out[1][1] and out[0][2] == out[1][2]
    assert np.array_equal(out[0][0], out[1][0])


@pytest.mark.parametrize("name", ["blocks31_c4", "general45x20x70", "tiny4"])
@pytest.mark.parametrize("nu,stream_launched", [((2, 1), False), ((2, 1), True), ((1, 1), False),
                                                ((1, 0), False)])
def test_3d_stop_test_in_the_next_sweep_is_bit_identical(name, nu, stream_launched, monkeypatch):
    """FP64 V-cycles take the stop test inside the next cycle's first fine
    sweep (its first colour a copy, its second colour's updates giving the
    residual), out of place, so the loop returns the iterate that sweep read.
    Against the separate norm pass: the same iterates bit for bit after an
    odd and an even number of cycles and at convergence, the same cycle
    counts, residuals equal to rounding.  V(1,0) has no fusion."""
    k, b = case(name)
    out = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("BMG3_FUSED_NORM", mode)
        for cap, tol in ((5, 1e-300), (6, 1e-300), (400, 1e-10)):
            h = bm.setup3(dev(k), bm.default_options(nu1=nu[0], nu2=nu[1], max_cycles=cap))
            if stream_launched:
                bm.profile_set(("norm",))
            try:
                x, info = h.solve(dev(b), tol=tol, allow_noconv=True)
            finally:
                bm.profile_set(())
            h.destroy()
            out[mode, cap] = (x.cpu().numpy(), info.cycles, info.rel_resid)
    a = oracle_h(name).levels[-1].a
    for cap in (5, 6, 400):
        (x0, c0, r0), (x1, c1, r1) = out["0", cap], out["1", cap]
        assert c0 == c1, (cap, c0, c1)
        assert np.array_equal(x0, x1), cap
        assert abs(r1 - r0) <= 1e-6 * r0 + 1e-15, (cap, r0, r1)
        rel = np.linalg.norm(b.ravel() - a @ x1.ravel()) / np.linalg.norm(b)
        assert abs(r1 - rel) <= 1e-6 * rel + 1e-15, (cap, r1, rel)
    assert out["1", 5][1] == 5 and out["1", 6][1] == 6
