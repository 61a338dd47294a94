"""Adjoint gradient on the GPU: autograd through the C ABI.

L = 0.5 ||u - u_obs||^2 with A(exp(theta)) u = b.  The GPU gradient (adjoint
solve on the same hierarchy + the assembly backward kernel) is checked
against the oracle's adjoint gradient (exact sparse solves) on reduced grids,
and against central finite differences (h = 1e-6) on 64 random cells of the
full 2047^2 log-normal field.

Finite differences at 4 million unknowns: L(theta +- h e_c) differ from
L(theta) in about the 12th digit, below the FP64 rounding of the sums and of
the solves.  The perturbed solutions are therefore formed exactly as
u_+- = u_0 + d_+-, where d_+- solves A_+- d = (A_0 - A_+-) u_0 (a right-hand
side supported on cell c and its neighbours, so d is solved to full relative
accuracy), and L_+ - L_- = sum (u_0 - u_obs)(d_+ - d_-) + 0.5 sum (d_+^2 - d_-^2).
This is the central difference itself, rearranged, not a linearisation.
"""
import numpy as np
import pytest

from oracle import boxmg_oracle as O
from paper_1803_02481_gb300 import inputs

torch = pytest.importorskip("torch")
import paper_1803_02481_gb300 as bm  # noqa: E402
from paper_1803_02481_gb300.autograd import solve as diff_solve  # noqa: E402

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("n,solver", [(127, "vcycle"), (255, "vcycle"), (127, "pcg"), (255, "pcg")])
def test_adjoint_gradient_matches_oracle(n, solver):
    """Forward and adjoint solves by V(2,1) cycles or by CG with the
    symmetric V(1,1) preconditioner: the same oracle gradient."""
    pr = inputs.adjoint_problem(n, seed=3)
    u_obs = O.direct_solve(np.exp(pr["theta_obs"]), pr["b"]) + 1e-3 * pr["eps"]
    g_o, u_o, lam_o = O.adjoint_gradient(pr["theta"], pr["b"], u_obs)
    theta = dev(pr["theta"]).requires_grad_(True)
    b = dev(pr["b"]).requires_grad_(True)
    u = diff_solve(theta, b, tol=1e-12, solver=solver)
    loss = 0.5 * ((u - dev(u_obs)) ** 2).sum()
    loss.backward()
    g = theta.grad.cpu().numpy()
    # solves to 1e-12 relative residual: u and lambda carry relative errors of
    # about 1e-12 times the conditioning of the field (< 1e3 here)
    assert np.abs(u.detach().cpu().numpy() - u_o).max() <= 1e-8 * np.abs(u_o).max()
    assert np.abs(g - g_o).max() <= 1e-7 * np.abs(g_o).max()
    assert np.abs(b.grad.cpu().numpy() - lam_o).max() <= 1e-7 * np.abs(lam_o).max()


def _faces(k, c, nx, ny):
    """(neighbour index or -1 for a boundary face) for the four faces of c."""
    j, i = divmod(c, nx)
    out = []
    for dj, di in ((0, -1), (0, 1), (-1, 0), (1, 0)):
        jj, ii = j + dj, i + di
        out.append(jj * nx + ii if 0 <= jj < ny and 0 <= ii < nx else -1)
    return out


def _delta_rhs(kf, u0f, c, kc_new, nx, ny):
    """(A_0 - A_new) u_0 where only k_c changes (dense flat arrays)."""
    rhs = {}
    kc = kf[c]
    for nb in _faces(kf, c, nx, ny):
        if nb < 0:
            da = 2.0 * kc_new - 2.0 * kc
            rhs[c] = rhs.get(c, 0.0) - da * u0f[c]
        else:
            a0 = 2.0 * kc * kf[nb] / (kc + kf[nb])
            a1 = 2.0 * kc_new * kf[nb] / (kc_new + kf[nb])
            da = a1 - a0
            flux = da * (u0f[c] - u0f[nb])
            rhs[c] = rhs.get(c, 0.0) - flux
            rhs[nb] = rhs.get(nb, 0.0) + flux
    return rhs


def test_adjoint_gradient_matches_central_differences_full_size():
    n = 2047
    pr = inputs.adjoint_problem(n, seed=3)
    theta = pr["theta"]
    b = dev(pr["b"])
    # observation: a solve on the perturbed field plus 1e-3 noise
    ho = bm.setup(dev(pr["theta_obs"]), bm.default_options(log_coefficients=1, max_cycles=500))
    u_obs_t, _ = ho.solve(b, tol=1e-11)
    ho.destroy()
    u_obs_t = u_obs_t + 1e-3 * dev(pr["eps"])
    theta_t = dev(theta).requires_grad_(True)
    u0_t = diff_solve(theta_t, b, tol=1e-11, adjoint_tol=1e-12, adjoint_max_cycles=120)
    loss = 0.5 * ((u0_t - u_obs_t) ** 2).sum()
    loss.backward()
    g = theta_t.grad.cpu().numpy().ravel()

    kf = np.exp(theta).ravel()
    u0f = u0_t.detach().cpu().numpy().ravel()
    w = (u0f - u_obs_t.cpu().numpy().ravel())
    rng = np.random.default_rng(33)
    cells = rng.choice(n * n, size=64, replace=False)
    h = 1e-6
    gmax = np.abs(g).max()
    fd = np.zeros(64)
    for m, c in enumerate(cells):
        d = {}
        for sgn in (1, -1):
            th = theta.ravel().copy()
            th[c] += sgn * h
            kc_new = np.exp(th[c])
            rhs = np.zeros(n * n)
            for q, v in _delta_rhs(kf, u0f, c, kc_new, n, n).items():
                rhs[q] = v
            hs = bm.setup(dev(th.reshape(n, n)), bm.default_options(log_coefficients=1, max_cycles=500))
            dd, _ = hs.solve(dev(rhs.reshape(n, n)), tol=1e-10)
            hs.destroy()
            d[sgn] = dd.cpu().numpy().ravel()
        dl = np.dot(w, d[1] - d[-1]) + 0.5 * (np.dot(d[1], d[1]) - np.dot(d[-1], d[-1]))
        fd[m] = dl / (2 * h)
    err = np.abs(fd - g[cells])
    assert np.all(err <= 1e-4 * np.abs(g[cells]) + 1e-6 * gmax), (err.max(), np.abs(g[cells]).max())
