"""Seeded synthetic inputs for the diffusion workloads of Section 5.

The paper's experiments (Section 5, Eq. (diffusion)/(diffusion_bc)) solve
-div(D grad u) = f on the unit square with u = 0 on the boundary.  These
generators produce cell coefficient fields ``k`` and right-hand sides ``b``
with the shapes and value distributions of the five workloads this library is
measured on.  They hold none of the multigrid method's arithmetic: both the
GPU path and the CPU oracle receive the arrays produced here.

Conventions
-----------
* Arrays are NumPy float64, shape ``(ny, nx)``, row-major: ``a[j, i]`` is the
  cell in column ``i`` (x, fast) and row ``j`` (y, slow).
* Every generator draws from ``numpy.random.default_rng(seed)`` (PCG64).  For
  one seed the draws happen in a fixed order: coefficients first, then the
  right-hand side, then anything else the workload needs.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

SIDES_BATCH = (63, 127, 255, 511, 1023)
SIDE_WEIGHTS_BATCH = (8, 4, 2, 1, 1)


def uniform_rhs(rng: np.random.Generator, nx: int, ny: int) -> np.ndarray:
    """i.i.d. uniform[-1, 1] right-hand side, shape (ny, nx)."""
    return rng.uniform(-1.0, 1.0, size=(ny, nx))


def block_field(rng: np.random.Generator, nx: int, ny: int, block: int,
                lo: float, hi: float) -> np.ndarray:
    """Piecewise-constant field 10**U on ``block`` x ``block`` cell blocks.

    U is uniform[lo, hi], one draw per block, blocks ordered row-major.  The
    last block in each direction is cut to what remains (4095 cells in
    64-cell blocks gives 64 blocks, the last 63 wide).
    """
    bx = -(-nx // block)
    by = -(-ny // block)
    u = rng.uniform(lo, hi, size=(by, bx))
    k = 10.0 ** u
    return np.repeat(np.repeat(k, block, axis=0), block, axis=1)[:ny, :nx].copy()


def _gauss_filter_axis(a: np.ndarray, ell: float, axis: int) -> np.ndarray:
    """Linear convolution along ``axis`` with exp(-d^2/ell^2), via a
    zero-padded FFT of twice the length (no wrap-around inside the grid);
    the transforms run on every host core."""
    n = a.shape[axis]
    m = 2 * n
    d = np.arange(m, dtype=np.float64)
    d = np.minimum(d, m - d)
    h = np.exp(-(d * d) / (ell * ell))
    hh = sfft.rfft(h)
    shape = [1] * a.ndim
    shape[axis] = hh.shape[0]
    fa = sfft.rfft(a, n=m, axis=axis, workers=-1)
    fa *= hh.reshape(shape)
    out = sfft.irfft(fa, n=m, axis=axis, workers=-1)
    sl = [slice(None)] * a.ndim
    sl[axis] = slice(0, n)
    return np.ascontiguousarray(out[tuple(sl)])


def gaussian_random_field(rng: np.random.Generator, nx: int, ny: int,
                          ell: float = 32.0) -> np.ndarray:
    """Zero-mean, unit-sample-variance Gaussian random field.

    Spectral synthesis of a field with squared-exponential covariance
    exp(-d^2 / (2 ell^2)) (d in cells): white noise is filtered by the
    Gaussian whose self-convolution is that covariance, exp(-d^2/ell^2).  The
    covariance is separable, so the 2D filter is two 1D FFT convolutions on a
    zero-padded periodic grid of twice the size.  The result is standardised
    to sample mean 0 and sample variance 1.
    """
    w = rng.standard_normal((ny, nx))
    g = _gauss_filter_axis(w, ell, axis=1)
    g = _gauss_filter_axis(g, ell, axis=0)
    g -= g.mean()
    g /= g.std()
    return g


# ---------------------------------------------------------------------------
# The five workloads.
# ---------------------------------------------------------------------------

def constant_problem(n: int = 255, seed: int = 0, nx: int | None = None,
                     ny: int | None = None):
    """Constant coefficient 1, uniform[-1,1] RHS (the 255 x 255 Poisson case)."""
    nx = n if nx is None else nx
    ny = n if ny is None else ny
    rng = np.random.default_rng(seed)
    k = np.ones((ny, nx))
    b = uniform_rhs(rng, nx, ny)
    return {"name": f"poisson_{nx}x{ny}", "k": k, "b": b}


def block_problem(n: int = 4095, seed: int = 1, block: int = 64,
                  lo: float = -4.0, hi: float = 4.0, nx: int | None = None,
                  ny: int | None = None):
    """Block-piecewise coefficients 10**U(lo, hi) on block x block cells
    (the 4095 x 4095, 64-cell-block, 10^[-4,4] case by default)."""
    nx = n if nx is None else nx
    ny = n if ny is None else ny
    rng = np.random.default_rng(seed)
    k = block_field(rng, nx, ny, block, lo, hi)
    b = uniform_rhs(rng, nx, ny)
    return {"name": f"blocks{block}_1e{int(hi - lo)}_{nx}x{ny}", "k": k, "b": b}


def lognormal_problem(n: int = 8191, seed: int = 2, ell: float = 32.0,
                      sigma: float = 2.0):
    """Log-normal field k = exp(sigma * g), g a GRF with correlation length
    ell cells (the 8191 x 8191 mixed-precision case by default)."""
    rng = np.random.default_rng(seed)
    g = gaussian_random_field(rng, n, n, ell)
    k = np.exp(sigma * g)
    b = uniform_rhs(rng, n, n)
    return {"name": f"lognormal_{n}", "k": k, "b": b}


def adjoint_problem(n: int = 2047, seed: int = 3, ell: float = 32.0):
    """Inputs of the adjoint-gradient case: log-coefficients theta = 2 g,
    RHS b, a perturbed field theta_obs = theta + 0.1 g' from which the
    observation is solved, and the observation noise eps ~ N(0, 1) (to be
    scaled by 1e-3).  Draw order: g, b, g', eps."""
    rng = np.random.default_rng(seed)
    g = gaussian_random_field(rng, n, n, ell)
    theta = 2.0 * g
    b = uniform_rhs(rng, n, n)
    g2 = gaussian_random_field(rng, n, n, ell)
    theta_obs = theta + 0.1 * g2
    eps = rng.standard_normal((n, n))
    return {"name": f"adjoint_{n}", "theta": theta, "b": b,
            "theta_obs": theta_obs, "eps": eps}


def batch_problems(count: int = 512, seed: int = 4, block: int = 16,
                   lo: float = -3.0, hi: float = 3.0,
                   sides=SIDES_BATCH, weights=SIDE_WEIGHTS_BATCH):
    """Many independent square problems of uneven size.

    Sides are drawn first (``rng.choice`` with the given weights), then for
    each problem in order its block coefficients 10**U(lo, hi) on
    block x block cells and its uniform[-1, 1] RHS.
    """
    rng = np.random.default_rng(seed)
    p = np.asarray(weights, dtype=np.float64)
    p = p / p.sum()
    ns = rng.choice(np.asarray(sides), size=count, p=p)
    probs = []
    for n in ns:
        n = int(n)
        k = block_field(rng, n, n, block, lo, hi)
        b = uniform_rhs(rng, n, n)
        probs.append({"n": n, "k": k, "b": b})
    return probs

