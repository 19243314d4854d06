"""Oracle: extrapolation of DMRG energies in the number of kept block states M.

TEST INFRASTRUCTURE ONLY (checks the library's host-side fits).

The method description fits the energies of runs at several M with
    E(M) = E_inf + X1 M^X2,
E_inf, X1 and X2 free, and takes E_inf as the truncation-free estimate; the 64Ge results
add an upper bound from a second-order polynomial fit.  Readings where the paper is
silent:
* both fits are ordinary least squares over the given points, equal weights;
* the power law is sought with X2 in [-8, -1e-4] (E converges as M grows); a best X2 on
  either end of that range means the data show no power-law approach and the fit fails;
* the polynomial is in x = 1/M, E = c0 + c1 x + c2 x^2, and its estimate is c0 (x -> 0).

The power-law fit follows from the model's structure: at a fixed X2 it is linear in
(E_inf, X1), solved by a library least-squares routine; X2 is located on a dense grid
and refined inside the best grid cell by bounded scalar minimisation.  Slow and plain.
"""
import numpy as np
from scipy.optimize import minimize_scalar

X2_LO, X2_HI = -8.0, -1e-4


def _check(M, E):
    M = np.asarray(M, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    if M.shape != E.shape or M.ndim != 1 or len(M) < 3:
        raise ValueError("need at least three (M, E) pairs")
    if not (np.all(np.isfinite(M)) and np.all(np.isfinite(E)) and np.all(M > 0)):
        raise ValueError("M must be positive and M, E finite")
    if len(np.unique(M)) < 3:
        raise ValueError("need at least three distinct M")
    return M, E


def _linear_at(M, E, x2):
    """Least-squares (E_inf, X1) at fixed X2 and the residual sum of squares."""
    A = np.stack([np.ones_like(M), M ** x2], axis=1)
    coef, *_ = np.linalg.lstsq(A, E, rcond=None)
    r = E - A @ coef
    return coef[0], coef[1], float(r @ r)


def fit_power(M, E, n_grid=20001):
    """E(M) = E_inf + X1 M^X2 by least squares.  Returns (E_inf, X1, X2, rms)."""
    M, E = _check(M, E)
    grid = np.linspace(X2_LO, X2_HI, n_grid)
    ss = np.array([_linear_at(M, E, b)[2] for b in grid])
    i = int(np.argmin(ss))
    if i == 0 or i == n_grid - 1:
        raise ValueError("no power-law minimum inside the X2 range")
    res = minimize_scalar(lambda b: _linear_at(M, E, b)[2], bounds=(grid[i - 1], grid[i + 1]),
                          method="bounded", options={"xatol": 1e-13})
    b = float(res.x) if res.fun <= ss[i] else float(grid[i])
    e_inf, x1, s = _linear_at(M, E, b)
    return e_inf, x1, b, float(np.sqrt(s / len(M)))


def fit_quadratic(M, E):
    """E = c0 + c1 / M + c2 / M^2 by least squares.  Returns (c0, c1, c2, rms)."""
    M, E = _check(M, E)
    x = 1.0 / M
    A = np.stack([np.ones_like(x), x, x * x], axis=1)
    coef, *_ = np.linalg.lstsq(A, E, rcond=None)
    r = E - A @ coef
    return float(coef[0]), float(coef[1]), float(coef[2]), float(np.sqrt(r @ r / len(M)))
