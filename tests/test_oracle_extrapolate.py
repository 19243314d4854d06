"""Pins of the oracle's energy extrapolation in the number of kept block states."""
import numpy as np
import pytest

from oracle.extrapolate import fit_power, fit_quadratic

MS = np.array([256.0, 512.0, 768.0, 1024.0, 2048.0, 3072.0, 4096.0])


def _noisy(seed, e_inf=-78.463, x1=40.0, x2=-0.9, noise=2e-4):
    rng = np.random.default_rng(seed)
    return e_inf + x1 * MS ** x2 + noise * rng.standard_normal(MS.size)


@pytest.mark.parametrize("e_inf,x1,x2", [(-78.463, 40.0, -0.9), (-304.182, 900.0, -1.7),
                                         (-0.5, 2.0, -0.05)])
def test_power_law_data_are_reproduced(e_inf, x1, x2):
    E = e_inf + x1 * MS ** x2
    a, b, c, rms = fit_power(MS, E)
    assert abs(a - e_inf) < 1e-7 * (1 + abs(e_inf))
    assert abs(c - x2) < 1e-6 * abs(x2)
    assert abs(b - x1) < 1e-5 * abs(x1)
    assert rms < 1e-9


def test_quadratic_data_are_reproduced():
    E = -305.5 + 310.0 / MS - 5.0e4 / MS ** 2
    c0, c1, c2, rms = fit_quadratic(MS, E)
    assert abs(c0 + 305.5) < 1e-10 and abs(c1 - 310.0) < 1e-6 and abs(c2 + 5.0e4) < 1e-2
    assert rms < 1e-12


def test_power_fit_is_a_least_squares_minimum():
    """On noisy data: the residual is orthogonal to both linear columns (normal equations
    of E_inf and X1), and no exponent on an independent fine scan does better."""
    E = _noisy(3)
    a, b, c, rms = fit_power(MS, E)
    r = E - (a + b * MS ** c)
    assert abs(r.sum()) < 1e-10 and abs(r @ MS ** c) < 1e-10
    assert abs(np.sqrt(r @ r / MS.size) - rms) < 1e-14
    for x2 in np.linspace(-3.0, -0.01, 3001):
        A = np.stack([np.ones_like(MS), MS ** x2], axis=1)
        coef = np.linalg.solve(A.T @ A, A.T @ E)
        s = E - A @ coef
        assert s @ s >= r @ r - 1e-15


def test_fit_equivariance():
    """Shift and scale of E, and a change of the unit of M, move the parameters as the
    model says (catches a wrong sign or a dropped factor)."""
    E = _noisy(5)
    a, b, c, _ = fit_power(MS, E)
    a2, b2, c2, _ = fit_power(MS, E + 10.0)
    assert abs(a2 - a - 10.0) < 1e-7 and abs(b2 - b) < 1e-5 * abs(b) and abs(c2 - c) < 1e-7
    a3, b3, c3, _ = fit_power(MS, 3.0 * E)
    assert abs(a3 - 3 * a) < 1e-6 and abs(b3 - 3 * b) < 1e-5 * abs(b) and abs(c3 - c) < 1e-7
    a4, b4, c4, _ = fit_power(2.0 * MS, E)
    assert abs(a4 - a) < 1e-7 and abs(b4 - b * 2.0 ** (-c)) < 1e-5 * abs(b)
    assert abs(c4 - c) < 1e-7
    q = fit_quadratic(MS, E)
    q2 = fit_quadratic(MS, E + 10.0)
    assert abs(q2[0] - q[0] - 10.0) < 1e-9 and abs(q2[1] - q[1]) < 1e-6


def test_rejected_inputs():
    with pytest.raises(ValueError):
        fit_power(MS[:2], MS[:2])
    with pytest.raises(ValueError):
        fit_power(np.array([256.0, 256.0, 512.0]), np.array([1.0, 2.0, 3.0]))
    with pytest.raises(ValueError):
        fit_quadratic(np.array([256.0, -1.0, 512.0]), np.array([1.0, 2.0, 3.0]))
    with pytest.raises(ValueError):      # energies falling linearly in M: no limit
        fit_power(MS, -1e-3 * MS)
