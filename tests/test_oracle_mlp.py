"""Pin of the oracle network: analytic gradient against central finite differences."""
import numpy as np

from oracle import mlp


def _random_problem(seed, B=16):
    rng = np.random.default_rng(seed)
    theta = rng.standard_normal(mlp.n_params()) * 0.1
    X = rng.standard_normal((B, mlp.N_IN))
    T = rng.standard_normal(B)
    return theta, X, T


def test_gradient_central_differences():
    theta, X, T = _random_problem(0)
    loss, g = mlp.loss_and_grad(theta, X, T)
    rng = np.random.default_rng(1)
    # every parameter group, a few coordinates each
    o = 0
    idx = []
    for s in mlp.SHAPES:
        k = int(np.prod(s))
        idx += list(o + rng.choice(k, size=min(k, 6), replace=False))
        o += k
    h = 1e-6
    for i in idx:
        tp = theta.copy()
        tm = theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_and_grad(tp, X, T)[0] - mlp.loss_and_grad(tm, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_loss_is_mean_squared_error_of_forward():
    theta, X, T = _random_problem(2)
    y, _ = mlp.forward(theta, X)
    assert abs(mlp.loss_and_grad(theta, X, T)[0] - np.mean((y - T) ** 2)) < 1e-14
    # a network with zero hidden weights outputs its last bias
    z = np.zeros_like(theta)
    z[-1] = 0.75
    assert np.allclose(mlp.forward(z, X)[0], 0.75)
