"""Pins of the oracle's spectral orbital ordering: the path graph's closed-form Fiedler
vector, recovery of a hidden chain order, the variational property of the Fiedler
vector, and brute force over every order of a small case whose optimum is known."""
import itertools
import math

import numpy as np
import pytest

from oracle.ordering import entanglement_distance, fiedler_order, fiedler_vector, laplacian


def _path(n, w=1.0):
    I = np.zeros((n, n))
    for i in range(n - 1):
        I[i, i + 1] = I[i + 1, i] = w
    return I


@pytest.mark.parametrize("n", [3, 8, 17])
def test_path_graph_closed_form(n):
    # L of the path: eigenvalues 2 - 2 cos(pi k / n), eigenvectors cos(pi k (i + 1/2) / n)
    v = fiedler_vector(_path(n, 0.7))
    ref = np.array([math.cos(math.pi * (i + 0.5) / n) for i in range(n)])
    ref /= np.linalg.norm(ref)
    assert np.max(np.abs(v - ref)) < 1e-10        # sign: site 0 positive (end tie)
    lam = v @ laplacian(_path(n, 0.7)) @ v
    assert abs(lam - 0.7 * (2 - 2 * math.cos(math.pi / n))) < 1e-12
    assert fiedler_order(_path(n)) == list(range(n))[::-1]


def test_hidden_chain_is_recovered():
    rng = np.random.default_rng(3)
    n = 24
    hidden = rng.permutation(n)                   # hidden[k] = site at position k
    pos = np.empty(n, dtype=int)
    pos[hidden] = np.arange(n)
    I = np.exp(-np.abs(pos[:, None] - pos[None, :]).astype(float))
    order = fiedler_order(I)
    assert order == list(hidden) or order == list(hidden[::-1])


def test_fiedler_vector_minimises_the_relaxed_distance():
    rng = np.random.default_rng(5)
    A = rng.random((10, 10))
    I = A + A.T
    L = laplacian(I)
    v = fiedler_vector(I)
    assert abs(v.sum()) < 1e-10 and abs(v @ v - 1) < 1e-12
    lam = v @ L @ v
    for _ in range(200):
        x = rng.standard_normal(10)
        x -= x.mean()
        x /= np.linalg.norm(x)
        assert x @ L @ x >= lam - 1e-12


def test_brute_force_optimum_on_a_small_case():
    """I_ij = exp(-|pos_i - pos_j|) for a hidden order of 7 orbitals: the hidden order (or
    its reverse) is the minimum of the entanglement distance over all 5040 orders, and
    the spectral ordering finds it."""
    rng = np.random.default_rng(8)
    n = 7
    hidden = rng.permutation(n)
    pos = np.empty(n, dtype=int)
    pos[hidden] = np.arange(n)
    I = np.exp(-np.abs(pos[:, None] - pos[None, :]).astype(float))
    best = min(itertools.permutations(range(n)), key=lambda o: entanglement_distance(I, o))
    d_best = entanglement_distance(I, best)
    assert abs(d_best - entanglement_distance(I, hidden)) < 1e-12
    assert abs(entanglement_distance(I, fiedler_order(I)) - d_best) < 1e-12
