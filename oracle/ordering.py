"""Oracle: orbital ordering from the mutual information by spectral graph theory.

TEST INFRASTRUCTURE ONLY (checks the library's host-side ordering).

The paper orders the orbitals along the chain by minimising the entanglement distance
I_dist = sum_ij I_ij |i - j|^eta with eta = 2, using spectral graph theory.  For eta = 2
and positions relaxed to real numbers x with sum x = 0 and |x| = 1, sum_ij I_ij (x_i -
x_j)^2 = 2 x^T L x with the graph Laplacian L = D - I (D = diag of the row sums of I,
diagonal of I ignored), so the minimiser is the eigenvector of the second smallest
eigenvalue of L (the Fiedler vector); sites are placed in the order of its components.
Readings where the paper is silent: the Fiedler vector is normalised and its sign fixed
so that, among the components within 1e-9 (relative) of the largest magnitude, the one of
the lowest site index is positive; sites are sorted by ascending component, equal
components by site index.  When the second and third eigenvalues coincide the Fiedler
vector is not unique and neither is the order (not used as a parity case).
"""
import numpy as np


def laplacian(I):
    W = np.array(I, dtype=np.float64)
    np.fill_diagonal(W, 0.0)
    return np.diag(W.sum(axis=1)) - W


def fiedler_vector(I):
    w, V = np.linalg.eigh(laplacian(I))
    v = V[:, 1] / np.linalg.norm(V[:, 1])
    a = np.abs(v)
    k = int(np.flatnonzero(a >= a.max() * (1.0 - 1e-9))[0])
    return -v if v[k] < 0 else v


def fiedler_order(I):
    """order[k] = the site placed at chain position k."""
    v = fiedler_vector(I)
    return sorted(range(len(v)), key=lambda i: (v[i], i))


def entanglement_distance(I, order, eta=2.0):
    """sum_{i != j} I_ij |pos(i) - pos(j)|^eta for the chain order `order`."""
    pos = np.empty(len(order), dtype=np.float64)
    pos[np.asarray(order)] = np.arange(len(order))
    W = np.array(I, dtype=np.float64)
    np.fill_diagonal(W, 0.0)
    return float(np.sum(W * np.abs(pos[:, None] - pos[None, :]) ** eta))
