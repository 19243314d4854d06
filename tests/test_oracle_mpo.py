"""Brute-force pin of the normal / complementary operator partition: for small chains,
sum_k (L_k P^{|R_k|}) (x) R_k rebuilt on the full Fock space equals H from Jordan-Wigner
matrices at every bond."""
import numpy as np
import pytest
import scipy.sparse as sp

from gen import make_problem
from oracle.hamiltonian import ChainHamiltonian, fock_matrix
from oracle.mpo import MPO, SITE_PARITY, mode

SITE = {"I": np.eye(2), "N": np.diag([0.0, 1.0]),
        "Cd": np.array([[0.0, 0.0], [1.0, 0.0]]), "C": np.array([[0.0, 1.0], [0.0, 0.0]])}


def _parity_diag(d):
    return np.array([(-1.0) ** bin(x).count("1") for x in range(d)])


def _check(prob, bonds=None):
    ch = ChainHamiltonian(prob)
    mpo = MPO(ch)
    N = ch.N
    H = fock_matrix(ch)
    left = [[sp.csr_matrix(np.ones((1, 1)))]]
    for s in range(N):
        d = left[-1][0].shape[0]
        P = sp.diags(_parity_diag(d))
        new = [sp.csr_matrix((2 * d, 2 * d)) for _ in mpo.labels[s + 1]]
        for (a, b, op, c) in mpo.W[s]:
            X = left[-1][a] @ P if SITE_PARITY[op] else left[-1][a]
            new[b] = new[b] + c * sp.kron(X, SITE[op], format="csr")
        left.append(new)
    assert abs(left[N][0] - H).max() < 1e-12
    right = [None] * (N + 1)
    right[N] = [sp.csr_matrix(np.ones((1, 1)))]
    Z = np.diag([1.0, -1.0])
    for s in range(N - 1, -1, -1):
        d = right[s + 1][0].shape[0]
        new = [sp.csr_matrix((2 * d, 2 * d)) for _ in mpo.labels[s]]
        for (a, b, op, c) in mpo.W[s]:
            w = SITE[op] @ Z if mpo.parity[s + 1][b] else SITE[op]
            new[a] = new[a] + c * sp.kron(w, right[s + 1][b], format="csr")
        right[s] = new
    assert abs(right[0][0] - H).max() < 1e-12
    modes = set()
    for b in (bonds if bonds is not None else range(-1, N)):
        Ls, Rs = left[b + 1], right[b + 1]
        P = sp.diags(_parity_diag(Ls[0].shape[0]))
        tot = sp.csr_matrix(H.shape)
        for k in range(len(Ls)):
            X = Ls[k] @ P if mpo.parity[b + 1][k] else Ls[k]
            tot = tot + sp.kron(X, Rs[k], format="csr")
        assert abs(tot - H).max() < 1e-11, b
        if 0 <= b < N:
            modes.add(mode(b, N))
    return modes


def test_partition_canonical_order():
    assert _check(make_problem("p3", 2, 2, 0, seed=11)) == {"N", "C"}


@pytest.mark.parametrize("seed", [1, 2])
def test_partition_shuffled_order(seed):
    p = make_problem("p3", 1, 1, 0, seed=11 + seed)
    rng = np.random.default_rng(seed)
    _check(p.with_order(rng.permutation(p.n_sites)))


def test_partition_twelve_sites():
    p = make_problem("p", 2, 2, 0, seed=12)
    rng = np.random.default_rng(3)
    assert _check(p.with_order(rng.permutation(p.n_sites)), bonds=[0, 4, 5, 6, 9]) == {"N", "C"}


def test_term_count_pf_mid_bond():
    """Operator products at the pf mid bond: 2 + 2N + 2 K^2 - K with K = 20 at most."""
    p = make_problem("pf", 4, 4, 0, seed=2)
    mpo = MPO(ChainHamiltonian(p))
    n = mpo.n_terms(19)
    assert n <= 2 + 80 + 2 * 400 - 20
    assert n > 600
