"""The library's orbital ordering (host code behind the C-ABI, no GPU needed) against the
oracle's: seeded weight matrices, a hidden chain, the path graph, mutual information of
an exact shell-model ground state, and the rejected inputs."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def P():
    from paper_1507_00161_gb300.build import build
    build()
    import paper_1507_00161_gb300 as P
    return P


def _separated(v, tol=1e-8):
    s = np.sort(v)
    return np.min(np.diff(s)) > tol


@pytest.mark.parametrize("seed", range(8))
def test_random_weights_match_oracle(P, seed):
    from oracle.ordering import fiedler_order, fiedler_vector, laplacian
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 41))
    A = rng.random((n, n)) ** 3
    I = A + A.T
    w = np.linalg.eigvalsh(laplacian(I))
    assert w[2] - w[1] > 1e-8 * w[-1]          # unique Fiedler vector
    v_ref = fiedler_vector(I)
    assert _separated(v_ref)
    order, v = P.fiedler_order(I)
    assert np.max(np.abs(v - v_ref)) < 1e-10
    assert order == fiedler_order(I)


def test_hidden_chain_and_path(P):
    rng = np.random.default_rng(3)
    n = 40
    hidden = rng.permutation(n)
    pos = np.empty(n, dtype=int)
    pos[hidden] = np.arange(n)
    I = np.exp(-0.5 * np.abs(pos[:, None] - pos[None, :]).astype(float))
    order, _ = P.fiedler_order(I)
    assert order == list(hidden) or order == list(hidden[::-1])
    path = np.diag(np.ones(9), 1) + np.diag(np.ones(9), -1)
    assert P.fiedler_order(path)[0] == list(range(10))[::-1]


def test_exact_ground_state_mutual_information(P):
    """All-pairs mutual information of the exact ground state of p-shell 2p+2n (from the
    determinant basis), ordered by the library and by the oracle."""
    from gen import make_problem
    from oracle.entropy import entropies
    from oracle.hamiltonian import ed_sector
    from oracle.ordering import fiedler_order
    from test_oracle_entropy import _rdm_from_determinants
    prob = make_problem("p", 2, 2, 0, seed=12)
    basis, H = ed_sector(prob, 2, 2, 0)
    v = np.linalg.eigh(H)[1][:, 0]
    n = prob.n_sites
    I = np.zeros((n, n))
    for a in range(n):
        for b in range(a + 1, n):
            I[a, b] = I[b, a] = entropies(_rdm_from_determinants(basis, v, a, b))[3]
    assert I.min() >= -1e-12 and I.max() > 1e-3
    order, vec = P.fiedler_order(I)
    from oracle.ordering import fiedler_vector
    if _separated(fiedler_vector(I)):
        assert order == fiedler_order(I)
    assert np.max(np.abs(vec - fiedler_vector(I))) < 1e-9


def test_rejected_inputs(P):
    good = np.ones((4, 4))
    bad = [np.ones((1, 1)), np.array([[0, 1, 2], [1, 0, 1], [1, 1, 0]], float),
           np.array([[0, -1, 1], [-1, 0, 1], [1, 1, 0]], float),
           np.array([[0, np.nan, 1], [np.nan, 0, 1], [1, 1, 0]]),
           np.array([[0, 1, 0, 0], [1, 0, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], float)]
    P.fiedler_order(good)
    for I in bad:
        with pytest.raises(P.DmrgError) as e:
            P.fiedler_order(I)
        assert e.value.code == P.DMRG_EINVAL


def test_ordering_of_a_dmrg_state(P):
    """The preprocessing chain on a small case: mutual information of every pair from a
    DMRG state (oracle), ordered by the library; the order found shortens the
    entanglement distance of the natural chain order."""
    from gen import make_problem, initial_mps
    from oracle.dmrg import OracleDMRG
    from oracle.entropy import mutual_information, state_amplitudes
    from oracle.ordering import entanglement_distance, fiedler_order, fiedler_vector
    prob = make_problem("p", 3, 3, 0, seed=5)
    o = OracleDMRG(prob, initial_mps(prob, 8, 5), tol=1e-10)
    o.sweep(10 ** 6)
    I, s = mutual_information(state_amplitudes(o), o.N)
    order, vec = P.fiedler_order(I)
    assert np.max(np.abs(vec - fiedler_vector(I))) < 1e-9
    if _separated(fiedler_vector(I)):
        assert order == fiedler_order(I)
    d_nat = entanglement_distance(I, list(range(o.N)))
    assert entanglement_distance(I, order) < 0.5 * d_nat
