"""All-pairs orbital mutual information on the device (dmrg_mutual_information) against
the plain definition: the oracle's DMRG run through the same sweeps and the same
left-to-right half sweep, its two-site wave function at every step written out in the
occupation basis (oracle.entropy.state_amplitudes), and each pair's two-orbital density
matrix taken from the step that pairs it on the device (pair (i, j): the step with j at the
left dot; the pairs with the last two chain positions: the last step).  Davidson tolerance
1e-10 on both sides.

* p 2p+3n (2M = 1, odd A: hops between equal-m orbitals of different j), sd 2p+2n and sd
  2p+1n (2M = 3) at truncated M on shuffled chain orders: I_ij within 1e-7 of the oracle's
  for every pair, the one-orbital entropies s_i within 1e-7, the step energies within 1e-8.
* p 2p+2n at complete bases: the state is the exact ground state, so I and s equal the
  mutual information of the exact-diagonalization eigenvector (mutual_information_dets).
"""
import dataclasses

import numpy as np
import pytest

from gen import make_problem, initial_mps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_1507_00161_gb300.build import build
    build()
    import paper_1507_00161_gb300 as P
    assert torch.cuda.is_available()
    return P


def _problem(space, Np, Nn, tM, seed, shuffle):
    prob = make_problem(space, Np, Nn, tM, seed=seed)
    if shuffle:
        order = np.random.default_rng(seed).permutation(prob.n_sites).astype(np.int32)
        prob = dataclasses.replace(prob, order=order)
    return prob


def _oracle_half_sweep(prob, init, M, sweeps):
    from oracle.dmrg import OracleDMRG
    from oracle.entropy import entropies, mutual_information, pair_rdm, state_amplitudes
    o = OracleDMRG(prob, init, tol=1e-10)
    for _ in range(sweeps):
        o.sweep(M)
    N = prob.n_sites
    I = np.zeros((N, N))
    s = None
    energies = []
    for p in range(1, N - 2):
        energies.append(o.run_step(p, "L", M).energy)
        amp = state_amplitudes(o)
        pairs = [(i, p) for i in range(p)]
        if p == N - 3:
            pairs += [(i, N - 2) for i in range(N - 2)] + [(i, N - 1) for i in range(N - 1)]
            _, s = mutual_information(amp, N)
        for i, j in pairs:
            I[i, j] = I[j, i] = entropies(pair_rdm(amp, i, j))[3]
    # chain positions -> the problem's sites
    order = np.asarray(prob.order)
    I_site = np.zeros_like(I)
    I_site[np.ix_(order, order)] = I
    s_site = np.zeros(N)
    s_site[order] = s
    return I_site, s_site, energies


@pytest.mark.parametrize("space,Np,Nn,tM,seed,M,shuffle", [
    ("p", 2, 3, 1, 7, 16, True), ("sd", 2, 2, 0, 1, 32, True), ("sd", 2, 1, 3, 4, 24, False)])
def test_mutual_information_equals_the_written_out_states(P, space, Np, Nn, tM, seed, M,
                                                          shuffle):
    prob = _problem(space, Np, Nn, tM, seed, shuffle)
    init = initial_mps(prob, M, seed + 5)
    I_ref, s_ref, e_ref = _oracle_half_sweep(prob, init, M, 1)
    d = P.DMRG(prob, dav_tol=1e-10)
    d.build_blocks(init)
    d.sweep(M)
    I, s, steps = d.mutual_information(M)
    d.close()
    assert np.max(np.abs([st["energy"] - e for st, e in zip(steps, e_ref)])) <= 1e-8
    assert np.allclose(I, I.T) and np.all(np.diag(I) == 0.0)
    assert np.max(np.abs(I - I_ref)) <= 1e-7, np.max(np.abs(I - I_ref))
    assert np.max(np.abs(s - s_ref)) <= 1e-7
    assert I.max() > 1e-3


@pytest.mark.parametrize("seed", [3, 1])
def test_mutual_information_at_complete_bases_is_exact(P, seed):
    """Seed 3: a J >= 1 ground state (its M = 0 member); seed 1: a J = 0 ground state, whose
    one-orbital entropies are equal over the m-substates of each j-shell (the paper's
    observation for the J = 0 states)."""
    from oracle.entropy import mutual_information_dets
    from oracle.hamiltonian import ed_sector
    prob = _problem("p", 2, 2, 0, seed, True)
    basis, H = ed_sector(prob, 2, 2, 0)
    w, V = np.linalg.eigh(H)
    I_ex, s_ex = mutual_information_dets(np.array(basis, dtype=np.uint64), V[:, 0],
                                         prob.n_sites)
    d = P.DMRG(prob, dav_tol=1e-11)
    d.build_blocks(initial_mps(prob, 10 ** 6, 8))
    d.sweep(10 ** 6)
    I, s, steps = d.mutual_information(10 ** 6)
    d.close()
    assert abs(steps[-1]["energy"] - w[0]) <= 1e-9
    assert np.max(np.abs(I - I_ex)) <= 1e-8
    assert np.max(np.abs(s - s_ex)) <= 1e-8
    if seed == 1:
        _, H2 = ed_sector(prob, 2, 2, 2)
        assert np.linalg.eigvalsh(H2)[0] > w[0] + 1.0      # no M = 1 state at E0: J = 0
        for sp in (0, 1):
            for orb in set(int(x) for x in prob.orbital):
                sel = (np.asarray(prob.species) == sp) & (np.asarray(prob.orbital) == orb)
                assert np.ptp(s[sel]) <= 1e-8, (sp, orb, s[sel])


def test_mutual_information_arguments(P):
    prob = make_problem("p", 2, 2, 0, seed=3)
    d = P.DMRG(prob)
    with pytest.raises(P.DmrgError):
        d.mutual_information(8)          # blocks not built
    d.build_blocks(initial_mps(prob, 8, 1))
    with pytest.raises(P.DmrgError):
        d.mutual_information(0)
    d.close()
