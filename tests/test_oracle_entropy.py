"""Pins of the oracle's dot-orbital density matrix and entropies.

At complete bases the DMRG wave function is the exact ground state, so the dot density
matrix must equal the one computed from the exact-diagonalization eigenvector in the
determinant basis (occupations, pair occupations and the hopping element
<c+_b c_a>, with the determinant signs of the site-index order, a convention independent
of the chain's Jordan-Wigner strings).  A chain order that puts orbitals of equal
(species, m) side by side makes the hopping element nonzero."""
import numpy as np
import pytest

from gen import make_problem, initial_mps
from oracle.dmrg import OracleDMRG
from oracle.entropy import dot_rdm, entropies
from oracle.hamiltonian import ed_sector


def _popcount(x):
    return bin(x).count("1")


def _rdm_from_determinants(basis, vec, a, b):
    """4 x 4 density matrix of sites a (first index bit) and b from a vector over
    determinants (bitmasks over site indices)."""
    index = {d: i for i, d in enumerate(basis)}
    rho = np.zeros((4, 4))
    x = 0.0
    for i, d in enumerate(basis):
        na, nb = (d >> a) & 1, (d >> b) & 1
        rho[2 * na + nb, 2 * na + nb] += vec[i] ** 2
        if na == 1 and nb == 0:         # <c+_b c_a>: remove a, then create b
            s = -1 if _popcount(d & ((1 << a) - 1)) & 1 else 1
            d1 = d ^ (1 << a)
            s = -s if _popcount(d1 & ((1 << b) - 1)) & 1 else s
            j = index.get(d1 | (1 << b))
            if j is not None:
                x += s * vec[j] * vec[i]
    rho[1, 2] = rho[2, 1] = x
    return rho


def _exact_run(prob, M0):
    basis, H = ed_sector(prob, prob.Np, prob.Nn, prob.two_Mz)
    w, V = np.linalg.eigh(H)
    o = OracleDMRG(prob, initial_mps(prob, M0, 5), tol=1e-11)
    o.sweep(10 ** 6)
    o.sweep(10 ** 6)
    return basis, V[:, 0], w, o


def _ordered_by_m(prob):
    """Chain order sorted by (species, 2m, orbital): equal (species, m) side by side."""
    keys = sorted(range(prob.n_sites),
                  key=lambda s: (int(prob.species[s]), int(prob.two_m[s]), int(prob.orbital[s])))
    return prob.with_order(keys)


@pytest.mark.parametrize("Np,Nn,two_M,seed,by_m", [(2, 2, 0, 12, False), (2, 1, 1, 3, True),
                                                   (2, 2, 4, 12, True)])
def test_dot_rdm_equals_exact_state(Np, Nn, two_M, seed, by_m):
    # hopping between equal-m orbitals of different j needs a state of nonzero J (a J = 0
    # state has a one-body density matrix diagonal in (j, m)): odd A, or 2M = 4
    prob = make_problem("p", Np, Nn, two_M, seed=seed)
    if by_m:
        prob = _ordered_by_m(prob)
    basis, v, w, o = _exact_run(prob, 6)
    assert w[1] - w[0] > 1e-3
    ch = o.ch
    hopping = 0
    for p in range(1, o.N - 2):
        o.run_step(p, "L", 10 ** 6)
        rho = dot_rdm(o.psi, o.psi_layout, o._prev_L, o._prev_R, ch.q[p], ch.q[p + 1])
        a, b = int(prob.order[p]), int(prob.order[p + 1])
        ref = _rdm_from_determinants(basis, v, a, b)
        assert np.max(np.abs(rho - ref)) < 1e-9, (p, rho, ref)
        assert abs(np.trace(rho) - 1.0) < 1e-12
        hopping += abs(ref[1, 2]) > 1e-6
        s_p, s_q, s_pq, I = entropies(rho)
        assert -1e-12 <= I <= 2 * np.log(2) + 1e-12 and s_pq <= s_p + s_q + 1e-12
    assert (hopping > 0) == by_m


def test_time_reversed_orbitals_have_equal_entropies():
    """A nondegenerate 2M = 0 eigenstate of a rotation- and time-reversal-invariant H has
    equal occupations of (species, j, m) and (species, j, -m): the one-orbital entropies
    gathered along a sweep come in equal pairs."""
    prob = make_problem("sd", 2, 2, 0, seed=1)
    o = OracleDMRG(prob, initial_mps(prob, 8, 5), tol=1e-11)
    o.sweep(400)
    s = {}
    for p in range(1, o.N - 2):
        o.run_step(p, "L", 400)
        rho = dot_rdm(o.psi, o.psi_layout, o._prev_L, o._prev_R, o.ch.q[p], o.ch.q[p + 1])
        sp, sq, _, _ = entropies(rho)
        s[int(prob.order[p])] = sp
        s[int(prob.order[p + 1])] = sq
    # positions 1..N-2 are dots at some step (the chain ends belong to one-site blocks)
    assert len(s) == prob.n_sites - 2
    pairs = 0
    for i in s:
        partner = [j for j in range(prob.n_sites)
                   if prob.species[j] == prob.species[i] and prob.orbital[j] == prob.orbital[i]
                   and prob.two_m[j] == -prob.two_m[i]]
        assert len(partner) == 1
        if partner[0] in s:
            assert abs(s[i] - s[partner[0]]) < 1e-8, (i, s[i], s[partner[0]])
            pairs += 1
    assert pairs >= prob.n_sites - 4
    assert max(s.values()) > 1e-3        # not a trivial (uncorrelated) state


@pytest.mark.parametrize("Np,Nn,two_M,seed,by_m,string_hops",
                         [(2, 2, 0, 12, False, False), (2, 1, 1, 3, False, True),
                          (2, 1, 1, 3, True, False)])
def test_every_pair_from_the_written_out_state(Np, Nn, two_M, seed, by_m, string_hops):
    """The DMRG state written out in the occupation basis (chain order) gives the density
    matrix of every orbital pair; at complete bases it equals the exact one, including the
    hopping element across Jordan-Wigner strings of any length."""
    from oracle.entropy import pair_rdm, state_amplitudes
    prob = make_problem("p", Np, Nn, two_M, seed=seed)
    if by_m:
        prob = _ordered_by_m(prob)
    basis, v, w, o = _exact_run(prob, 6)
    amp = state_amplitudes(o)
    assert abs(sum(a * a for a in amp.values()) - 1.0) < 1e-12
    assert len(amp) == len(basis)
    hop = 0.0
    for i in range(o.N):
        for j in range(i + 1, o.N):
            ref = _rdm_from_determinants(basis, v, int(prob.order[i]), int(prob.order[j]))
            assert np.max(np.abs(pair_rdm(amp, i, j) - ref)) < 1e-10, (i, j)
            hop = max(hop, abs(ref[1, 2]) if j > i + 1 else 0.0)
    # natural order: equal-m orbitals of different j lie apart, so a nonzero-J state hops
    # across Jordan-Wigner strings; ordered by m they are neighbours
    assert (hop > 1e-3) == string_hops


def test_written_out_state_at_truncated_m():
    """At truncated M the written-out state is normalised and its dot pair is the dot
    density matrix read off the two-site wave function, at every step of a half sweep (the
    blocks of the next bonds still hold the previous sweep's bases, which the expansion of
    the superblock at p must not read)."""
    from oracle.entropy import pair_rdm, state_amplitudes
    prob = make_problem("sd", 2, 2, 0, seed=1)
    o = OracleDMRG(prob, initial_mps(prob, 6, 5), tol=1e-10)
    o.sweep(6)
    for p in range(1, o.N - 2):
        o.run_step(p, "L", 8)
        amp = state_amplitudes(o)
        assert abs(sum(a * a for a in amp.values()) - 1.0) < 1e-12
        ref = dot_rdm(o.psi, o.psi_layout, o._prev_L, o._prev_R, o.ch.q[p], o.ch.q[p + 1])
        assert np.max(np.abs(pair_rdm(amp, p, p + 1) - ref)) < 1e-12


def test_mutual_information_dets_equals_pairwise_definition():
    """The vectorised all-pairs mutual information of a determinant-basis state equals the
    plain per-pair definition (pair_rdm) on the exact sd 2p+2n and odd p-shell ground
    states (natural chain order: site index = chain position)."""
    from oracle.entropy import mutual_information, mutual_information_dets
    for space, Np, Nn, tM, seed in (("sd", 2, 2, 0, 1), ("p", 2, 1, 1, 3)):
        p = make_problem(space, Np, Nn, tM, seed=seed)
        basis, H = ed_sector(p, Np, Nn, tM)
        w, V = np.linalg.eigh(H)
        v = V[:, 0]
        amp = {int(b): float(a) for b, a in zip(basis, v)}
        I_ref, s_ref = mutual_information(amp, p.n_sites)
        I, s = mutual_information_dets(np.array(basis, dtype=np.uint64), v, p.n_sites)
        assert np.max(np.abs(I - I_ref)) <= 1e-12
        assert np.max(np.abs(s - s_ref)) <= 1e-12
        assert np.max(I) > 0.0
