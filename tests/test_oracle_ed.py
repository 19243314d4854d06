"""Pins of the oracle's Eq. (1) Hamiltonian and exact diagonalization."""
import numpy as np
import pytest

from gen.shell import SPACES, draw_tbre, make_problem, pairing_problem, problem_from_j, _like_pairs, _pn_pairs
from oracle.hamiltonian import ed_sector, ed_lowest


def _two_body_spectrum(space_name, seed, channel):
    """Eigenvalues of two particles from the J-scheme: union over J of
    eig(V_J + diag(eps_a + eps_b)) over the allowed pairs (each J once at 2M = 0)."""
    space = SPACES[space_name]
    eps, vpp, vpn = draw_tbre(space, seed)
    V, pairs_of = (vpp, _like_pairs) if channel == "pp" else (vpn, _pn_pairs)
    out = []
    jmax2 = 2 * max(o.two_j for o in space.orbitals)
    for tJ in range(0, jmax2 + 1, 2):
        pairs = pairs_of(space, tJ)
        if not pairs:
            continue
        A = np.zeros((len(pairs), len(pairs)))
        for x, (a, b) in enumerate(pairs):
            A[x, x] += eps[a] + eps[b]
            for y, (c, d) in enumerate(pairs):
                A[x, y] += V.get((tJ, a, b, c, d), 0.0)
        out.extend(np.linalg.eigvalsh(A))
    return np.sort(np.array(out))


@pytest.mark.parametrize("space", ["sd", "p", "pf"])
def test_two_like_particles_spectrum(space):
    p = make_problem(space, 2, 0, 0, seed=5)
    _, H = ed_sector(p, 2, 0, 0)
    w = np.linalg.eigvalsh(H)
    ref = _two_body_spectrum(space, 5, "pp")
    assert w.shape == ref.shape
    assert np.max(np.abs(w - ref)) < 1e-12
    # the neutron copy of the same draw
    _, Hn = ed_sector(p, 0, 2, 0)
    assert np.max(np.abs(np.linalg.eigvalsh(Hn) - ref)) < 1e-12


@pytest.mark.parametrize("space", ["sd", "p"])
def test_proton_neutron_spectrum(space):
    p = make_problem(space, 1, 1, 0, seed=6)
    _, H = ed_sector(p, 1, 1, 0)
    w = np.linalg.eigvalsh(H)
    ref = _two_body_spectrum(space, 6, "pn")
    assert w.shape == ref.shape
    assert np.max(np.abs(w - ref)) < 1e-12


@pytest.mark.parametrize("npairs", [1, 2, 3, 4])
def test_seniority_closed_form(npairs):
    """Single j = 7/2 shell, V_{J=0} = -G Omega: H = -G S+S, ground state
    E = -G n (Omega - n + 1) with Omega = 4 (Talmi / Racah seniority)."""
    G = 0.7
    omega = 4
    E = -G * npairs * (omega - npairs + 1)
    p = pairing_problem("f7", G, 2 * npairs, 0)
    assert abs(ed_lowest(p)[0] - E) < 1e-12
    p = pairing_problem("f7", G, 0, 2 * npairs)
    assert abs(ed_lowest(p)[0] - E) < 1e-12


def test_one_body_closed_form():
    eps = [1.0, 0.3, 2.0]          # d5/2, s1/2, d3/2
    p = problem_from_j("sd", eps, {}, {}, 3, 3, 0)
    # per species: s1/2 filled (2 x 0.3) plus one particle in d5/2
    assert abs(ed_lowest(p)[0] - 2 * (2 * 0.3 + 1.0)) < 1e-13


def test_j_multiplets_contained():
    """Rotational invariance: every level at 2M = 4 (J >= 2) and 2M = 2 reappears at 2M = 0."""
    p = make_problem("p", 2, 2, 0, seed=8)
    w0 = np.linalg.eigvalsh(ed_sector(p, 2, 2, 0)[1])
    for tM in (2, 4):
        w = np.linalg.eigvalsh(ed_sector(p, 2, 2, tM)[1])
        for x in w:
            assert np.min(np.abs(w0 - x)) < 1e-10
    p = make_problem("sd", 2, 1, 1, seed=9)
    w1 = np.linalg.eigvalsh(ed_sector(p, 2, 1, 1)[1])
    w5 = np.linalg.eigvalsh(ed_sector(p, 2, 1, 5)[1])
    for x in w5:
        assert np.min(np.abs(w1 - x)) < 1e-10


def test_hamiltonian_symmetric():
    p = make_problem("sd", 2, 2, 0, seed=1)
    _, H = ed_sector(p, 2, 2, 0)
    assert H.shape == (640, 640)
    assert np.array_equal(H, H.T)
