"""Pins of the oracle's matrix-free Lanczos (oracle/lanczos.c), which gives the exact
energy of sectors too large for a dense matrix (the pf 4p+4n space).  Each pin compares
it with something it shares no code with: the dense Python matrix, textbook closed
forms, rotational invariance and the generator's dimension count."""
import numpy as np
import pytest

from gen.shell import make_problem, mscheme_dimension, pairing_problem, problem_from_j
from oracle.hamiltonian import (ed_lowest, ed_sector, lanczos_lowest, mscheme_apply,
                                mscheme_basis, mscheme_dim)


def _dense_in_lanczos_order(p, Np, Nn, tM):
    basis, H = ed_sector(p, Np, Nn, tM)
    idx = {b: i for i, b in enumerate(basis)}
    perm = np.array([idx[int(m)] for m in mscheme_basis(p, Np, Nn, tM)])
    return H[np.ix_(perm, perm)]


@pytest.mark.parametrize("space,Np,Nn,tM,seed", [("sd", 2, 2, 0, 1), ("sd", 3, 2, 1, 4),
                                                  ("p", 2, 3, 3, 7), ("sd", 0, 3, 1, 2)])
def test_product_equals_dense_matrix(space, Np, Nn, tM, seed):
    """y = H x of the C code = the dense matrix of ed_sector (same determinants)."""
    p = make_problem(space, Np, Nn, tM, seed=seed)
    H = _dense_in_lanczos_order(p, Np, Nn, tM)
    x = np.random.default_rng(seed).standard_normal(H.shape[0])
    y = mscheme_apply(p, x, threads=3)
    assert np.max(np.abs(H @ x - y)) <= 1e-12 * np.max(np.abs(H @ x))


@pytest.mark.parametrize("space,Np,Nn,tM,seed", [("sd", 2, 2, 0, 1), ("sd", 3, 2, 1, 4),
                                                  ("p", 2, 2, 0, 8), ("sd", 2, 2, 4, 1),
                                                  ("pfg", 1, 1, 4, 5)])
def test_lowest_equals_dense_eigh(space, Np, Nn, tM, seed):
    p = make_problem(space, Np, Nn, tM, seed=seed)
    r = lanczos_lowest(p, Np, Nn, tM, tol=1e-10, threads=2, want_vector=True)
    e = ed_lowest(p, Np, Nn, tM)[0]
    assert abs(r["energy"] - e) <= 1e-10
    assert r["residual"] <= 1e-9
    assert abs(np.linalg.norm(r["vector"]) - 1.0) <= 1e-12
    H = _dense_in_lanczos_order(p, Np, Nn, tM)
    v = r["vector"]
    assert abs(v @ H @ v - e) <= 1e-10


@pytest.mark.parametrize("npairs", [1, 2, 3, 4])
def test_seniority_closed_form(npairs):
    """Single j = 7/2 shell with only V_{J=0} = -G Omega: the seniority-zero ground state
    has E = -G n (Omega - n + 1), Omega = 4 (Talmi / Racah)."""
    G = 0.7
    E = -G * npairs * (4 - npairs + 1)
    for Np, Nn in ((2 * npairs, 0), (0, 2 * npairs)):
        r = lanczos_lowest(pairing_problem("f7", G, Np, Nn), tol=1e-11, threads=1)
        assert abs(r["energy"] - E) <= 1e-10


def test_one_body_closed_form():
    eps = [1.0, 0.3, 2.0]          # d5/2, s1/2, d3/2
    p = problem_from_j("sd", eps, {}, {}, 3, 3, 0)
    r = lanczos_lowest(p, tol=1e-11, threads=1)
    assert abs(r["energy"] - 2 * (2 * 0.3 + 1.0)) <= 1e-10


def test_rotational_invariance():
    """The lowest 2M = 4 level (J >= 2) lies at or above the lowest 2M = 0 level and is
    one of the 2M = 0 levels (multiplet containment)."""
    p = make_problem("sd", 2, 2, 0, seed=3)
    e0 = lanczos_lowest(p, 2, 2, 0, tol=1e-10, threads=2)["energy"]
    e4 = lanczos_lowest(p, 2, 2, 4, tol=1e-10, threads=2)["energy"]
    w0 = np.linalg.eigvalsh(ed_sector(p, 2, 2, 0)[1])
    assert e4 >= e0 - 1e-10
    assert np.min(np.abs(w0 - e4)) <= 1e-9


@pytest.mark.parametrize("space,Np,Nn,tM", [("sd", 2, 2, 0), ("pf", 4, 4, 0), ("pf", 8, 8, 0),
                                             ("sd", 3, 2, 1)])
def test_dimension_equals_generator_count(space, Np, Nn, tM):
    p = make_problem(space, Np, Nn, tM, seed=1)
    assert mscheme_dim(p) == mscheme_dimension(space, Np, Nn, tM)


def test_rejects_non_hermitian_list():
    p = make_problem("sd", 2, 2, 0, seed=1)
    vv = p.v_val.copy()
    t = next(x for x, (i, j, k, l) in enumerate(p.v_idx.tolist()) if (i, j) != (k, l))
    vv[t] += 1.0
    import dataclasses
    q = dataclasses.replace(p, v_val=vv)
    with pytest.raises(ValueError):
        lanczos_lowest(q)


def test_stored_pfg_sweep_is_variational():
    """The stored oracle sweep on the pf+g9/2 space (tests/golden/pfg_2p2n_M4.json: 2p+2n,
    2M_z = 4, M = 16) lies above the exact energy of that sector (Lanczos, dimension 15,372)
    at every step, and the exact 2M_z = 4 energy lies above the 2M_z = 0 one (rotational
    invariance: the M_z = 2 states are the J >= 2 states of the M_z = 0 spectrum)."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "pfg_2p2n_M4.json")
    with open(path) as f:
        g = json.load(f)
    p4 = make_problem("pfg", 2, 2, 4, seed=5)
    r4 = lanczos_lowest(p4, tol=1e-10, threads=2)
    assert r4["dim"] == 15372 == mscheme_dimension("pfg", 2, 2, 4)
    assert r4["residual"] <= 1e-9
    for st in g["steps"]:
        assert st["energy"] >= r4["energy"] - 1e-9, (st["p"], st["dir"])
    r0 = lanczos_lowest(make_problem("pfg", 2, 2, 0, seed=5), tol=1e-10, threads=2)
    assert r4["energy"] >= r0["energy"] - 1e-9
