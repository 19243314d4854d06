"""Input generator: PRNG, Clebsch-Gordan coefficients, m-scheme dimensions."""
import math

import numpy as np
import pytest

from gen import SplitMix64, cg, make_problem, mscheme_dimension, initial_mps


def test_splitmix_reference_values():
    # published SplitMix64 outputs for seed 1234567 (first three draws)
    r = SplitMix64(1234567)
    assert [r.next_u64() for _ in range(3)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_splitmix_bulk_equals_scalar():
    a, b = SplitMix64(99), SplitMix64(99)
    xs = [a.gauss() for _ in range(7)] + [a.uniform()]
    ys = list(b.gausses(7)) + [b.uniform()]
    assert xs == ys


@pytest.mark.parametrize("tj1,tj2", [(1, 1), (3, 1), (5, 3), (7, 7), (9, 5)])
def test_cg_orthonormal(tj1, tj2):
    """sum_{m1} <j1 m1 j2 M-m1|J M><j1 m1 j2 M-m1|J' M> = delta_JJ' (unitarity)."""
    for tM in range(-(tj1 + tj2), tj1 + tj2 + 1, 2):
        Js = [J for J in range(abs(tj1 - tj2), tj1 + tj2 + 1, 2) if J >= abs(tM)]
        for J in Js:
            for Jp in Js:
                s = sum(cg(tj1, m1, tj2, tM - m1, J, tM) * cg(tj1, m1, tj2, tM - m1, Jp, tM)
                        for m1 in range(-tj1, tj1 + 1, 2))
                assert abs(s - (1.0 if J == Jp else 0.0)) < 1e-13


@pytest.mark.parametrize("tj", [1, 3, 5, 7, 9])
def test_cg_closed_forms(tj):
    # <j m j -m|0 0> = (-1)^(j-m)/sqrt(2j+1)
    for tm in range(-tj, tj + 1, 2):
        assert abs(cg(tj, tm, tj, -tm, 0, 0) - (-1) ** ((tj - tm) // 2) / math.sqrt(tj + 1)) < 1e-14
    # stretched state
    assert abs(cg(tj, tj, 3, 3, tj + 3, tj + 3) - 1.0) < 1e-14
    # exchange symmetry <j1 m1 j2 m2|JM> = (-1)^(j1+j2-J) <j2 m2 j1 m1|JM>
    for J in range(abs(tj - 3), tj + 4, 2):
        for m1 in range(-tj, tj + 1, 2):
            for m2 in (-3, -1, 1, 3):
                ph = (-1) ** ((tj + 3 - J) // 2)
                assert abs(cg(tj, m1, 3, m2, J, m1 + m2) - ph * cg(3, m2, tj, m1, J, m1 + m2)) < 1e-14


def test_dimension_integers():
    # pf 8p+8n at J_z=0: "1.1 x 10^9" (56Ni in the pf shell)
    assert mscheme_dimension("pf", 8, 8, 0) == 1087455228
    assert mscheme_dimension("sd", 2, 2, 0) == 640
    assert mscheme_dimension("pf", 4, 4, 0) == 1963461
    # pf+g9/2 12p+12n, both parities (the paper's 1.7e14 counts positive parity only)
    assert mscheme_dimension("pfg", 12, 12, 0) == 345133964269907


def test_vbar_hermitian_and_conserving():
    p = make_problem("pf", 4, 4, 0, seed=2)
    d = {tuple(k): v for k, v in zip(p.v_idx.tolist(), p.v_val.tolist())}
    for (i, j, k, l), v in d.items():
        assert i < j and k < l
        assert d[(k, l, i, j)] == v
        qi = lambda s: (int(p.species[s] == 0), int(p.species[s] == 1), int(p.two_m[s]))
        a = tuple(x + y for x, y in zip(qi(i), qi(j)))
        b = tuple(x + y for x, y in zip(qi(k), qi(l)))
        assert a == b
        assert (p.l[i] + p.l[j]) % 2 == (p.l[k] + p.l[l]) % 2


def test_initial_mps_isometries():
    p = make_problem("sd", 2, 2, 0, seed=1)
    m = initial_mps(p, 16, 3)
    for Us in m.U:
        for U in Us:
            assert np.allclose(U.T @ U, np.eye(U.shape[1]), atol=1e-13)
    assert max(sum(x) for x in m.m) <= 16 + len(max(m.m, key=len))
