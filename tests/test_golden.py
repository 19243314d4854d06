"""Values the paper prints, checked against counts made here: the m-scheme dimensions of
tests/golden/paper_dimensions.txt.  The count is a dynamic program over the single-particle
states of the valence space (occupied or empty), independent of the sector tables of the
generator, and is cross-checked against them for both parities together."""
import os
from collections import defaultdict

import pytest

from gen.shell import SPACES, mscheme_dimension, site_table

HERE = os.path.dirname(os.path.abspath(__file__))


def _fixtures():
    rows = []
    for line in open(os.path.join(HERE, "golden", "paper_dimensions.txt")):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            rows.append((f[0], int(f[1]), int(f[2]), int(f[3]), f[4], f[5]))
    return rows


def _count(space, Np, Nn, two_M):
    """Determinants with Np protons, Nn neutrons and 2M = two_M, by parity (0 = +)."""
    d = defaultdict(int)
    d[(0, 0, 0, 0)] = 1
    for s in site_table(SPACES[space]):
        nd = defaultdict(int)
        for (a, b, m, par), c in d.items():
            nd[(a, b, m, par)] += c
            a2, b2 = a + (s["species"] == 0), b + (s["species"] == 1)
            if a2 <= Np and b2 <= Nn:
                nd[(a2, b2, m + s["two_m"], par ^ (s["l"] & 1))] += c
        d = nd
    return d[(Np, Nn, two_M, 0)], d[(Np, Nn, two_M, 1)]


def _round_sig(x, printed):
    mant = printed.lower().split("e")[0]
    sig = len(mant.replace(".", "").lstrip("0"))
    return float(f"{x:.{sig - 1}e}")


@pytest.mark.parametrize("row", _fixtures(), ids=lambda r: f"{r[0]}-{r[1]}p{r[2]}n")
def test_printed_mscheme_dimensions(row):
    space, Np, Nn, two_M, parity, printed = row
    pos, neg = _count(space, Np, Nn, two_M)
    assert pos + neg == mscheme_dimension(space, Np, Nn, two_M)
    n = pos + neg if parity == "both" else pos
    assert _round_sig(n, printed) == float(printed), (n, printed)
