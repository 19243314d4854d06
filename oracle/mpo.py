"""Oracle: the partition of H into left-block and right-block operator products at every
bond, with normal and complementary operators (two-site superblock of Section "In the
two-site DMRG variant ... Xi_l (x) Lambda_{i+1} (x) Lambda_{i+2} (x) Xi_r"; the operator
algebra is not spelled out in the paper and follows the quantum-chemistry DMRG it cites).

TEST INFRASTRUCTURE ONLY.

Bond b lies between chain positions b and b+1: left sites Lb = {0..b}, right Rb =
{b+1..N-1}.  With the antisymmetrised W (two-body part 1/4 sum W_ijkl c+_i c+_j c_l c_k),
every term of H splits as (operator on Lb) x (operator on Rb), fermionic order left then
right:

    H = H^L 1 + 1 H^R
      + sum_{i in L} [ c+_i S^R_i - c_i (S^R_i)^+ ]          S^R_i = 1/2 sum_{jkl in R} W_ijkl c+_j c_l c_k
      + sum_{j in R} [ S^L_j c+_j - (S^L_j)^+ c_j ]          S^L_j = 1/2 sum_{ikl in L} W_ijkl c+_i c_l c_k
      + pair terms, written with normal operators on the side with fewer sites:
        normal left  (|L| <= |R|):  sum_{i<j in L} [A_ij P^R_ij + A_ij^+ P^R_ij^+] + sum_{i,k in L} B_ik Q^R_ik
        complementary left:         sum_{k<l in R} [P^L_kl c_l c_k + P^L_kl^+ c+_k c+_l] + sum_{j,l in R} Q^L_jl c+_j c_l
      A_ij = c+_i c+_j, B_ik = c+_i c_k,  P^L_kl = sum_{i<j in L} W_ijkl c+_i c+_j,
      Q^L_jl = sum_{i,k in L} W_ijkl c+_i c_k.

The left operators of bond s follow from those of bond s-1 and the site-s operators
{1, n, c+, c} (``W[s]``: entries (a, b, site_op, coef), meaning left_b += left_a . op),
which is a matrix-product operator; the right operators of bond s-1 are
right_a = sum_b W[s][a,b] op . right_b with the same entries, and H = sum_k L_k R_k at
every bond.  Labels that are structurally zero (unreachable from the vacuum identity or
not reaching the final H) are removed.
"""
from __future__ import annotations

from typing import Dict, List, Tuple

OPS = {"I": (0, 0), "N": (0, 0), "Cd": (1, 0), "C": (-1, 1)}
# site operator -> (sigma_out, sigma_in) of its single nonzero entry(ies), parity
SITE_ENTRIES = {"I": [(0, 0), (1, 1)], "N": [(1, 1)], "Cd": [(1, 0)], "C": [(0, 1)]}
SITE_PARITY = {"I": 0, "N": 0, "Cd": 1, "C": 1}


def mode(b: int, N: int) -> str:
    """'N' (normal pair operators on the left) when the left has no more sites."""
    return "N" if (b + 1) <= (N - b - 1) else "C"


def _labels(b: int, N: int):
    L = list(range(0, b + 1))
    R = list(range(b + 1, N))
    out = [("I",), ("H",)]
    out += [("Cd", i) for i in L] + [("C", i) for i in L]
    out += [("S", j) for j in R] + [("Sd", j) for j in R]
    if mode(b, N) == "N":
        out += [("A", i, j) for i in L for j in L if i < j]
        out += [("Ad", i, j) for i in L for j in L if i < j]
        out += [("B", i, k) for i in L for k in L]
    else:
        out += [("P", k, l) for k in R for l in R if k < l]
        out += [("Pd", k, l) for k in R for l in R if k < l]
        out += [("Q", j, l) for j in R for l in R]
    return out


def label_parity(lab) -> int:
    return 1 if lab[0] in ("Cd", "C", "S", "Sd") else 0


def label_dq(lab, q) -> tuple:
    """Quantum-number change the left operator applies to a left ket."""
    z = (0, 0, 0)
    add = lambda a, b: (a[0] + b[0], a[1] + b[1], a[2] + b[2])
    neg = lambda a: (-a[0], -a[1], -a[2])
    t = lab[0]
    if t in ("I", "H"):
        return z
    if t == "Cd":
        return q[lab[1]]
    if t == "C":
        return neg(q[lab[1]])
    if t == "S":
        return neg(q[lab[1]])
    if t == "Sd":
        return q[lab[1]]
    if t == "A":
        return add(q[lab[1]], q[lab[2]])
    if t == "Ad":
        return neg(add(q[lab[1]], q[lab[2]]))
    if t == "B":
        return add(q[lab[1]], neg(q[lab[2]]))
    if t == "P":
        return add(q[lab[1]], q[lab[2]])
    if t == "Pd":
        return neg(add(q[lab[1]], q[lab[2]]))
    if t == "Q":
        return add(q[lab[2]], neg(q[lab[1]]))
    raise ValueError(lab)


def _site_entries(s: int, ch, prev: List[tuple], cur: List[tuple]):
    """Entries (a_label, b_label, op, coef) of W[s]: left_b(s) += left_a(s-1) . op_s."""
    N = ch.N
    W = ch.W
    Lp = list(range(0, s))          # left sites at bond s-1
    mprev = mode(s - 1, N)
    mcur = mode(s, N)
    prevset = set(prev)
    E = []

    def add(a, b, op, c):
        if c != 0.0 and a in prevset:
            E.append((a, b, op, c))

    for lab in cur:
        t = lab[0]
        if t == "I":
            add(("I",), lab, "I", 1.0)
        elif t == "H":
            add(("H",), lab, "I", 1.0)
            add(("I",), lab, "N", float(ch.eps[s]))
            add(("S", s), lab, "Cd", 1.0)
            add(("Sd", s), lab, "C", -1.0)
            if mprev == "N":
                for i in Lp:
                    for k in Lp:
                        add(("B", i, k), lab, "N", W(i, s, k, s))
            else:
                add(("Q", s, s), lab, "N", 1.0)
        elif t in ("Cd", "C"):
            i = lab[1]
            if i < s:
                add(lab, lab, "I", 1.0)
            else:
                add(("I",), lab, t, 1.0)
        elif t == "S":
            j = lab[1]
            add(lab, lab, "I", 1.0)
            if mprev == "N":
                for k in Lp:
                    for l in Lp:
                        if k < l:
                            add(("Ad", k, l), lab, "Cd", W(s, j, k, l))
                for i in Lp:
                    for k in Lp:
                        add(("B", i, k), lab, "C", -W(i, j, k, s))
            else:
                add(("Pd", s, j), lab, "Cd", 1.0)
                add(("Q", j, s), lab, "C", -1.0)
            for k in Lp:
                add(("C", k), lab, "N", W(s, j, k, s))
        elif t == "Sd":
            j = lab[1]
            add(lab, lab, "I", 1.0)
            if mprev == "N":
                for k in Lp:
                    for l in Lp:
                        if k < l:
                            add(("A", k, l), lab, "C", W(s, j, k, l))
                for x in Lp:
                    for y in Lp:       # label B_xy = c+_x c_y  with coefficient -W(y,j,x,s)
                        add(("B", x, y), lab, "Cd", -W(y, j, x, s))
            else:
                add(("P", s, j), lab, "C", 1.0)
                add(("Q", s, j), lab, "Cd", -1.0)
            for k in Lp:
                add(("Cd", k), lab, "N", W(s, j, k, s))
        elif t in ("A", "Ad"):
            i, j = lab[1], lab[2]
            if j < s:
                add(lab, lab, "I", 1.0)
            elif t == "A":
                add(("Cd", i), lab, "Cd", 1.0)
            else:
                add(("C", i), lab, "C", -1.0)
        elif t == "B":
            i, k = lab[1], lab[2]
            if i < s and k < s:
                add(lab, lab, "I", 1.0)
            elif i == s and k < s:
                add(("C", k), lab, "Cd", -1.0)
            elif k == s and i < s:
                add(("Cd", i), lab, "C", 1.0)
            else:
                add(("I",), lab, "N", 1.0)
        elif t in ("P", "Pd"):
            k, l = lab[1], lab[2]
            if mprev == "N":
                src = "A" if t == "P" else "Ad"
                for i in Lp:
                    for j in Lp:
                        if i < j:
                            add((src, i, j), lab, "I", W(i, j, k, l))
            else:
                add(lab, lab, "I", 1.0)
            for i in Lp:
                if t == "P":
                    add(("Cd", i), lab, "Cd", W(i, s, k, l))
                else:
                    add(("C", i), lab, "C", -W(i, s, k, l))
        elif t == "Q":
            j, l = lab[1], lab[2]
            if mprev == "N":
                for i in Lp:
                    for k in Lp:
                        add(("B", i, k), lab, "I", W(i, j, k, l))
            else:
                add(lab, lab, "I", 1.0)
            for k in Lp:
                add(("C", k), lab, "Cd", -W(s, j, k, l))
            for i in Lp:
                add(("Cd", i), lab, "C", W(i, j, s, l))
            add(("I",), lab, "N", W(s, j, s, l))
        else:
            raise ValueError(lab)
    return E


class MPO:
    """labels[b] for b = -1..N-1 (index b+1) and W[s] entries as integer label indices:
    (a_idx at bond s-1, b_idx at bond s, op, coef)."""

    def __init__(self, ch):
        N = ch.N
        self.N = N
        raw_labels = [[("I",)]] + [_labels(b, N) for b in range(N)]
        raw_labels[N] = [("H",)]                       # only the full H survives at the end
        raw_W = []
        for s in range(N):
            raw_W.append(_site_entries(s, ch, raw_labels[s], raw_labels[s + 1]))
        # prune: forward reachability from the vacuum identity, backward from H
        alive_f = [set([("I",)])]
        for s in range(N):
            nxt = set(b for (a, b, op, c) in raw_W[s] if a in alive_f[s])
            alive_f.append(nxt)
        alive_b = [None] * (N + 1)
        alive_b[N] = set([("H",)])
        for s in range(N - 1, -1, -1):
            alive_b[s] = set(a for (a, b, op, c) in raw_W[s] if b in alive_b[s + 1])
        self.labels = []
        for b in range(N + 1):
            keep = alive_f[b] & alive_b[b]
            self.labels.append([lab for lab in raw_labels[b] if lab in keep])
        self.index = [{lab: x for x, lab in enumerate(ls)} for ls in self.labels]
        self.W = []
        for s in range(N):
            ia, ib = self.index[s], self.index[s + 1]
            self.W.append([(ia[a], ib[b], op, c) for (a, b, op, c) in raw_W[s]
                           if a in ia and b in ib])
        self.parity = [[label_parity(l) for l in ls] for ls in self.labels]
        self.dq = [[label_dq(l, ch.q) for l in ls] for ls in self.labels]
        # consistency: every entry carries the quantum numbers and parity of its labels
        for s in range(N):
            qs = ch.q[s]
            for (a, b, op, c) in self.W[s]:
                dop = {"I": (0, 0, 0), "N": (0, 0, 0), "Cd": qs,
                       "C": (-qs[0], -qs[1], -qs[2])}[op]
                da, db = self.dq[s][a], self.dq[s + 1][b]
                assert (da[0] + dop[0], da[1] + dop[1], da[2] + dop[2]) == db, (s, a, b, op)
                assert (self.parity[s][a] + SITE_PARITY[op]) % 2 == self.parity[s + 1][b]

    def n_terms(self, b: int) -> int:
        """Number of operator products L_k R_k at bond b (b = 0..N-2)."""
        return len(self.labels[b + 1])
