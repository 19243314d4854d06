"""Oracle: the shell-model Hamiltonian of Eq. (1) and its exact diagonalization.

TEST INFRASTRUCTURE ONLY -- imported by tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg; never by the product path.

H = sum_i eps_i n_i + sum_{i<j,k<l} Vbar[ij,kl] c+_i c+_j c_l c_k     (Eq. 1, with the
antisymmetrised matrix elements of the input convention), on occupation-number states of
m-scheme orbitals (the C^2 representation: each orbital empty or occupied).

* ``ed_sector``: the m-scheme determinant basis of fixed (N_p, N_n, 2M) and the dense
  matrix of H in it, by applying every term to every determinant with the
  fermionic sign (-1)^(number of occupied orbitals before the acted-on one).
* ``fock_matrix``: H on the whole Fock space of a tiny system from Jordan-Wigner
  matrices, c_i = Z x .. x Z x a x 1 x .. x 1 (sites in chain order).
* ``ChainHamiltonian``: the same H with site indices replaced by chain positions
  (position c holds site order[c]); pairs are re-sorted with the sign of the swap.
"""
from __future__ import annotations

import itertools
from typing import Dict, List, Tuple

import numpy as np
import scipy.sparse as sp


def _popcount(x: int) -> int:
    return bin(x).count("1")


def _apply_term(state: int, i: int, j: int, k: int, l: int):
    """c+_i c+_j c_l c_k |state>: returns (sign, new_state) or None."""
    s = state
    sign = 1
    for op, x in (("a", k), ("a", l), ("c", j), ("c", i)):
        bit = 1 << x
        if op == "a":
            if not (s & bit):
                return None
            if _popcount(s & (bit - 1)) & 1:
                sign = -sign
            s ^= bit
        else:
            if s & bit:
                return None
            if _popcount(s & (bit - 1)) & 1:
                sign = -sign
            s |= bit
    return sign, s


def sector_basis(prob, Np: int, Nn: int, two_M: int) -> List[int]:
    """All determinants (bitmasks over canonical site indices) of the sector, sorted."""
    N = prob.n_sites
    p_sites = [s for s in range(N) if prob.species[s] == 0]
    n_sites = [s for s in range(N) if prob.species[s] == 1]
    out = []
    for pc in itertools.combinations(p_sites, Np):
        mp = sum(int(prob.two_m[s]) for s in pc)
        maskp = sum(1 << s for s in pc)
        for nc in itertools.combinations(n_sites, Nn):
            if mp + sum(int(prob.two_m[s]) for s in nc) == two_M:
                out.append(maskp | sum(1 << s for s in nc))
    out.sort()
    return out


def ed_sector(prob, Np: int, Nn: int, two_M: int):
    """Dense H in the m-scheme sector; returns (basis, H)."""
    basis = sector_basis(prob, Np, Nn, two_M)
    index = {b: x for x, b in enumerate(basis)}
    by_kl: Dict[Tuple[int, int], List[Tuple[int, int, float]]] = {}
    for (i, j, k, l), v in zip(prob.v_idx.tolist(), prob.v_val.tolist()):
        by_kl.setdefault((k, l), []).append((i, j, v))
    n = len(basis)
    H = np.zeros((n, n))
    eps = prob.eps
    for col, s in enumerate(basis):
        occ = [x for x in range(prob.n_sites) if (s >> x) & 1]
        H[col, col] += sum(eps[x] for x in occ)
        for a in range(len(occ)):
            for b in range(a + 1, len(occ)):
                for (i, j, v) in by_kl.get((occ[a], occ[b]), ()):
                    r = _apply_term(s, i, j, occ[a], occ[b])
                    if r is None:
                        continue
                    sg, t = r
                    H[index[t], col] += sg * v
    return basis, H


def ed_lowest(prob, Np=None, Nn=None, two_M=None, k: int = 1):
    Np = prob.Np if Np is None else Np
    Nn = prob.Nn if Nn is None else Nn
    two_M = prob.two_Mz if two_M is None else two_M
    _, H = ed_sector(prob, Np, Nn, two_M)
    w = np.linalg.eigvalsh(H)
    return w[:k]


class ChainHamiltonian:
    """H of a Problem in chain positions: eps[c], site quantum numbers q[c] =
    (1,0,2m) for a proton, (0,1,2m) for a neutron, and the antisymmetrised W4(i,j,k,l)
    over chain positions with W4(i,j,k,l) = -W4(j,i,k,l) = -W4(i,j,l,k), such that
    the two-body part is 1/4 sum_{ijkl} W4 c+_i c+_j c_l c_k."""

    def __init__(self, prob):
        order = [int(x) for x in prob.order]
        pos = {s: c for c, s in enumerate(order)}
        self.N = len(order)
        self.target = (prob.Np, prob.Nn, prob.two_Mz)
        self.eps = np.array([prob.eps[s] for s in order], dtype=np.float64)
        self.q = [((1, 0, int(prob.two_m[s])) if prob.species[s] == 0
                   else (0, 1, int(prob.two_m[s]))) for s in order]
        self.vbar: Dict[Tuple[int, int, int, int], float] = {}
        for (i, j, k, l), v in zip(prob.v_idx.tolist(), prob.v_val.tolist()):
            ci, cj, ck, cl = pos[i], pos[j], pos[k], pos[l]
            sg = 1.0
            if ci > cj:
                ci, cj, sg = cj, ci, -sg
            if ck > cl:
                ck, cl, sg = cl, ck, -sg
            key = (ci, cj, ck, cl)
            self.vbar[key] = self.vbar.get(key, 0.0) + sg * v
        self.w4: Dict[Tuple[int, int, int, int], float] = {}
        for (i, j, k, l), v in self.vbar.items():
            if v == 0.0:
                continue
            self.w4[(i, j, k, l)] = v
            self.w4[(j, i, k, l)] = -v
            self.w4[(i, j, l, k)] = -v
            self.w4[(j, i, l, k)] = v

    def W(self, i, j, k, l) -> float:
        return self.w4.get((i, j, k, l), 0.0)


def fock_matrix(ch: ChainHamiltonian):
    """H on the full 2^N Fock space (chain order, site 0 most significant), sparse."""
    N = ch.N
    Z = sp.csr_matrix(np.diag([1.0, -1.0]))
    I2 = sp.identity(2, format="csr")
    a = sp.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]]))
    cs = []
    for i in range(N):
        m = sp.identity(1, format="csr")
        for t in range(N):
            m = sp.kron(m, Z if t < i else (a if t == i else I2), format="csr")
        cs.append(m)
    dim = 2 ** N
    H = sp.csr_matrix((dim, dim))
    for i in range(N):
        H = H + ch.eps[i] * (cs[i].T @ cs[i])
    for (i, j, k, l), v in ch.vbar.items():
        if v != 0.0:
            H = H + v * (cs[i].T @ cs[j].T @ cs[l] @ cs[k])
    return H.tocsr()
