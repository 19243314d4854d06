"""Seeded random right-canonical starting state (replaces the paper's CI-DEAS warm-up).

Chain positions c = 0..N-1 hold sites order[c].  Bond b lies between positions b and
b+1; the right block of bond b holds positions b+1..N-1.  The right block of bond N-2
(one site) keeps every target-compatible state.  For b = N-3 down to 2 the right block
of bond b is a truncation of the enlarged space  (site b+1) (x) (right block of bond b+1):

* enlarged sector Q = q_block + q_sigma; its rows are ordered piece by piece, site state
  sigma = 0 first (block sector Q), then sigma = 1 (block sector Q - q_site), and inside a
  piece by block state;
* a sector is kept only if it is target compatible: positions 0..b can hold q_T - Q;
* kept dimension m_Q = min(D_Q, ceil(M0 * full_Q / sum_Q' full_Q')), full_Q the
  Fock-space dimension of sector Q on positions b+1..N-1;
* U_Q (D_Q x m_Q) has orthonormal columns: Gaussian entries drawn in (bond, sector, row,
  col) order from SplitMix64(seed), then the Q factor of a thin QR with R's diagonal made
  positive (unique for full column rank).

Sectors are (N_p, N_n, 2M) triples in lexicographic order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Dict, List, Tuple

import numpy as np

from .prng import SplitMix64
from .shell import Problem, count_sector_dims


@dataclass
class InitialMPS:
    M0: int
    bonds: List[int]                 # b = N-3 ... 2, build order
    sectors: List[List[tuple]]       # per bond: kept sectors (canonical order)
    D: List[List[int]]               # enlarged dims per sector
    m: List[List[int]]               # kept dims per sector
    U: List[List[np.ndarray]]        # D x m isometries

    def flat(self):
        """Arrays for the C-ABI: bond_ptr [n_bonds+1], sec (n,5) int32 rows
        (Np, Nn, 2M, D, m), u_off int64 [n+1], u (float64)."""
        rows, uo, us = [], [0], []
        bond_ptr = [0]
        for b in range(len(self.bonds)):
            for q, D, m, U in zip(self.sectors[b], self.D[b], self.m[b], self.U[b]):
                rows.append((q[0], q[1], q[2], D, m))
                us.append(np.ascontiguousarray(U, dtype=np.float64).ravel())
                uo.append(uo[-1] + D * m)
            bond_ptr.append(len(rows))
        return (np.array(self.bonds, dtype=np.int32), np.array(bond_ptr, dtype=np.int32),
                np.array(rows, dtype=np.int32).reshape(-1, 5),
                np.array(uo, dtype=np.int64),
                np.concatenate(us) if us else np.zeros(0, dtype=np.float64))


def _chain_qn(prob: Problem):
    sp = [int(prob.species[s]) for s in prob.order]
    tm = [int(prob.two_m[s]) for s in prob.order]
    return sp, tm


def _site_q(sp: int, tm: int) -> tuple:
    return (1, 0, tm) if sp == 0 else (0, 1, tm)


def _sub(a, b):
    return (a[0] - b[0], a[1] - b[1], a[2] - b[2])


def _add(a, b):
    return (a[0] + b[0], a[1] + b[1], a[2] + b[2])


def initial_mps(prob: Problem, M0: int, seed: int) -> InitialMPS:
    N = prob.n_sites
    sp, tm = _chain_qn(prob)
    qT = (prob.Np, prob.Nn, prob.two_Mz)
    rng = SplitMix64(seed)
    # right block of bond N-2: site N-1, all compatible states
    left_full = count_sector_dims(sp[:N - 1], tm[:N - 1])
    blk: Dict[tuple, int] = {}
    for q in ((0, 0, 0), _site_q(sp[N - 1], tm[N - 1])):
        if left_full.get(_sub(qT, q), 0) > 0:
            blk[q] = 1
    out = InitialMPS(M0, [], [], [], [], [])
    for b in range(N - 3, 1, -1):
        s = b + 1
        qs = _site_q(sp[s], tm[s])
        left_full = count_sector_dims(sp[:b + 1], tm[:b + 1])
        right_full = count_sector_dims(sp[b + 1:], tm[b + 1:])
        enl = {}
        for q, d in blk.items():
            for Q in (q, _add(q, qs)):
                enl[Q] = enl.get(Q, 0) + d
        compat = sorted(Q for Q in enl if left_full.get(_sub(qT, Q), 0) > 0)
        tot_full = sum(right_full[Q] for Q in compat)
        secs, Ds, ms, Us = [], [], [], []
        for Q in compat:
            D = enl[Q]
            m = min(D, int(math.ceil(M0 * right_full[Q] / tot_full)))
            if m == 0:
                continue
            A = rng.gausses(D * m).reshape(D, m)
            Qm, R = np.linalg.qr(A)
            sg = np.sign(np.diag(R))
            sg[sg == 0] = 1.0
            Qm = Qm * sg[None, :]
            secs.append(Q)
            Ds.append(D)
            ms.append(m)
            Us.append(Qm)
        out.bonds.append(b)
        out.sectors.append(secs)
        out.D.append(Ds)
        out.m.append(ms)
        out.U.append(Us)
        blk = {Q: m for Q, m in zip(secs, ms)}
    return out
