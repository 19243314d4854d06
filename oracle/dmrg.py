"""Oracle: plain two-site DMRG in FP64 with block-sparse (N_p, N_n, 2M) sectors.

TEST INFRASTRUCTURE ONLY -- imported by tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg; the CUDA library never calls it.

What it follows (the paper gives the scheme, not the mechanics):
* superblock Xi_l (x) Lambda_{i+1} (x) Lambda_{i+2} (x) Xi_r on the ordered orbital chain,
  left block of i orbitals, right block of N-i-2 (two-site variant); the enlarged left
  block is Xi_l (x) Lambda_{i+1}, the enlarged right block Lambda_{i+2} (x) Xi_r;
* block bases from unitary transformations by the SVD theorem while sweeping left to
  right and back ("sweeping back and forth"); here: eigenvectors of the reduced density
  matrix of the enlarged block, M block states kept;
* variational minimisation of the energy of Eq. (1): the lowest eigenpair of the
  superblock Hamiltonian by Davidson's method;
* truncation error = discarded weight.

Readings where the paper is silent (they are the same in the CUDA library):
* operators: normal / complementary partition of ``oracle.mpo``; Jordan-Wigner signs:
  (O_L . o_site) -> (O_L P_L^{|o|}) (x) o,  (o_site . O_R) -> (o P_site^{|O_R|}) (x) O_R,
  superblock term sign (-1)^{|R_k| N(q_L)}, P = (-1)^(particle number);
* enlarged sector Q: piece sigma=0 (block sector Q) first, then sigma=1 (Q - q_site);
  only sectors whose complement can reach the target are kept;
* Davidson: x0 normalised; Ritz pair of the projected matrix (projected matrix entries
  <v_i, H v_j> for i <= j); Ritz vector sign: largest |y_i| positive (lowest i on ties);
  residual r = H x - theta x; stop when |r| <= tol or after max_iter products;
  correction t_i = r_i / (theta - D_i) with |theta - D_i| clamped to >= 1e-8 keeping its
  sign (+ at zero); classical Gram-Schmidt twice; at max_sub vectors restart from the two
  lowest Ritz vectors with projected matrix diag(theta_0, theta_1);
* truncation: rho per sector, eigenvalues clipped at 0; if more states than M: sort by
  lambda descending, ties by sector then index; with lambda_M the M-th, keep every state
  with lambda >= max(lambda_M (1 - 1e-10), 1e-14) (never splits a degenerate multiplet);
  otherwise keep all.  Dynamic block state selection (DBSS, optional): M is the ceiling,
  m_min the floor (keep all when there are at most min(m_min, M) states), and the count
  at the cut is the fewest k >= min(m_min, M), k <= min(M, total), whose discarded weight
  1 - (lambda_1 + ... + lambda_k) (descending, summed in that order) is at most the
  target, else min(M, total); the same multiplet and 1e-14 rules follow.  Eigenvector
  sign: largest |component| positive (lowest index on ties); kept states of a sector in
  descending lambda;
* initial guess: the uniform vector at the first step, then White's transformation of
  the previous wave function through the new block basis and the stored basis of the
  neighbouring block; the same wave function when a sweep turns around.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np

from .hamiltonian import ChainHamiltonian
from .mpo import MPO, SITE_ENTRIES, SITE_PARITY


def _add(a, b):
    return (a[0] + b[0], a[1] + b[1], a[2] + b[2])


def _sub(a, b):
    return (a[0] - b[0], a[1] - b[1], a[2] - b[2])


def full_counts(qs: List[tuple]) -> Dict[tuple, int]:
    """Number of occupation states per (N_p, N_n, 2M) of sites with quantum numbers qs."""
    cnt = {(0, 0, 0): 1}
    for q in qs:
        new = dict(cnt)
        for k, c in cnt.items():
            kk = _add(k, q)
            new[kk] = new.get(kk, 0) + c
        cnt = new
    return cnt


@dataclass
class Block:
    """Block basis (sectors in lexicographic order with dims) and its operators:
    ops[label_index] = {(q_out, q_in): dense block}."""
    sectors: List[tuple]
    dims: Dict[tuple, int]
    ops: List[Dict[Tuple[tuple, tuple], np.ndarray]]
    # enlarged-block piece layout: Q -> [(sigma, q_block, offset, d)]
    pieces: Optional[Dict[tuple, list]] = None


def _pieces(blk: Block, qs: tuple, compat) -> Tuple[List[tuple], Dict[tuple, int], dict]:
    enl = {}
    for q in blk.sectors:
        for sg in (0, 1):
            Q = _add(q, qs) if sg else q
            enl.setdefault(Q, []).append((sg, q))
    secs = sorted(Q for Q in enl if compat(Q))
    pieces, dims = {}, {}
    for Q in secs:
        off = 0
        lst = []
        for sg, q in sorted(enl[Q]):
            d = blk.dims[q]
            lst.append((sg, q, off, d))
            off += d
        pieces[Q] = lst
        dims[Q] = off
    return secs, dims, pieces


def enlarge_left(blk: Block, s: int, mpo: MPO, ch: ChainHamiltonian) -> Block:
    """Operators of bond s on (block of bond s-1) (x) site s."""
    qs = ch.q[s]
    right = full_counts(ch.q[s + 1:])
    qT = ch.target
    secs, dims, pieces = _pieces(blk, qs, lambda Q: right.get(_sub(qT, Q), 0) > 0)
    poff = {(Q, sg, q): off for Q in secs for (sg, q, off, d) in pieces[Q]}
    nlab = len(mpo.labels[s + 1])
    ops: List[dict] = [dict() for _ in range(nlab)]
    for (a, b, op, coef) in mpo.W[s]:
        par = SITE_PARITY[op]
        for (qo, qi), X in blk.ops[a].items():
            for (so, si) in SITE_ENTRIES[op]:
                Qo = _add(qo, qs) if so else qo
                Qi = _add(qi, qs) if si else qi
                if Qo not in dims or Qi not in dims:
                    continue
                sign = -1.0 if (par and (qi[0] + qi[1]) % 2) else 1.0
                key = (Qo, Qi)
                if key not in ops[b]:
                    ops[b][key] = np.zeros((dims[Qo], dims[Qi]))
                ro, ri = poff[(Qo, so, qo)], poff[(Qi, si, qi)]
                ops[b][key][ro:ro + X.shape[0], ri:ri + X.shape[1]] += coef * sign * X
    return Block(secs, dims, ops, pieces)


def enlarge_right(blk: Block, s: int, mpo: MPO, ch: ChainHamiltonian) -> Block:
    """Operators of bond s-1 on site s (x) (block of bond s)."""
    qs = ch.q[s]
    left = full_counts(ch.q[:s])
    qT = ch.target
    secs, dims, pieces = _pieces(blk, qs, lambda Q: left.get(_sub(qT, Q), 0) > 0)
    poff = {(Q, sg, q): off for Q in secs for (sg, q, off, d) in pieces[Q]}
    nlab = len(mpo.labels[s])
    ops: List[dict] = [dict() for _ in range(nlab)]
    par_b = mpo.parity[s + 1]
    for (a, b, op, coef) in mpo.W[s]:
        for (qo, qi), X in blk.ops[b].items():
            for (so, si) in SITE_ENTRIES[op]:
                Qo = _add(qo, qs) if so else qo
                Qi = _add(qi, qs) if si else qi
                if Qo not in dims or Qi not in dims:
                    continue
                sign = -1.0 if (par_b[b] and si) else 1.0
                key = (Qo, Qi)
                if key not in ops[a]:
                    ops[a][key] = np.zeros((dims[Qo], dims[Qi]))
                ro, ri = poff[(Qo, so, qo)], poff[(Qi, si, qi)]
                ops[a][key][ro:ro + X.shape[0], ri:ri + X.shape[1]] += coef * sign * X
    return Block(secs, dims, ops, pieces)


def vacuum(label_count: int, which: int) -> Block:
    ops = [dict() for _ in range(label_count)]
    ops[which][((0, 0, 0), (0, 0, 0))] = np.ones((1, 1))
    return Block([(0, 0, 0)], {(0, 0, 0): 1}, ops)


def project(enl: Block, U: Dict[tuple, np.ndarray]) -> Block:
    """New block = kept states of the enlarged block: O' = U^T O U."""
    secs = [Q for Q in enl.sectors if Q in U and U[Q].shape[1] > 0]
    dims = {Q: U[Q].shape[1] for Q in secs}
    ops = []
    for op in enl.ops:
        new = {}
        for (Qo, Qi), X in op.items():
            if Qo in dims and Qi in dims:
                new[(Qo, Qi)] = U[Qo].T @ X @ U[Qi]
        ops.append(new)
    return Block(secs, dims, ops)


# ----------------------------------------------------------------------------------
# superblock wave function and H_eff
# ----------------------------------------------------------------------------------
@dataclass
class Layout:
    blocks: List[Tuple[tuple, tuple, int, int, int]]   # (Q_L, Q_R, dL, dR, offset)
    size: int

    def index(self):
        return {b[0]: b for b in self.blocks}


def psi_layout(Lenl: Block, Renl: Block, qT) -> Layout:
    out, off = [], 0
    for QL in Lenl.sectors:
        QR = _sub(qT, QL)
        if QR in Renl.dims:
            dL, dR = Lenl.dims[QL], Renl.dims[QR]
            out.append((QL, QR, dL, dR, off))
            off += dL * dR
    return Layout(out, off)


class SuperBlock:
    def __init__(self, Lenl: Block, Renl: Block, parity: List[int], qT):
        self.L, self.R, self.parity, self.qT = Lenl, Renl, parity, qT
        self.layout = psi_layout(Lenl, Renl, qT)
        self.n_apply = 0

    def apply(self, x: np.ndarray) -> np.ndarray:
        """y = sum_k (-1)^{|R_k| N(Q_L)} L_k psi R_k^T, block by block."""
        lay = self.layout
        idx = lay.index()
        y = np.zeros(lay.size)
        for k, (Lk, Rk) in enumerate(zip(self.L.ops, self.R.ops)):
            pk = self.parity[k]
            for (QLo, QLi), Lblk in Lk.items():
                if QLi not in idx or QLo not in idx:
                    continue
                _, QRi, dLi, dRi, oi = idx[QLi]
                _, QRo, dLo, dRo, oo = idx[QLo]
                Rblk = Rk.get((QRo, QRi))
                if Rblk is None:
                    continue
                sign = -1.0 if (pk and (QLi[0] + QLi[1]) % 2) else 1.0
                psi = x[oi:oi + dLi * dRi].reshape(dLi, dRi)
                y[oo:oo + dLo * dRo] += sign * (Lblk @ psi @ Rblk.T).ravel()
        self.n_apply += 1
        return y

    def diagonal(self) -> np.ndarray:
        lay = self.layout
        d = np.zeros(lay.size)
        for Lk, Rk in zip(self.L.ops, self.R.ops):
            for (QL, QR, dL, dR, off) in lay.blocks:
                Lb = Lk.get((QL, QL))
                Rb = Rk.get((QR, QR))
                if Lb is None or Rb is None:
                    continue
                d[off:off + dL * dR] += np.outer(np.diag(Lb), np.diag(Rb)).ravel()
        return d


def _sign_fix(y: np.ndarray) -> np.ndarray:
    i = int(np.argmax(np.abs(y)))
    return -y if y[i] < 0 else y


def davidson(apply, diag, x0, tol=1e-8, max_iter=100, max_sub=24):
    """Lowest eigenpair; returns (theta, x, n_products, |r|)."""
    x0 = x0 / np.linalg.norm(x0)
    V = [x0]
    AV = [apply(x0)]
    nprod = 1
    Hs = np.array([[V[0] @ AV[0]]])
    while True:
        w, Y = np.linalg.eigh(Hs)
        theta = w[0]
        y = _sign_fix(Y[:, 0])
        x = sum(y[i] * V[i] for i in range(len(V)))
        Ax = sum(y[i] * AV[i] for i in range(len(V)))
        r = Ax - theta * x
        rn = float(np.linalg.norm(r))
        if rn <= tol or nprod >= max_iter:
            return float(theta), x / np.linalg.norm(x), nprod, rn
        den = theta - diag
        small = np.abs(den) < 1e-8
        den[small] = np.where(den[small] < 0, -1e-8, 1e-8)
        t = r / den
        if len(V) >= max_sub:
            y1 = _sign_fix(Y[:, 1])
            x1 = sum(y1[i] * V[i] for i in range(len(V)))
            Ax1 = sum(y1[i] * AV[i] for i in range(len(V)))
            V, AV = [x, x1], [Ax, Ax1]
            Hs = np.array([[w[0], 0.0], [0.0, w[1]]])
        tn0 = np.linalg.norm(t)
        for _ in range(2):
            for v in V:
                t = t - (v @ t) * v
        tn = np.linalg.norm(t)
        if tn <= 1e-14 * max(tn0, 1e-300):
            return float(theta), x / np.linalg.norm(x), nprod, rn
        t = t / tn
        At = apply(t)
        nprod += 1
        k = len(V)
        Hn = np.zeros((k + 1, k + 1))
        Hn[:k, :k] = Hs
        for i in range(k):
            Hn[i, k] = Hn[k, i] = V[i] @ At
        Hn[k, k] = t @ At
        V.append(t)
        AV.append(At)
        Hs = Hn


def davidson_roots(apply, diag, guesses, tol=1e-8, max_iter=100, max_sub=24, n_roots=2):
    """The n_roots (1 or 2) lowest eigenpairs, for targeting several states at once (the
    2+ excitation energies).  Same iteration as ``davidson``; the subspace starts from
    the first guess, later guesses enter it before any correction; each iteration adds
    the correction of the lowest root whose residual is above tol (root 0 while fewer
    vectors than roots exist); stop when every root's residual is at most tol, or after
    max_iter products.  Returns (thetas, normalised vectors, n_products, residuals)."""
    x0 = guesses[0] / np.linalg.norm(guesses[0])
    V = [x0]
    AV = [apply(x0)]
    nprod = 1
    Hs = np.array([[V[0] @ AV[0]]])
    pending = [g for g in guesses[1:n_roots]]
    while True:
        w, Y = np.linalg.eigh(Hs)
        k = len(V)
        xs, Axs, rs, rns = [], [], [], []
        for j in range(min(n_roots, k)):
            y = _sign_fix(Y[:, j])
            x = sum(y[i] * V[i] for i in range(k))
            Ax = sum(y[i] * AV[i] for i in range(k))
            xs.append(x)
            Axs.append(Ax)
            rs.append(Ax - w[j] * x)
            rns.append(float(np.linalg.norm(rs[-1])))
        done = k >= n_roots and all(rn <= tol for rn in rns)
        if done or nprod >= max_iter:
            return ([float(v) for v in w[:len(xs)]], [x / np.linalg.norm(x) for x in xs], nprod,
                    rns)
        t = None
        if pending:                       # a further guess, orthogonalised like a correction
            t = pending.pop(0).copy()
            tn0 = np.linalg.norm(t)
            for _ in range(2):
                for v in V:
                    t = t - (v @ t) * v
            if np.linalg.norm(t) <= 1e-14 * max(tn0, 1e-300):
                t = None
        if t is None:
            j = next((j for j, rn in enumerate(rns) if rn > tol), 0)
            den = w[j] - diag
            small = np.abs(den) < 1e-8
            den[small] = np.where(den[small] < 0, -1e-8, 1e-8)
            t = rs[j] / den
            if k >= max_sub:              # restart from the two lowest Ritz vectors
                y1 = _sign_fix(Y[:, 1])
                x1 = sum(y1[i] * V[i] for i in range(k))
                Ax1 = sum(y1[i] * AV[i] for i in range(k))
                V, AV = [xs[0], x1], [Axs[0], Ax1]
                Hs = np.array([[w[0], 0.0], [0.0, w[1]]])
            tn0 = np.linalg.norm(t)
            for _ in range(2):
                for v in V:
                    t = t - (v @ t) * v
            if np.linalg.norm(t) <= 1e-14 * max(tn0, 1e-300):
                return ([float(v) for v in w[:len(xs)]], [x / np.linalg.norm(x) for x in xs],
                        nprod, rns)
        t = t / np.linalg.norm(t)
        At = apply(t)
        nprod += 1
        k = len(V)
        Hn = np.zeros((k + 1, k + 1))
        Hn[:k, :k] = Hs
        for i in range(k):
            Hn[i, k] = Hn[k, i] = V[i] @ At
        Hn[k, k] = t @ At
        V.append(t)
        AV.append(At)
        Hs = Hn


# ----------------------------------------------------------------------------------
# truncation by the reduced density matrix
# ----------------------------------------------------------------------------------
def dbss_count(w_desc, k_min: int, k_max: int, target: float) -> int:
    """Dynamic block state selection (method section, DBSS with an a priori truncation
    error): the fewest states k, k_min <= k <= k_max, whose discarded weight
    1 - (w_1 + ... + w_k) is at most ``target``; k_max when no k qualifies.  The weights
    come sorted descending and are summed in that order."""
    kept = 0.0
    for k in range(1, k_max + 1):
        kept += float(w_desc[k - 1])
        if k >= k_min and 1.0 - kept <= target:
            return k
    return k_max


def truncate(psi: np.ndarray, lay: Layout, enl: Block, side: str, M: int, m_min: int = 0,
             trunc_target: float = 0.0):
    """Returns (U per kept sector, kept count per sector, truncation error, eigenvalues).

    psi: one wave function, or several as the rows of a 2-D array (targeted states), whose
    density matrices are averaged with equal weights.  trunc_target > 0 selects
    dynamically: M is the ceiling, m_min the floor, and the count at the cut is
    ``dbss_count``; otherwise M states are kept."""
    vecs = [psi] if psi.ndim == 1 else list(psi)
    rho = {}
    for (QL, QR, dL, dR, off) in lay.blocks:
        for v in vecs:
            P = v[off:off + dL * dR].reshape(dL, dR)
            part = (P @ P.T if side == "L" else P.T @ P) / len(vecs)
            Q = QL if side == "L" else QR
            rho[Q] = rho[Q] + part if Q in rho else part
    evals, evecs = {}, {}
    for Q in enl.sectors:
        d = enl.dims[Q]
        R = rho.get(Q, np.zeros((d, d)))
        w, V = np.linalg.eigh(R)
        w = np.clip(w[::-1], 0.0, None)
        V = V[:, ::-1]
        evals[Q], evecs[Q] = w, V
    allv = [(-evals[Q][i], Q, i) for Q in enl.sectors for i in range(enl.dims[Q])]
    total = len(allv)
    dbss = trunc_target > 0.0
    floor = min(m_min, M) if dbss else M
    if total <= floor:
        keep = {Q: enl.dims[Q] for Q in enl.sectors}
    else:
        allv.sort()
        k = min(M, total)
        if dbss:
            k = dbss_count([-v[0] for v in allv], floor, k, trunc_target)
        lamM = -allv[k - 1][0]
        thr = max(lamM * (1.0 - 1e-10), 1e-14)
        keep = {Q: int(np.sum(evals[Q] >= thr)) for Q in enl.sectors}
    U = {}
    kept_w = 0.0
    for Q in enl.sectors:
        m = keep[Q]
        if m == 0:
            continue
        cols = [_sign_fix(evecs[Q][:, c]) for c in range(m)]
        U[Q] = np.stack(cols, axis=1)
        kept_w += float(np.sum(evals[Q][:m]))
    trunc = max(0.0, 1.0 - kept_w)
    return U, keep, trunc, evals


# ----------------------------------------------------------------------------------
# sweeps
# ----------------------------------------------------------------------------------
@dataclass
class StepResult:
    p: int
    direction: str
    energy: float
    n_products: int
    residual: float
    trunc_err: float
    kept: Dict[tuple, int]
    energy1: float = float("nan")     # second targeted state (two-state targeting)


class OracleDMRG:
    def __init__(self, prob, init_mps, tol=1e-8, max_iter=100, max_sub=24, m_min=0,
                 trunc_target=0.0, n_roots=1):
        self.m_min, self.trunc_target = m_min, trunc_target   # DBSS (trunc_target > 0)
        self.n_roots = n_roots        # 2: the two lowest states targeted together
        self.psi1 = None              # second targeted state of the last step
        self.ch = ch = ChainHamiltonian(prob)
        self.mpo = mpo = MPO(ch)
        self.N = N = ch.N
        self.tol, self.max_iter, self.max_sub = tol, max_iter, max_sub
        self.left: Dict[int, Block] = {}
        self.right: Dict[int, Block] = {}
        self.UL: Dict[int, Dict[tuple, np.ndarray]] = {}
        self.UR: Dict[int, Dict[tuple, np.ndarray]] = {}
        # left block of bond 0: site 0, every compatible state
        e = enlarge_left(vacuum(1, 0), 0, mpo, ch)
        self.UL[0] = {Q: np.eye(e.dims[Q]) for Q in e.sectors}
        self.left[0] = project(e, self.UL[0])
        # right block of bond N-2: site N-1, every compatible state
        e = enlarge_right(vacuum(1, 0), N - 1, mpo, ch)
        self.UR[N - 2] = {Q: np.eye(e.dims[Q]) for Q in e.sectors}
        self.right[N - 2] = project(e, self.UR[N - 2])
        # right blocks N-3 .. 2 from the starting state
        for bi, b in enumerate(init_mps.bonds):
            e = enlarge_right(self.right[b + 1], b + 1, mpo, ch)
            U = {}
            for Q, D, m, Um in zip(init_mps.sectors[bi], init_mps.D[bi], init_mps.m[bi],
                                   init_mps.U[bi]):
                Q = tuple(Q)
                if e.dims.get(Q) != D:
                    raise ValueError(f"starting state does not match bond {b} sector {Q}")
                U[Q] = np.asarray(Um)
            self.UR[b] = U
            self.right[b] = project(e, U)
        self.psi = None
        self.psi_layout = None
        self.psi_at = None            # (p, enlarged blocks) the stored psi belongs to
        self.history: List[StepResult] = []

    # -- superblock at position p (dots p, p+1)
    def superblock(self, p: int) -> SuperBlock:
        Lenl = enlarge_left(self.left[p - 1], p, self.mpo, self.ch)
        Renl = enlarge_right(self.right[p + 1], p + 1, self.mpo, self.ch)
        return SuperBlock(Lenl, Renl, self.mpo.parity[p + 1], self.ch.target)

    def _guess(self, p: int, direction: str, sb: SuperBlock, old=None) -> np.ndarray:
        """White's prediction of the wave function at position p from the previous one
        (``old``: another vector of the previous step, default its ground state)."""
        lay = sb.layout
        if self.psi is None:
            return np.ones(lay.size) / math.sqrt(max(lay.size, 1))
        old = self.psi if old is None else old
        if self.psi_at[0] == p:
            return old.copy()
        olay = self.psi_layout
        new = np.zeros(lay.size)
        nidx = lay.index()
        q = self.ch.q
        if direction == "L":
            # previous step at p-1 truncated the left: psi(l s_{p-1}, s_p r) ->
            # U^T psi, then r (right block of bond p) expanded into s_{p+1} r'
            U, Ur = self.UL[p - 1], self.UR[p]
            for (QL, QR, dL, dR, off) in olay.blocks:
                if QL not in U:
                    continue
                X = U[QL].T @ old[off:off + dL * dR].reshape(dL, dR)
                for (sg, qr, coff, dr) in self._prev_R.pieces[QR]:
                    QLn = _add(QL, q[p]) if sg else QL
                    if qr not in Ur or QLn not in nidx:
                        continue
                    _, QRn, dLn, dRn, offn = nidx[QLn]
                    if QRn != qr:
                        continue
                    rof = [o for (s_, q_, o, d_) in sb.L.pieces[QLn] if s_ == sg and q_ == QL][0]
                    blk = new[offn:offn + dLn * dRn].reshape(dLn, dRn)
                    blk[rof:rof + X.shape[0], :] += X[:, coff:coff + dr] @ Ur[qr].T
        else:
            # previous step at p+1 truncated the right: psi(l s_{p+1}, s_{p+2} r) ->
            # psi V, then l (left block of bond p) expanded into l'' s_p
            V, Ul = self.UR[p + 1], self.UL[p]
            for (QL, QR, dL, dR, off) in olay.blocks:
                if QR not in V:
                    continue
                X = old[off:off + dL * dR].reshape(dL, dR) @ V[QR]
                for (sg, ql, roff, dl) in self._prev_L.pieces[QL]:
                    if ql not in Ul or ql not in nidx:
                        continue
                    _, QRn, dLn, dRn, offn = nidx[ql]
                    if QRn != (_add(QR, q[p + 1]) if sg else QR):
                        continue
                    cof = [o for (s_, q_, o, d_) in sb.R.pieces[QRn] if s_ == sg and q_ == QR][0]
                    blk = new[offn:offn + dLn * dRn].reshape(dLn, dRn)
                    blk[:, cof:cof + X.shape[1]] += Ul[ql] @ X[roff:roff + dl, :]
        nrm = np.linalg.norm(new)
        if nrm == 0.0:
            return np.ones(lay.size) / math.sqrt(max(lay.size, 1))
        return new / nrm

    def run_step(self, p: int, direction: str, M: int) -> StepResult:
        sb = self.superblock(p)
        x0 = self._guess(p, direction, sb)
        diag = sb.diagonal()
        theta1, x1 = float("nan"), None
        if self.n_roots == 1:
            theta, x, nprod, rn = davidson(sb.apply, diag, x0, self.tol, self.max_iter,
                                           self.max_sub)
            target = x
        else:
            guesses = [x0]
            if self.psi1 is not None:
                guesses.append(self._guess(p, direction, sb, self.psi1))
            th, xs, nprod, rns = davidson_roots(sb.apply, diag, guesses, self.tol,
                                                self.max_iter, self.max_sub, 2)
            if len(xs) < 2:
                raise ValueError("superblock too small for two targeted states")
            theta, theta1, x, x1, rn = th[0], th[1], xs[0], xs[1], max(rns)
            target = np.stack([x, x1])
        if direction == "L":
            U, keep, tr, _ = truncate(target, sb.layout, sb.L, "L", M, self.m_min,
                                      self.trunc_target)
            self.UL[p] = U
            self.left[p] = project(sb.L, U)
        else:
            U, keep, tr, _ = truncate(target, sb.layout, sb.R, "R", M, self.m_min,
                                      self.trunc_target)
            self.UR[p] = U
            self.right[p] = project(sb.R, U)
        self.psi, self.psi_layout, self.psi_at = x, sb.layout, (p, direction)
        self.psi1 = x1
        self._prev_L, self._prev_R = sb.L, sb.R
        res = StepResult(p, direction, theta, nprod, rn, tr, keep, theta1)
        self.history.append(res)
        return res

    def sweep(self, M: int) -> List[StepResult]:
        """One round trip: p = 1..N-3 left to right, then N-3..1 right to left."""
        out = []
        for p in range(1, self.N - 2):
            out.append(self.run_step(p, "L", M))
        for p in range(self.N - 3, 0, -1):
            out.append(self.run_step(p, "R", M))
        return out
