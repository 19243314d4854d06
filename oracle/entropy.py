"""Oracle: orbital entropies of the two dot orbitals of a two-site DMRG step.

TEST INFRASTRUCTURE ONLY (checks the library's dot reduced density matrix).

The paper quantifies each orbital's share of the correlation by the one-orbital von
Neumann entropy s_i = -Tr rho_i ln rho_i of its reduced density matrix, and the
correlation of two orbitals by the mutual information built from s_i, s_j and the
two-orbital entropy s_ij.  Readings where the paper is silent or garbled:
* the mutual information is I_ij = s_i + s_j - s_ij (non-negative; the printed formula
  has the opposite overall sign);
* natural logarithms;
* ``dot_rdm``: the two dot orbitals p, p+1 of a step, read directly off the two-site wave
  function psi(l, n_p, n_{p+1}, r) (what the library computes);
* ``state_amplitudes`` / ``pair_rdm`` / ``mutual_information``: every pair, from the
  state written out in the occupation basis of the chain (small cases only; the plain
  definition that a device implementation for all pairs will be checked against);
* ``mutual_information_dets``: the same matrix from a state given as arrays (determinant
  bitmasks, amplitudes), vectorised over determinants for the exact pf-shell ground state
  (dimension ~2e6) whose mutual information orders the chain of the pf 4p+4n workload.

Basis of the two-orbital matrix: index 2 n_p + n_{p+1} (|00>, |01>, |10>, |11>),
    rho[a, b] = sum_{l, r} psi(l, a, r) psi(l, b, r).
Particle numbers and 2M are conserved, so rho is diagonal except for the |01>, |10>
element, which is nonzero only when the two orbitals carry the same (species, m); with
the Jordan-Wigner strings in chain order it equals <c+_{p+1} c_p> (no string lies
between neighbours, and the one to the left of p cancels).
"""
import numpy as np


def _add(a, b):
    return (a[0] + b[0], a[1] + b[1], a[2] + b[2])


def dot_rdm(psi, layout, Lenl, Renl, q_p, q_p1):
    """Two-orbital reduced density matrix of the dot orbitals (4 x 4, basis above).

    psi: the wave function in ``layout`` (one dense block per enlarged-left sector);
    Lenl, Renl: the enlarged blocks with their piece lists (site state 0 first);
    q_p, q_p1: the quantum numbers (N_p, N_n, 2m) of the two dot orbitals."""
    rho = np.zeros((4, 4))
    blocks = {QL: (QR, dL, dR, off) for (QL, QR, dL, dR, off) in layout.blocks}
    for QL, (QR, dL, dR, off) in blocks.items():
        P = psi[off:off + dL * dR].reshape(dL, dR)
        for (sl, ql, ro, dl) in Lenl.pieces[QL]:
            for (sr, qr, co, dr) in Renl.pieces[QR]:
                a = 2 * sl + sr
                rho[a, a] += float(np.sum(P[ro:ro + dl, co:co + dr] ** 2))
    if tuple(q_p) == tuple(q_p1):
        x = 0.0
        for QL, (QR, dL, dR, off) in blocks.items():
            P = psi[off:off + dL * dR].reshape(dL, dR)
            for (sl, ql, ro, dl) in Lenl.pieces[QL]:
                if sl != 1:
                    continue
                for (sr, qr, co, dr) in Renl.pieces[QR]:
                    if sr != 0:
                        continue
                    # partner amplitude psi(l, 0, 1, r): left sector ql (piece 0),
                    # right sector QR + q_p1 (piece 1 over the same block sector qr)
                    if ql not in blocks:
                        continue
                    QR2, dL2, dR2, off2 = blocks[ql]
                    if QR2 != _add(QR, q_p1):
                        continue
                    ro2 = [o for (s_, q_, o, d_) in Lenl.pieces[ql] if s_ == 0 and q_ == ql]
                    co2 = [o for (s_, q_, o, d_) in Renl.pieces[QR2] if s_ == 1 and q_ == qr]
                    if not ro2 or not co2:
                        continue
                    P2 = psi[off2:off2 + dL2 * dR2].reshape(dL2, dR2)
                    x += float(np.sum(P[ro:ro + dl, co:co + dr] *
                                      P2[ro2[0]:ro2[0] + dl, co2[0]:co2[0] + dr]))
        rho[1, 2] = rho[2, 1] = x
    return rho


def _vn(w):
    w = np.asarray(w, dtype=np.float64)
    w = w[w > 0.0]
    return float(-np.sum(w * np.log(w)))


def entropies(rho):
    """(s_p, s_{p+1}, s_{p,p+1}, I_{p,p+1}) of a dot density matrix."""
    s_p = _vn([rho[0, 0] + rho[1, 1], rho[2, 2] + rho[3, 3]])
    s_q = _vn([rho[0, 0] + rho[2, 2], rho[1, 1] + rho[3, 3]])
    s_pq = _vn(np.linalg.eigvalsh(rho))
    return s_p, s_q, s_pq, s_p + s_q - s_pq


# ----------------------------------------------------------------------------------
# every orbital pair, from the state written out in the occupation basis
# ----------------------------------------------------------------------------------
def _block_patterns(o, p=None):
    """Left blocks (bonds 0..N-3) and right blocks (bonds 2..N-2) of an OracleDMRG as
    {sector: (occupation bitmasks over chain positions, coefficients patterns x m)}; with p
    given, only the blocks the superblock at p is built from (left bonds < p, right bonds
    > p), which are consistent with each other in the middle of a sweep."""
    from .dmrg import enlarge_left, enlarge_right, vacuum
    N = o.N
    left, right = {}, {}
    prev = {(0, 0, 0): ([0], np.ones((1, 1)))}
    for b in range(0, N - 2 if p is None else p):
        if b not in o.UL:
            break
        blk = vacuum(1, 0) if b == 0 else o.left[b - 1]
        enl = enlarge_left(blk, b, o.mpo, o.ch)
        cur = {}
        for Q, U in o.UL[b].items():
            pats, E = _enlarged(enl.pieces[Q], prev, lambda pat, sg: pat | (sg << b), enl.dims[Q])
            cur[Q] = (pats, E @ U)
        left[b] = prev = cur
    prev = {(0, 0, 0): ([0], np.ones((1, 1)))}
    for b in range(N - 2, 1 if p is None else p, -1):
        if b not in o.UR:
            break
        blk = vacuum(1, 0) if b == N - 2 else o.right[b + 1]
        enl = enlarge_right(blk, b + 1, o.mpo, o.ch)
        cur = {}
        for Q, U in o.UR[b].items():
            pats, E = _enlarged(enl.pieces[Q], prev, lambda pat, sg: pat | (sg << (b + 1)),
                                enl.dims[Q])
            cur[Q] = (pats, E @ U)
        right[b] = prev = cur
    return left, right


def _enlarged(pieces, blocks, place, D):
    """Occupation-basis vectors of an enlarged sector's states: piece (sigma, q, off, d)
    holds the d states of block sector q with the site in state sigma."""
    pats, cols = [], []
    for (sg, q, off, d) in pieces:
        bp, C = blocks[q]
        for k, pat in enumerate(bp):
            pats.append(place(pat, sg))
            row = np.zeros(D)
            row[off:off + d] = C[k]
            cols.append(row)
    return pats, np.array(cols)


def state_amplitudes(o):
    """The wave function of the last step of an OracleDMRG written out: {occupation
    bitmask over chain positions: amplitude} (tensor basis in chain order)."""
    p = o.psi_at[0]
    left, right = _block_patterns(o, p)
    lb, rb = left[p - 1], right[p + 1]
    Lenl, Renl = o._prev_L, o._prev_R
    amp = {}
    for (QL, QR, dL, dR, off) in o.psi_layout.blocks:
        pl, EL = _enlarged(Lenl.pieces[QL], lb, lambda pat, sg: pat | (sg << p), dL)
        pr, ER = _enlarged(Renl.pieces[QR], rb, lambda pat, sg: pat | (sg << (p + 1)), dR)
        A = EL @ o.psi[off:off + dL * dR].reshape(dL, dR) @ ER.T
        for i, a in enumerate(pl):
            for j, c in enumerate(pr):
                if A[i, j] != 0.0:
                    amp[a | c] = amp.get(a | c, 0.0) + A[i, j]
    return amp


def pair_rdm(amp, i, j):
    """Two-orbital density matrix of chain positions i < j from occupation amplitudes:
    basis 2 n_i + n_j, off-diagonal element <c+_j c_i> (the Jordan-Wigner string gives
    (-1)^(number of occupied positions strictly between i and j))."""
    rho = np.zeros((4, 4))
    x = 0.0
    between = ((1 << j) - 1) & ~((1 << (i + 1)) - 1)
    for pat, a in amp.items():
        ni, nj = (pat >> i) & 1, (pat >> j) & 1
        rho[2 * ni + nj, 2 * ni + nj] += a * a
        if ni == 1 and nj == 0:
            partner = amp.get((pat ^ (1 << i)) | (1 << j))
            if partner is not None:
                sign = -1.0 if bin(pat & between).count("1") & 1 else 1.0
                x += sign * partner * a
    rho[1, 2] = rho[2, 1] = x
    return rho


def mutual_information(amp, n):
    """n x n matrix I_ij of the chain positions (zero diagonal) and the one-orbital
    entropies s_i."""
    I = np.zeros((n, n))
    s = np.zeros(n)
    for i in range(n):
        for j in range(i + 1, n):
            si, sj, _, mi = entropies(pair_rdm(amp, i, j))
            I[i, j] = I[j, i] = mi
            s[i], s[j] = si, sj
    return I, s


def mutual_information_dets(masks, amps, n):
    """n x n mutual information I_ij (zero diagonal) and one-orbital entropies s_i of a
    state over determinants: masks (uint64 bitmasks over n orbitals, any order), amps
    (real amplitudes, normalised).  Same definition as ``pair_rdm``: basis 2 n_i + n_j,
    off-diagonal element <c+_j c_i> with the string sign (-1)^(occupied orbitals strictly
    between i and j); the partner determinant is looked up by binary search and counts
    only if present (absent partners lie outside the state's sector)."""
    masks = np.asarray(masks, dtype=np.uint64)
    amps = np.asarray(amps, dtype=np.float64)
    order = np.argsort(masks)
    sm, sa = masks[order], amps[order]
    prob = sa * sa
    bits = ((sm[:, None] >> np.arange(n, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(bool)
    occ = bits.T.astype(np.float64) @ prob                       # <n_i>
    both = (bits.T.astype(np.float64) * prob) @ bits.astype(np.float64)   # <n_i n_j>
    I = np.zeros((n, n))
    s = np.zeros(n)
    for i in range(n):
        p1 = occ[i]
        s[i] = _vn([1.0 - p1, p1])
    for i in range(n):
        for j in range(i + 1, n):
            rho = np.zeros((4, 4))
            n11 = both[i, j]
            n10 = occ[i] - n11
            n01 = occ[j] - n11
            rho[3, 3] = n11
            rho[2, 2] = n10
            rho[1, 1] = n01
            rho[0, 0] = 1.0 - n11 - n10 - n01
            sel = bits[:, i] & ~bits[:, j]
            x = 0.0
            if sel.any():
                src = sm[sel]
                partner = (src ^ np.uint64(1 << i)) | np.uint64(1 << j)
                pos = np.searchsorted(sm, partner)
                pos = np.minimum(pos, sm.shape[0] - 1)
                hit = sm[pos] == partner
                if hit.any():
                    between = np.uint64(((1 << j) - 1) & ~((1 << (i + 1)) - 1))
                    cnt = _popcount64(src[hit] & between)
                    sign = np.where(cnt & 1, -1.0, 1.0)
                    x = float(np.sum(sign * sa[sel][hit] * sa[pos[hit]]))
            rho[1, 2] = rho[2, 1] = x
            si, sj, _, mi = entropies(rho)
            I[i, j] = I[j, i] = mi
    return I, s


def _popcount64(v):
    v = np.asarray(v, dtype=np.uint64)
    c = np.zeros(v.shape, dtype=np.int64)
    for b in range(64):
        c += ((v >> np.uint64(b)) & np.uint64(1)).astype(np.int64)
    return c
