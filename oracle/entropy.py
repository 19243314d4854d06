"""Oracle: orbital entropies of the two dot orbitals of a two-site DMRG step.

TEST INFRASTRUCTURE ONLY (checks the library's dot reduced density matrix).

The paper quantifies each orbital's share of the correlation by the one-orbital von
Neumann entropy s_i = -Tr rho_i ln rho_i of its reduced density matrix, and the
correlation of two orbitals by the mutual information built from s_i, s_j and the
two-orbital entropy s_ij.  Readings where the paper is silent or garbled:
* the mutual information is I_ij = s_i + s_j - s_ij (non-negative; the printed formula
  has the opposite overall sign);
* natural logarithms;
* here only the two dot orbitals p, p+1 of a step are treated: their two-orbital density
  matrix is read directly off the two-site wave function psi(l, n_p, n_{p+1}, r), so a
  sweep yields s_i for every orbital and I_{p,p+1} for every neighbouring pair.

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
