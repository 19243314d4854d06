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
* ``lanczos_lowest``: the exact lowest eigenpair of a sector too large for a dense
  matrix (the pf 4p+4n space, dimension 1,963,461), by the Lanczos method with full
  reorthogonalisation in FP64 (plain C in ``oracle/lanczos.c``, matrix-free: every term
  of H applied to every determinant).  ``mscheme_apply`` exposes its y = H x and
  ``mscheme_basis`` its determinant order, for the checks against the dense matrix.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
from typing import Dict, List, Optional, Tuple

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


# ----------------------------------------------------------------------------------
# large sectors: matrix-free Lanczos in plain C (oracle/lanczos.c)
# ----------------------------------------------------------------------------------
_HERE = os.path.dirname(os.path.abspath(__file__))
_LANCZOS_SRC = os.path.join(_HERE, "lanczos.c")
_LANCZOS_SO = os.path.join(_HERE, "_build", "liblanczos.so")
_lanczos = None


def build_lanczos(force: bool = False) -> str:
    """Compile oracle/lanczos.c with gcc into oracle/_build/ (when missing or stale)."""
    os.makedirs(os.path.dirname(_LANCZOS_SO), exist_ok=True)
    stale = (force or not os.path.exists(_LANCZOS_SO)
             or os.path.getmtime(_LANCZOS_SO) < os.path.getmtime(_LANCZOS_SRC))
    if stale:
        tmp = _LANCZOS_SO + ".%d.tmp" % os.getpid()
        subprocess.run(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-pthread", "-o", tmp,
                        _LANCZOS_SRC, "-lm"], check=True, capture_output=True)
        os.replace(tmp, _LANCZOS_SO)
    return _LANCZOS_SO


def _lib():
    global _lanczos
    if _lanczos is None:
        lib = ctypes.CDLL(build_lanczos())
        P, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        lib.mscheme_dim.argtypes = [i32, P, P, i32, i32, i32]
        lib.mscheme_dim.restype = i64
        lib.mscheme_basis.argtypes = [i32, P, P, i32, i32, i32, P]
        lib.mscheme_basis.restype = i32
        lib.mscheme_apply.argtypes = [i32, P, P, P, i64, P, P, i32, i32, i32, P, P, i32]
        lib.mscheme_apply.restype = i32
        lib.mscheme_lanczos.argtypes = [i32, P, P, P, i64, P, P, i32, i32, i32, i32,
                                        ctypes.c_double, i32, P, P, P]
        lib.mscheme_lanczos.restype = i32
        _lanczos = lib
    return _lanczos


def _arrays(prob):
    sp = np.ascontiguousarray(prob.species, dtype=np.int8)
    tm = np.ascontiguousarray(prob.two_m, dtype=np.int8)
    eps = np.ascontiguousarray(prob.eps, dtype=np.float64)
    vi = np.ascontiguousarray(prob.v_idx, dtype=np.int32).reshape(-1)
    vv = np.ascontiguousarray(prob.v_val, dtype=np.float64)
    return sp, tm, eps, vi, vv


def _check_hermitian(prob):
    """The row-by-row product uses <s|H|t> = <t|H|s>: the list must hold (kl,ij) with the
    value of every (ij,kl)."""
    table = {}
    for (i, j, k, l), v in zip(prob.v_idx.tolist(), prob.v_val.tolist()):
        table[(i, j, k, l)] = table.get((i, j, k, l), 0.0) + v
    for (i, j, k, l), v in table.items():
        if table.get((k, l, i, j)) != v:
            raise ValueError("two-body list is not Hermitian at %s" % ((i, j, k, l),))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a.size else None


def _sector(prob, Np, Nn, two_M):
    return (prob.Np if Np is None else Np, prob.Nn if Nn is None else Nn,
            prob.two_Mz if two_M is None else two_M)


def mscheme_dim(prob, Np=None, Nn=None, two_M=None) -> int:
    Np, Nn, two_M = _sector(prob, Np, Nn, two_M)
    sp, tm, _, _, _ = _arrays(prob)
    d = _lib().mscheme_dim(int(prob.n_sites), _p(sp), _p(tm), Np, Nn, two_M)
    if d < 0:
        raise ValueError("invalid sector")
    return int(d)


def mscheme_basis(prob, Np=None, Nn=None, two_M=None) -> np.ndarray:
    """Determinant bitmasks (canonical site indices) in the Lanczos vector order."""
    Np, Nn, two_M = _sector(prob, Np, Nn, two_M)
    sp, tm, _, _, _ = _arrays(prob)
    out = np.zeros(mscheme_dim(prob, Np, Nn, two_M), dtype=np.uint64)
    rc = _lib().mscheme_basis(int(prob.n_sites), _p(sp), _p(tm), Np, Nn, two_M, _p(out))
    if rc != 0:
        raise ValueError("invalid sector")
    return out


def mscheme_apply(prob, x, Np=None, Nn=None, two_M=None, threads: Optional[int] = None):
    """y = H x in the basis of ``mscheme_basis``."""
    Np, Nn, two_M = _sector(prob, Np, Nn, two_M)
    _check_hermitian(prob)
    sp, tm, eps, vi, vv = _arrays(prob)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros_like(x)
    rc = _lib().mscheme_apply(int(prob.n_sites), _p(sp), _p(tm), _p(eps), int(vv.shape[0]),
                              _p(vi), _p(vv), Np, Nn, two_M, _p(x), _p(y),
                              int(threads or os.cpu_count() or 1))
    if rc != 0:
        raise ValueError("invalid problem or sector (%d)" % rc)
    return y


def lanczos_lowest(prob, Np=None, Nn=None, two_M=None, tol: float = 1e-9,
                   max_iter: int = 300, threads: Optional[int] = None,
                   want_vector: bool = False):
    """Exact lowest eigenpair of the sector by Lanczos with full reorthogonalisation.

    Returns dict(energy, residual = |H x - E x| recomputed, estimate, steps, dim[, vector
    in the order of ``mscheme_basis``]).  Raises if the tolerance was not reached."""
    Np, Nn, two_M = _sector(prob, Np, Nn, two_M)
    _check_hermitian(prob)
    sp, tm, eps, vi, vv = _arrays(prob)
    dim = mscheme_dim(prob, Np, Nn, two_M)
    vec = np.zeros(dim) if want_vector else np.zeros(0)
    info = np.zeros(2, dtype=np.int64)
    out = np.zeros(3)
    rc = _lib().mscheme_lanczos(int(prob.n_sites), _p(sp), _p(tm), _p(eps), int(vv.shape[0]),
                                _p(vi), _p(vv), Np, Nn, two_M, int(max_iter), float(tol),
                                int(threads or os.cpu_count() or 1), _p(vec) if want_vector
                                else None, _p(info), _p(out))
    if rc < 0:
        raise ValueError("invalid problem or sector (%d)" % rc)
    if rc == 1:
        raise RuntimeError("Lanczos did not reach tol=%g in %d steps (residual %g)"
                           % (tol, max_iter, out[2]))
    res = dict(energy=float(out[0]), residual=float(out[1]), estimate=float(out[2]),
               steps=int(info[0]), dim=int(info[1]))
    if want_vector:
        res["vector"] = vec
    return res
