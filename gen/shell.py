"""Shell-model problems of Eq. (1): valence spaces, m-scheme sites, and a J-coupled
two-body random ensemble converted to antisymmetrised m-scheme matrix elements.

Conventions (the paper states Eq. (1) but no ensemble and no sign convention):

* Sites are m-scheme spin-orbitals alpha = (n, l, j, m, tau_z) (Eq. 1).  Canonical site
  index: orbitals in the space's order, inside an orbital 2m ascending, and for each
  (orbital, m) first the proton then the neutron site ("interleaved p/n").
* The Hamiltonian handed to both the oracle and the CUDA library is

      H = sum_i eps_i n_i + sum_{i<j, k<l} Vbar[ij,kl] c+_i c+_j c_l c_k ,

  with the list holding both (ij,kl) and (kl,ij).  Relative to the paper's
  "- 1/2 sum V c+ c+ c c" this is Vbar[ij,kl] = -(V_ijkl - V_ijlk); for a zero-mean
  Gaussian ensemble the sign flip does not change the distribution.
* Random ensemble (recipe of the synthetic workloads): one eps per j-orbital, shared by
  protons and neutrons, eps ~ U[0, 4) MeV, drawn first in orbital order; then Gaussian
  J-coupled two-body matrix elements with sigma = 1 MeV, channel pp(=nn, one shared draw)
  then pn, J ascending, bra pair (a,b) then ket pair (c,d) >= (a,b) lexicographically,
  parity (-1)^(la+lb) = (-1)^(lc+ld) enforced, a <= b and J even when a == b for like
  particles, all ordered (a_p, b_n) for pn.  The J matrices are symmetric.
* J -> m conversion with Clebsch-Gordan coefficients (Racah's closed formula, exact
  rational arithmetic, rounded once to FP64):
      like particles: Vbar(a alpha b beta, c gamma d delta)
          = sqrt((1+d_ab)(1+d_cd)) sum_J <ja ma jb mb|J M><jc mc jd md|J M> V_J(ab,cd)
      pn:   V(a_p b_n, c_p d_n) = sum_J <..|J M><..|J M> V^pn_J(ab,cd), reordered to the
            canonical i<j, k<l form with the fermionic sign of the reordering.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from fractions import Fraction
from functools import lru_cache
from typing import Dict, List, Sequence, Tuple

import numpy as np

from .prng import SplitMix64


@dataclass(frozen=True)
class Orbital:
    name: str
    n: int
    l: int
    two_j: int


_ORB = {
    "s1/2": Orbital("s1/2", 1, 0, 1),
    "p3/2": Orbital("p3/2", 0, 1, 3),
    "p1/2": Orbital("p1/2", 0, 1, 1),
    "d5/2": Orbital("d5/2", 0, 2, 5),
    "d3/2": Orbital("d3/2", 0, 2, 3),
    "f7/2": Orbital("f7/2", 0, 3, 7),
    "f5/2": Orbital("f5/2", 0, 3, 5),
    "p3/2'": Orbital("p3/2", 1, 1, 3),
    "p1/2'": Orbital("p1/2", 1, 1, 1),
    "g9/2": Orbital("g9/2", 0, 4, 9),
}


@dataclass(frozen=True)
class Space:
    name: str
    orbitals: Tuple[Orbital, ...]

    @property
    def states_per_species(self) -> int:
        return sum(o.two_j + 1 for o in self.orbitals)

    @property
    def n_sites(self) -> int:
        return 2 * self.states_per_species


SPACES: Dict[str, Space] = {
    # toy spaces for brute-force pins
    "p": Space("p", (_ORB["p3/2"], _ORB["p1/2"])),
    "f7": Space("f7", (_ORB["f7/2"],)),
    "p3": Space("p3", (_ORB["p3/2"],)),
    # sd shell (28Si-like, Section on 28Si / USD)
    "sd": Space("sd", (_ORB["d5/2"], _ORB["s1/2"], _ORB["d3/2"])),
    # pf shell (56Ni / 64Ge with KB3 / GXPF1A)
    "pf": Space("pf", (_ORB["f7/2"], _ORB["p3/2'"], _ORB["f5/2"], _ORB["p1/2'"])),
    # pf + g9/2 (64Ge extended space)
    "pfg": Space("pfg", (_ORB["f7/2"], _ORB["p3/2'"], _ORB["f5/2"], _ORB["p1/2'"],
                         _ORB["g9/2"])),
}


def site_table(space: Space):
    """Canonical site list: dicts with species (0=p,1=n), orbital index, two_j, l, two_m."""
    sites = []
    for a, o in enumerate(space.orbitals):
        for two_m in range(-o.two_j, o.two_j + 1, 2):
            for sp in (0, 1):
                sites.append(dict(species=sp, orbital=a, two_j=o.two_j, l=o.l, two_m=two_m))
    return sites


def _site_index(space: Space):
    idx = {}
    for s, st in enumerate(site_table(space)):
        idx[(st["species"], st["orbital"], st["two_m"])] = s
    return idx


# ----------------------------------------------------------------------------------
# Clebsch-Gordan coefficients, Racah's formula (all arguments doubled integers)
# ----------------------------------------------------------------------------------
@lru_cache(maxsize=None)
def cg(tj1: int, tm1: int, tj2: int, tm2: int, tJ: int, tM: int) -> float:
    """<j1 m1 j2 m2 | J M> with doubled arguments, Racah's closed formula, exact in
    rational arithmetic up to the final square root."""
    if tm1 + tm2 != tM:
        return 0.0
    if abs(tm1) > tj1 or abs(tm2) > tj2 or abs(tM) > tJ:
        return 0.0
    if (tj1 + tm1) % 2 or (tj2 + tm2) % 2 or (tJ + tM) % 2:
        return 0.0
    if tJ < abs(tj1 - tj2) or tJ > tj1 + tj2 or (tj1 + tj2 + tJ) % 2:
        return 0.0
    f = math.factorial
    a = (tJ + tj1 - tj2) // 2
    b = (tJ - tj1 + tj2) // 2
    c = (tj1 + tj2 - tJ) // 2
    d = (tj1 + tj2 + tJ) // 2 + 1
    pre = Fraction((tJ + 1) * f(a) * f(b) * f(c), f(d))
    pre *= (f((tJ + tM) // 2) * f((tJ - tM) // 2) * f((tj1 - tm1) // 2) * f((tj1 + tm1) // 2)
            * f((tj2 - tm2) // 2) * f((tj2 + tm2) // 2))
    s = Fraction(0)
    k = 0
    while True:
        args = [k, c - k, (tj1 - tm1) // 2 - k, (tj2 + tm2) // 2 - k,
                (tJ - tj2 + tm1) // 2 + k, (tJ - tj1 - tm2) // 2 + k]
        if c - k < 0 or (tj1 - tm1) // 2 - k < 0 or (tj2 + tm2) // 2 - k < 0:
            break
        if min(args) >= 0:
            den = 1
            for x in args:
                den *= f(x)
            s += Fraction((-1) ** k, den)
        k += 1
    val = math.sqrt(pre.numerator / pre.denominator) if pre > 0 else 0.0
    # sign and magnitude of s exactly, then combine
    return float(s) * val if s != 0 else 0.0


# ----------------------------------------------------------------------------------
# problem container
# ----------------------------------------------------------------------------------
@dataclass
class Problem:
    space: Space
    species: np.ndarray      # int8 [N]
    orbital: np.ndarray      # int16 [N]
    two_j: np.ndarray        # int8 [N]
    l: np.ndarray            # int8 [N]
    two_m: np.ndarray        # int8 [N]
    eps: np.ndarray          # float64 [N]
    v_idx: np.ndarray        # int32 [n_v, 4]  (i<j, k<l), both (ij,kl) and (kl,ij)
    v_val: np.ndarray        # float64 [n_v]
    order: np.ndarray        # int32 [N] chain position -> site
    Np: int
    Nn: int
    two_Mz: int
    label: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_sites(self) -> int:
        return int(self.species.shape[0])

    def with_order(self, order) -> "Problem":
        order = np.asarray(order, dtype=np.int32)
        assert sorted(order.tolist()) == list(range(self.n_sites))
        return Problem(self.space, self.species, self.orbital, self.two_j, self.l,
                       self.two_m, self.eps, self.v_idx, self.v_val, order, self.Np,
                       self.Nn, self.two_Mz, self.label, dict(self.meta))

    def with_target(self, Np, Nn, two_Mz) -> "Problem":
        return Problem(self.space, self.species, self.orbital, self.two_j, self.l,
                       self.two_m, self.eps, self.v_idx, self.v_val, self.order, Np, Nn,
                       two_Mz, self.label, dict(self.meta))


def _like_pairs(space: Space, tJ: int):
    out = []
    orbs = space.orbitals
    for a in range(len(orbs)):
        for b in range(a, len(orbs)):
            ja, jb = orbs[a].two_j, orbs[b].two_j
            if tJ < abs(ja - jb) or tJ > ja + jb:
                continue
            if a == b and (tJ // 2) % 2 == 1:
                continue
            out.append((a, b))
    return out


def _pn_pairs(space: Space, tJ: int):
    out = []
    orbs = space.orbitals
    for a in range(len(orbs)):
        for b in range(len(orbs)):
            ja, jb = orbs[a].two_j, orbs[b].two_j
            if abs(ja - jb) <= tJ <= ja + jb:
                out.append((a, b))
    return out


def draw_tbre(space: Space, seed: int, sigma: float = 1.0, eps_range=(0.0, 4.0)):
    """Draw (eps per orbital, V_J pp dict, V_J pn dict) from the seeded ensemble.

    Dict keys are (2J, a, b, c, d) and hold both (ab,cd) and (cd,ab)."""
    rng = SplitMix64(seed)
    orbs = space.orbitals
    eps_orb = [eps_range[0] + (eps_range[1] - eps_range[0]) * rng.uniform() for _ in orbs]
    jmax2 = 2 * max(o.two_j for o in orbs)
    vpp, vpn = {}, {}
    for chan, pairs_of, store in (("pp", _like_pairs, vpp), ("pn", _pn_pairs, vpn)):
        for tJ in range(0, jmax2 + 1, 2):
            pairs = pairs_of(space, tJ)
            for x, (a, b) in enumerate(pairs):
                for (c, d) in pairs[x:]:
                    if (orbs[a].l + orbs[b].l) % 2 != (orbs[c].l + orbs[d].l) % 2:
                        continue
                    g = sigma * rng.gauss()
                    store[(tJ, a, b, c, d)] = g
                    store[(tJ, c, d, a, b)] = g
    return eps_orb, vpp, vpn


def mscheme_from_j(space: Space, vpp: dict, vpn: dict):
    """J-coupled matrix elements -> canonical m-scheme list {(i,j,k,l): Vbar}."""
    idx = _site_index(space)
    orbs = space.orbitals
    acc: Dict[Tuple[int, int, int, int], float] = {}

    def ms(a):
        tj = orbs[a].two_j
        return range(-tj, tj + 1, 2)

    for (tJ, a, b, c, d), val in vpp.items():
        ja, jb, jc, jd = (orbs[x].two_j for x in (a, b, c, d))
        fac = math.sqrt((2.0 if a == b else 1.0) * (2.0 if c == d else 1.0))
        for ma in ms(a):
            for mb in ms(b):
                if a == b and ma >= mb:
                    continue
                tM = ma + mb
                c1 = cg(ja, ma, jb, mb, tJ, tM)
                if c1 == 0.0:
                    continue
                for mc in ms(c):
                    md = tM - mc
                    if abs(md) > jd or (c == d and mc >= md):
                        continue
                    c2 = cg(jc, mc, jd, md, tJ, tM)
                    if c2 == 0.0:
                        continue
                    for sp in (0, 1):
                        key = (idx[(sp, a, ma)], idx[(sp, b, mb)], idx[(sp, c, mc)],
                               idx[(sp, d, md)])
                        acc[key] = acc.get(key, 0.0) + fac * c1 * c2 * val
    for (tJ, a, b, c, d), val in vpn.items():
        ja, jb, jc, jd = (orbs[x].two_j for x in (a, b, c, d))
        for ma in ms(a):
            for mb in ms(b):
                tM = ma + mb
                c1 = cg(ja, ma, jb, mb, tJ, tM)
                if c1 == 0.0:
                    continue
                for mc in ms(c):
                    md = tM - mc
                    if abs(md) > jd:
                        continue
                    c2 = cg(jc, mc, jd, md, tJ, tM)
                    if c2 == 0.0:
                        continue
                    i0, j0 = idx[(0, a, ma)], idx[(1, b, mb)]
                    k0, l0 = idx[(0, c, mc)], idx[(1, d, md)]
                    s = 1.0
                    if i0 > j0:
                        i0, j0, s = j0, i0, -s
                    if k0 > l0:
                        k0, l0, s = l0, k0, -s
                    key = (i0, j0, k0, l0)
                    acc[key] = acc.get(key, 0.0) + s * c1 * c2 * val
    return acc


def _assemble(space: Space, eps_orb, acc, Np, Nn, two_Mz, label, meta) -> Problem:
    sites = site_table(space)
    N = len(sites)
    # exact Hermiticity: (kl,ij) takes the value accumulated for (ij,kl) when ij < kl
    for key in list(acc):
        i, j, k, l = key
        if (i, j) < (k, l):
            acc[(k, l, i, j)] = acc[key]
    keys = sorted(k for k, v in acc.items() if v != 0.0)
    v_idx = np.array(keys, dtype=np.int32).reshape(-1, 4)
    v_val = np.array([acc[k] for k in keys], dtype=np.float64)
    return Problem(
        space=space,
        species=np.array([s["species"] for s in sites], dtype=np.int8),
        orbital=np.array([s["orbital"] for s in sites], dtype=np.int16),
        two_j=np.array([s["two_j"] for s in sites], dtype=np.int8),
        l=np.array([s["l"] for s in sites], dtype=np.int8),
        two_m=np.array([s["two_m"] for s in sites], dtype=np.int8),
        eps=np.array([eps_orb[s["orbital"]] for s in sites], dtype=np.float64),
        v_idx=v_idx, v_val=v_val, order=np.arange(N, dtype=np.int32),
        Np=Np, Nn=Nn, two_Mz=two_Mz, label=label, meta=meta)


def make_problem(space_name: str, Np: int, Nn: int, two_Mz: int = 0, seed: int = 1,
                 sigma: float = 1.0, label: str = "") -> Problem:
    """Random J-coupled two-body ensemble on a valence space, in m-scheme."""
    space = SPACES[space_name]
    eps_orb, vpp, vpn = draw_tbre(space, seed, sigma)
    acc = mscheme_from_j(space, vpp, vpn)
    return _assemble(space, eps_orb, acc, Np, Nn, two_Mz,
                     label or f"{space_name}-{Np}p{Nn}n-M{two_Mz}-s{seed}",
                     dict(seed=seed, sigma=sigma, eps_orb=eps_orb))


def problem_from_j(space_name: str, eps_orb, vpp: dict, vpn: dict, Np: int, Nn: int,
                   two_Mz: int = 0, label: str = "") -> Problem:
    """Problem from explicit J-coupled matrix elements (keys (2J,a,b,c,d), both orders)."""
    space = SPACES[space_name]
    acc = mscheme_from_j(space, vpp, vpn)
    return _assemble(space, list(eps_orb), acc, Np, Nn, two_Mz, label or "custom", {})


def pairing_problem(space_name: str, G: float, Np: int, Nn: int) -> Problem:
    """Single-j pairing Hamiltonian -G S+S per species: only V_{J=0}(jj,jj) = -G*Omega,
    Omega = (2j+1)/2, no pn interaction, eps = 0."""
    space = SPACES[space_name]
    assert len(space.orbitals) == 1
    omega = (space.orbitals[0].two_j + 1) / 2.0
    vpp = {(0, 0, 0, 0, 0): -G * omega}
    return problem_from_j(space_name, [0.0], vpp, {}, Np, Nn, 0, f"pairing-{space_name}")


# ----------------------------------------------------------------------------------
# sector counting (integer): full Fock-space dimensions per (Np, Nn, 2M)
# ----------------------------------------------------------------------------------
def count_sector_dims(species: Sequence[int], two_m: Sequence[int]) -> Dict[tuple, int]:
    """Number of occupation-number states of the given sites per (Np, Nn, 2M)."""
    cnt = {(0, 0, 0): 1}
    for sp, tm in zip(species, two_m):
        new = dict(cnt)
        for (a, b, m), c in cnt.items():
            key = (a + 1, b, m + tm) if sp == 0 else (a, b + 1, m + tm)
            new[key] = new.get(key, 0) + c
        cnt = new
    return cnt


def mscheme_dimension(space_name: str, Np: int, Nn: int, two_Mz: int) -> int:
    space = SPACES[space_name]
    sites = site_table(space)
    d = count_sector_dims([s["species"] for s in sites], [s["two_m"] for s in sites])
    return d.get((Np, Nn, two_Mz), 0)
