"""Writes tests/golden/c2_pf4p4n.json: stored expected values of the pf 4p+4n workload
(40 m-scheme sites, 4 protons + 4 neutrons, 2M = 0, m-scheme dimension 1,963,461, random
J-coupled two-body ensemble seed 2), computed by the oracle only (oracle/ and gen/).

1. The exact ground-state energy by the oracle's Lanczos (full reorthogonalisation, FP64,
   residual |H x - E x| <= 1e-9).
2. The chain order: the mutual information I_ij of that exact ground state (all orbital
   pairs, oracle.entropy.mutual_information_dets), then the Fiedler order of its graph
   Laplacian (oracle.ordering.fiedler_order: the paper's spectral ordering with eta = 2).
   The paper takes I_ij from a preparatory DMRG state at small M; the exact state is the
   limit of that state, and using it makes the order independent of the truncation.
3. Two sweeps of the oracle DMRG at M = 256 on the problem in that order, from the seeded
   starting state (gen.initial_mps, M0 = 256, seed 2002), Davidson residual tolerance
   1e-10 (tighter than the default 1e-8, so that the tolerance-level differences between
   two implementations' eigenvectors, which later truncations carry forward, stay far below
   the 1e-8 MeV comparison): every step's energy, Davidson product count, truncation error
   and the kept states per sector of the new block.

    python tests/golden/make_c2.py [--dmrg-only]     (about half an hour on 8 cores;
                                                      --dmrg-only keeps steps 1-2 from the
                                                      stored file)
"""
import dataclasses
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from gen import initial_mps, make_problem                              # noqa: E402
from oracle.dmrg import OracleDMRG                                     # noqa: E402
from oracle.entropy import mutual_information_dets                     # noqa: E402
from oracle.hamiltonian import lanczos_lowest, mscheme_basis           # noqa: E402
from oracle.ordering import fiedler_order, fiedler_vector              # noqa: E402

OUT = os.path.join(HERE, "c2_pf4p4n.json")
SPACE, NP, NN, TM, SEED, M, MPS_SEED, SWEEPS, DAV_TOL = "pf", 4, 4, 0, 2, 256, 2002, 2, 1e-10


def main(dmrg_only=False):
    t0 = time.time()
    prob = make_problem(SPACE, NP, NN, TM, seed=SEED)
    if dmrg_only:
        with open(OUT) as f:
            old = json.load(f)
        exact, mi, order = old["exact"], old["mutual_information"], old["order"]
    else:
        lz = lanczos_lowest(prob, tol=1e-9, max_iter=400, want_vector=True)
        print("lanczos", lz["energy"], lz["residual"], lz["steps"], time.time() - t0, flush=True)
        masks = mscheme_basis(prob)
        I, s = mutual_information_dets(masks, lz["vector"], prob.n_sites)
        v = fiedler_vector(I)
        order = [int(x) for x in fiedler_order(I)]
        w = np.linalg.eigvalsh(np.diag(I.sum(axis=1)) - I)
        print("order", order, "gap", w[2] - w[1], time.time() - t0, flush=True)
        exact = {"energy": lz["energy"], "residual": lz["residual"], "dim": lz["dim"],
                 "lanczos_steps": lz["steps"]}
        mi = {"source": "exact ground state (Lanczos)",
              "fiedler_vector": [float(x) for x in v],
              "laplacian_gap_2_3": float(w[2] - w[1]),
              "s_i": [float(x) for x in s]}
    po = dataclasses.replace(prob, order=np.array(order, dtype=np.int32))
    o = OracleDMRG(po, initial_mps(po, M, MPS_SEED), tol=DAV_TOL)
    sweeps = []
    for sw in range(SWEEPS):
        steps = []
        for r in o.sweep(M):
            steps.append({"p": r.p, "dir": 0 if r.direction == "L" else 1,
                          "energy": r.energy, "n_products": r.n_products,
                          "trunc_err": r.trunc_err,
                          "kept": sorted([list(q) + [int(k)] for q, k in r.kept.items() if k])})
        sweeps.append({"M": M, "steps": steps})
        print("sweep", sw, steps[-1]["energy"], time.time() - t0, flush=True)
    out = {
        "workload": "pf shell, 40 m-scheme sites, 4p+4n, 2M=0, seed %d" % SEED,
        "generator": "gen.make_problem('%s', %d, %d, %d, seed=%d)" % (SPACE, NP, NN, TM, SEED),
        "exact": exact,
        "mutual_information": mi,
        "order": order,
        "dmrg": {"M": M, "mps_seed": MPS_SEED, "dav_tol": DAV_TOL, "sweeps": sweeps},
        "seconds": time.time() - t0,
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", OUT, time.time() - t0)


if __name__ == "__main__":
    main(dmrg_only="--dmrg-only" in sys.argv)
