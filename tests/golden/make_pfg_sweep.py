"""Writes tests/golden/pfg_2p2n_M4.json: stored expected values of one oracle sweep on the
pf+g9/2 space (60 m-scheme sites, the space of the 64Ge calculations) with a target of
nonzero angular-momentum projection: 2 protons + 2 neutrons, 2M_z = 4, random J-coupled
two-body ensemble seed 5, seeded starting state (gen.initial_mps, M0 = 16, seed 5005),
one sweep at M = 16 (114 two-site steps).  Per step: the energy, the truncation error and
the kept states per sector of the new block.  Everything comes from oracle/ and gen/ only.

    python tests/golden/make_pfg_sweep.py          (about a minute on one core)
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from gen import initial_mps, make_problem      # noqa: E402
from oracle.dmrg import OracleDMRG             # noqa: E402

OUT = os.path.join(HERE, "pfg_2p2n_M4.json")
SPACE, NP, NN, TM, SEED, M, MPS_SEED = "pfg", 2, 2, 4, 5, 16, 5005


def compute():
    """The stored record (a dict), computed from oracle/ and gen/."""
    t0 = time.time()
    prob = make_problem(SPACE, NP, NN, TM, seed=SEED)
    o = OracleDMRG(prob, initial_mps(prob, M, MPS_SEED))
    steps = []
    for r in o.sweep(M):
        steps.append({"p": r.p, "dir": 0 if r.direction == "L" else 1, "energy": r.energy,
                      "trunc_err": r.trunc_err,
                      "kept": sorted([list(q) + [int(k)] for q, k in r.kept.items() if k])})
    out = {"workload": "pf+g9/2 shell, 60 m-scheme sites, 2p+2n, 2M_z=4, seed %d" % SEED,
           "generator": "gen.make_problem('%s', %d, %d, %d, seed=%d)" % (SPACE, NP, NN, TM, SEED),
           "M": M, "mps_seed": MPS_SEED, "steps": steps, "seconds": time.time() - t0}
    return out


def main():
    out = compute()
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", OUT, out["steps"][-1]["energy"], out["seconds"])


if __name__ == "__main__":
    main()
