"""Writes tests/golden/heff_pos1_<case>.json: the oracle's H_eff psi at the first two-site
position (identical, gauge-free inputs: the blocks come from the seeded starting state
only) for the two pf-shell workloads whose full products are too slow to recompute inside
a test on the CPU:
  pf4p4n: pf shell, 4p+4n, 2M=0, seed 2, starting state M0 = 1024, seed 2002;
  pf8p8n: pf shell, 8p+8n, 2M=0, seed 3, starting state M0 = 4096, seed 3003 (the
          headline workload).
Input: x = numpy.random.default_rng(7).standard_normal(size).  Stored: the layout of the
wave function (left sector, d_L, d_R, offset per block), |y|, y at 4096 evenly spaced
indices, and <v_j, y> for v_j = default_rng(100 + j).standard_normal(size), j = 0..3.
Everything comes from oracle/ and gen/ only.

    python tests/golden/make_heff_pos1.py pf4p4n|pf8p8n
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from gen import initial_mps, make_problem      # noqa: E402
from oracle.dmrg import OracleDMRG             # noqa: E402

CASES = {"pf4p4n": ("pf", 4, 4, 0, 2, 1024, 2002), "pf8p8n": ("pf", 8, 8, 0, 3, 4096, 3003)}


def compute(name):
    """The stored record of one case (a dict), computed from oracle/ and gen/."""
    space, Np, Nn, tM, seed, M0, mseed = CASES[name]
    t0 = time.time()
    prob = make_problem(space, Np, Nn, tM, seed=seed)
    o = OracleDMRG(prob, initial_mps(prob, M0, mseed))
    sb = o.superblock(1)
    t1 = time.time()
    size = sb.layout.size
    x = np.random.default_rng(7).standard_normal(size)
    y = sb.apply(x)
    t2 = time.time()
    idx = np.unique(np.linspace(0, size - 1, 4096).astype(np.int64))
    out = {
        "case": name, "space": space, "Np": Np, "Nn": Nn, "two_Mz": tM, "seed": seed, "M0": M0,
        "mps_seed": mseed, "position": 1, "size": int(size),
        "blocks": [[list(QL), int(dL), int(dR), int(off)]
                   for (QL, QR, dL, dR, off) in sb.layout.blocks],
        "norm": float(np.linalg.norm(y)),
        "sample_index": [int(i) for i in idx],
        "sample_value": [float(y[i]) for i in idx],
        "projections": [float(np.random.default_rng(100 + j).standard_normal(size) @ y)
                        for j in range(4)],
        "seconds": {"setup": t1 - t0, "product": t2 - t1},
    }
    return out


def main(name):
    out = compute(name)
    with open(os.path.join(HERE, "heff_pos1_%s.json" % name), "w") as f:
        json.dump(out, f)
    print(name, out["seconds"], out["size"])


if __name__ == "__main__":
    main(sys.argv[1])
