"""GPU parity on the pf+g9/2 space (60 m-scheme sites, the space of the 64Ge calculations),
through the C-ABI, with targets of nonzero angular-momentum projection.

* pf+g9/2 2p+2n, 2M_z = 4 (seed 5), one FP64 sweep at M = 16 from the seeded starting state
  against the oracle's sweep stored in tests/golden/pfg_2p2n_M4.json (written by
  tests/golden/make_pfg_sweep.py from oracle/ only): all 114 steps' energies within
  1e-8 MeV, truncation errors within 1e-10, the kept states per sector bit-exact.
* The pf+g9/2 12p+12n workload (2M_z = 0 and 4, seed 4) at M = 128: mixed and FP64 Davidson
  on identical superblocks along the first steps of a sweep, energies within 1e-8 MeV; every
  sector of every new left block (sites 0..p) is completed to the target by some state of
  the sites p+1..59 (Fock-space counting), and at most M states are kept.
"""
import json
import os

import numpy as np
import pytest

from gen import make_problem, initial_mps
from gen.shell import count_sector_dims

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "pfg_2p2n_M4.json")


@pytest.fixture(scope="module")
def P():
    from paper_1507_00161_gb300.build import build
    build()
    import paper_1507_00161_gb300 as P
    assert torch.cuda.is_available()
    return P


def test_pfg_sweep_matches_oracle(P):
    with open(GOLDEN) as f:
        g = json.load(f)
    prob = make_problem("pfg", 2, 2, 4, seed=5)
    assert prob.n_sites == 60
    M = g["M"]
    d = P.DMRG(prob)
    d.build_blocks(initial_mps(prob, M, g["mps_seed"]))
    N = prob.n_sites
    seq = [(p, 0) for p in range(1, N - 2)] + [(p, 1) for p in range(N - 3, 0, -1)]
    assert len(seq) == len(g["steps"])
    worst = 0.0
    for (p, dr), ref in zip(seq, g["steps"]):
        assert (ref["p"], ref["dir"]) == (p, dr)
        st = d.step(p, dr, M)
        worst = max(worst, abs(st["energy"] - ref["energy"]))
        assert abs(st["energy"] - ref["energy"]) <= 1e-8, (p, dr)
        assert abs(st["trunc_err"] - ref["trunc_err"]) <= 1e-10, (p, dr)
        qn, dims = d.block_sectors(dr, p)
        kept = sorted([list(map(int, q)) + [int(m)] for q, m in zip(qn, dims) if m])
        assert kept == ref["kept"], (p, dr)
    d.close()
    print("[pfg 2p+2n 2M=4] worst step energy difference vs oracle: %.2e MeV" % worst)


@pytest.mark.parametrize("two_mz", [0, 4])
def test_pfg_workload_mixed_equals_fp64_on_identical_superblocks(P, two_mz):
    prob = make_problem("pfg", 12, 12, two_mz, seed=4)
    M = 128
    sp = [int(prob.species[s]) for s in prob.order]
    tm = [int(prob.two_m[s]) for s in prob.order]
    d = P.DMRG(prob)
    d.build_blocks(initial_mps(prob, M, 4004))
    for p in range(1, 13):
        if p % 4 == 0:
            d.set_options(precision=P.MIXED_FP32)
            e_m, st_m = d.davidson(p)
            d.set_options(precision=P.FP64)
            e_d, st_d = d.davidson(p)
            assert st_m["converged"] and st_d["converged"]
            assert abs(e_m - e_d) <= 1e-8, (p, e_m, e_d)
        d.step(p, 0, M)
        qn, dims = d.block_sectors(0, p)
        rest = count_sector_dims(sp[p + 1:], tm[p + 1:])
        for (a, b, m), k in zip(np.asarray(qn).tolist(), dims.tolist()):
            if k:
                assert rest.get((12 - a, 12 - b, two_mz - m), 0) > 0, (p, a, b, m)
        assert 0 < int(np.sum(dims)) <= M
    d.close()
