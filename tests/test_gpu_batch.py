"""Batch mode: several independent problems swept in lockstep with one fused H_eff
launch per Davidson iteration (replayed as a CUDA graph) give the same energies as
sweeping each problem alone, and the oracle's energies."""
import numpy as np
import pytest

from gen import make_problem, initial_mps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

INSTANCES = [("sd", 2, 2, 1001, 32), ("pf", 2, 3, 1002, 48), ("sd", 3, 3, 1003, 64),
             ("p", 2, 2, 1004, 16)]


@pytest.fixture(scope="module")
def P():
    from paper_1507_00161_gb300.build import build
    build()
    import paper_1507_00161_gb300 as P
    return P


def _contexts(P, precision, own_streams=False):
    out = []
    for space, Np, Nn, seed, M in INSTANCES:
        tm = 0 if (Np + Nn) % 2 == 0 else 1
        prob = make_problem(space, Np, Nn, tm, seed=seed)
        # batch contexts on streams of their own: their host work runs concurrently
        st = torch.cuda.Stream() if own_streams else None
        d = P.DMRG(prob, precision=precision, stream=st)
        d._stream_ref = st
        d.build_blocks(initial_mps(prob, M, seed + 7))
        out.append(d)
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_sweep_equals_single_sweeps(P, precision):
    Ms = [x[4] for x in INSTANCES]
    alone = _contexts(P, precision)
    e_alone = [[d.sweep(M)[1] for _ in range(2)] for d, M in zip(alone, Ms)]
    ctxs = _contexts(P, precision, own_streams=True)
    b = P.Batch(ctxs)
    e1, st1 = b.sweep(Ms)
    e2, st2 = b.sweep(Ms)
    for i in range(len(INSTANCES)):
        assert abs(e1[i] - e_alone[i][0]) < 1e-10, (i, e1[i], e_alone[i][0])
        assert abs(e2[i] - e_alone[i][1]) < 1e-10, (i, e2[i], e_alone[i][1])
    assert st1["products"] > 0 and st1["heff_seconds"] > 0
    b.close()


def test_batch_sweep_equals_oracle(P):
    """FP64 batch of four instances (p and sd shells, even and odd particle numbers) against
    the oracle's sweeps from the same starting states: the energy of each instance after
    each of two sweeps within 1e-8 MeV."""
    from oracle.dmrg import OracleDMRG
    inst = [("p", 2, 2, 1004, 8), ("sd", 2, 2, 1001, 24), ("sd", 3, 2, 1005, 32),
            ("p", 1, 2, 1006, 6)]
    ctxs, oracles, Ms = [], [], []
    for space, Np, Nn, seed, M in inst:
        tm = (Np + Nn) % 2
        prob = make_problem(space, Np, Nn, tm, seed=seed)
        init = initial_mps(prob, M, seed + 7)
        st = torch.cuda.Stream()
        d = P.DMRG(prob, precision=P.FP64, stream=st)
        d._stream_ref = st
        d.build_blocks(init)
        ctxs.append(d)
        oracles.append(OracleDMRG(prob, init))
        Ms.append(M)
    b = P.Batch(ctxs)
    for sweep in range(2):
        e, _ = b.sweep(Ms)
        for i, (o, M) in enumerate(zip(oracles, Ms)):
            ref = o.sweep(M)[-1].energy
            assert abs(e[i] - ref) <= 1e-8, (sweep, i, e[i], ref)
    b.close()
