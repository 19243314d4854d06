"""Host-side checks of the C-ABI library that need no GPU: it builds for sm_103a, loads,
exports every entry point the header declares, and rejects invalid problems before any
device work."""
import ctypes
import os
import re

import numpy as np
import pytest

from gen import make_problem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1507_00161_gb300.build import build
    build()
    import paper_1507_00161_gb300 as P
    return P


def test_header_symbols_exported(lib):
    hdr = open(os.path.join(ROOT, "include", "dmrg.h")).read()
    declared = set(re.findall(r"^(?:int|int64_t|const char\*)\s+(dmrg_\w+)\(", hdr, re.M))
    assert "dmrg_batch_sweep" in declared
    assert declared == set(lib.EXPORTED)
    so = lib.load_library()
    for name in declared:
        assert hasattr(so, name), name


def _bad(lib, prob, **kw):
    with pytest.raises(lib.DmrgError) as e:
        lib.DMRG(prob, **kw)
    return e.value.code


def test_rejects_invalid_problems(lib):
    p = make_problem("p", 2, 2, 0, seed=3)
    # order not a permutation
    q = p.with_order(np.arange(p.n_sites))
    q.order = q.order.copy()
    q.order[0] = q.order[1]
    assert _bad(lib, q) == lib.DMRG_EINVAL
    # two-body entry that breaks 2M conservation
    q = p.with_order(p.order)
    q.v_idx = p.v_idx.copy()
    q.v_val = p.v_val.copy()
    i = int(np.argmax(q.v_idx[:, 0] != q.v_idx[:, 2]))
    q.v_idx[i, 0], q.v_idx[i, 1] = 0, 1
    q.v_idx[i, 2], q.v_idx[i, 3] = 0, 3
    assert _bad(lib, q) == lib.DMRG_EINVAL
    # non-Hermitian list
    q = p.with_order(p.order)
    q.v_val = p.v_val.copy()
    off = np.nonzero((p.v_idx[:, 0] != p.v_idx[:, 2]) | (p.v_idx[:, 1] != p.v_idx[:, 3]))[0]
    q.v_val[off[0]] += 1.0
    assert _bad(lib, q) == lib.DMRG_EINVAL
    # bad Davidson options
    assert _bad(lib, p, dav_max_sub=2) == lib.DMRG_EINVAL


@pytest.mark.parametrize("space,Np,Nn,seed", [("sd", 2, 2, 1), ("p", 2, 3, 4), ("pf", 4, 4, 2)])
def test_operator_partition_counts_match_oracle(lib, space, Np, Nn, seed):
    """The library's host-side operator partition has, at every bond, exactly as many
    operator products as the oracle's (both prune labels that cannot connect the vacuum to
    the full Hamiltonian), on a shuffled chain order: the number of superblock terms the
    paper's two-block Hamiltonian sums over."""
    from oracle.hamiltonian import ChainHamiltonian
    from oracle.mpo import MPO
    p = make_problem(space, Np, Nn, (Np + Nn) % 2, seed=seed)
    rng = np.random.default_rng(seed)
    p = p.with_order(rng.permutation(p.n_sites))
    d = lib.DMRG(p)     # validates and builds the partition; no device work
    m = MPO(ChainHamiltonian(p))
    got = [d.partition_terms(b) for b in range(p.n_sites - 1)]
    ref = [m.n_terms(b) for b in range(p.n_sites - 1)]
    d.close()
    assert got == ref
    assert max(got) > 2 * p.n_sites     # pair operators appear in the middle
    with pytest.raises(lib.DmrgError):
        d2 = lib.DMRG(p)
        try:
            d2.partition_terms(p.n_sites - 1)
        finally:
            d2.close()
