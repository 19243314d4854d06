"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle on identical
seeded inputs.

Tolerances: H_eff psi 1e-12 relative norm (identical, gauge-free inputs at the first
position); Davidson/sweep energies 1e-8 MeV absolute; sector tables and kept dimensions
bit-exact."""
import numpy as np
import pytest

from gen import make_problem, initial_mps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_1507_00161_gb300.build import build
    build()
    import paper_1507_00161_gb300 as P
    assert torch.cuda.is_available()
    return P


CASES = [("p", 2, 2, 12, 5), ("sd", 2, 2, 1, 16), ("sd", 3, 2, 7, 24)]


def _oracle(prob, init):
    from oracle.dmrg import OracleDMRG
    return OracleDMRG(prob, init)


@pytest.mark.parametrize("space,Np,Nn,seed,M0", CASES)
def test_heff_first_position(P, space, Np, Nn, seed, M0):
    prob = make_problem(space, Np, Nn, 1 if (Np + Nn) % 2 else 0, seed=seed)
    init = initial_mps(prob, M0, seed + 100)
    o = _oracle(prob, init)
    sb = o.superblock(1)
    d = P.DMRG(prob)
    d.build_blocks(init)
    lay = d.psi_layout(1)
    ref = [(QL, dL, dR, off) for (QL, QR, dL, dR, off) in sb.layout.blocks]
    assert [tuple(x) for x in lay["qn_left"]] == [r[0] for r in ref]
    assert list(lay["dl"]) == [r[1] for r in ref]
    assert list(lay["dr"]) == [r[2] for r in ref]
    assert list(lay["off"]) == [r[3] for r in ref]
    rng = np.random.default_rng(seed)
    for _ in range(3):
        x = rng.standard_normal(sb.layout.size)
        y_ref = sb.apply(x)
        xd = torch.tensor(x, dtype=torch.float64, device="cuda")
        yd = torch.empty_like(xd)
        d.heff_apply(1, xd, yd)
        y = yd.cpu().numpy()
        assert np.linalg.norm(y - y_ref) <= 1e-12 * np.linalg.norm(y_ref)
    # mixed path (FP32 storage, split-TF32 tensor-core products): FP32-level accuracy
    d.set_options(precision=P.MIXED_FP32)
    d.heff_apply(1, xd, yd)
    y = yd.cpu().numpy()
    assert np.linalg.norm(y - y_ref) <= 2e-6 * np.linalg.norm(y_ref)


@pytest.mark.parametrize("space,Np,Nn,seed,M0", CASES[:2])
def test_davidson_first_step(P, space, Np, Nn, seed, M0):
    prob = make_problem(space, Np, Nn, 0, seed=seed)
    init = initial_mps(prob, M0, seed + 100)
    o = _oracle(prob, init)
    sb = o.superblock(1)
    from oracle.dmrg import davidson
    x0 = np.ones(sb.layout.size)
    e_ref, x_ref, nprod_ref, _ = davidson(sb.apply, sb.diagonal(), x0)
    d = P.DMRG(prob)
    d.build_blocks(init)
    out = torch.empty(sb.layout.size, dtype=torch.float64, device="cuda")
    e, st = d.davidson(1, out=out)
    assert abs(e - e_ref) < 1e-8
    assert st["n_products"] == nprod_ref
    x = out.cpu().numpy()
    assert abs(abs(x @ x_ref) - 1.0) < 1e-8


@pytest.mark.parametrize("space,Np,Nn,seed,M0", CASES)
def test_mixed_energy_is_fp64_accurate(P, space, Np, Nn, seed, M0):
    # mixed path: FP32 products inside Davidson, energy = FP64 Rayleigh quotient of the
    # converged vector; the bound is the FP64 tolerance, not the FP32 one
    prob = make_problem(space, Np, Nn, 1 if (Np + Nn) % 2 else 0, seed=seed)
    init = initial_mps(prob, M0, seed + 100)
    o = _oracle(prob, init)
    sb = o.superblock(1)
    from oracle.dmrg import davidson
    e_ref, _, _, _ = davidson(sb.apply, sb.diagonal(), np.ones(sb.layout.size))
    d = P.DMRG(prob, precision=P.MIXED_FP32)
    d.build_blocks(init)
    e, _ = d.davidson(1)
    assert abs(e - e_ref) < 1e-8, (e, e_ref)


def _compare_sweeps(P, prob, init, M, nsweeps, m_min=0, trunc_target=0.0, n_roots=1):
    from oracle.dmrg import OracleDMRG
    o = OracleDMRG(prob, init, m_min=m_min, trunc_target=trunc_target, n_roots=n_roots)
    d = P.DMRG(prob)
    d.build_blocks(init)
    if trunc_target > 0:
        d.set_dbss(m_min, trunc_target)
    if n_roots > 1:
        d.set_roots(n_roots)
    kept_all = []
    for sw in range(nsweeps):
        ref = o.sweep(M)
        got, e_last = d.sweep(M)
        for r, g in zip(ref, got):
            assert (r.p, 0 if r.direction == "L" else 1) == (g["p"], g["dir"])
            assert abs(r.energy - g["energy"]) < 1e-8, (sw, r.p, r.direction, r.energy, g["energy"])
            if n_roots > 1:
                assert abs(r.energy1 - g["energy1"]) < 1e-8, (sw, r.p, r.direction)
            else:
                assert np.isnan(g["energy1"])
            assert sum(r.kept.values()) == g["kept"], (sw, r.p, r.direction)
            assert abs(r.trunc_err - g["trunc_err"]) < 1e-9
            kept_all.append(g["kept"])
        # block bases after the sweep: sectors and dimensions bit-exact
        for b in range(0, prob.n_sites - 2):
            if b in o.left:
                qn, dims = d.block_sectors(0, b)
                blk = o.left[b]
                assert [tuple(x) for x in qn] == blk.sectors
                assert list(dims) == [blk.dims[q] for q in blk.sectors]
        for b in range(2, prob.n_sites - 1):
            if b in o.right:
                qn, dims = d.block_sectors(1, b)
                blk = o.right[b]
                assert [tuple(x) for x in qn] == blk.sectors
                assert list(dims) == [blk.dims[q] for q in blk.sectors]
    d.kept_all = kept_all
    return o, d


def test_sweeps_p_shell_truncated(P):
    prob = make_problem("p", 2, 2, 0, seed=12)
    _compare_sweeps(P, prob, initial_mps(prob, 5, 5), 8, 3)


def test_sweeps_sd_shell_m64(P):
    """sd shell, 2p+2n (m-scheme dimension 640), M = 64."""
    prob = make_problem("sd", 2, 2, 0, seed=1)
    _compare_sweeps(P, prob, initial_mps(prob, 64, 5), 64, 2)


@pytest.mark.parametrize("space,Np,Nn,seed,M0,M,m_min,target",
                         [("p", 2, 2, 12, 5, 8, 3, 1e-3), ("sd", 2, 2, 1, 16, 64, 16, 1e-4),
                          ("sd", 3, 2, 7, 24, 96, 8, 1e-5)])
def test_dbss_sweeps(P, space, Np, Nn, seed, M0, M, m_min, target):
    """Dynamic block state selection: per-step energies, kept counts, truncation errors
    and block sectors against the oracle's DBSS sweeps."""
    prob = make_problem(space, Np, Nn, 1 if (Np + Nn) % 2 else 0, seed=seed)
    _, d = _compare_sweeps(P, prob, initial_mps(prob, M0, seed + 100), M, 2, m_min, target)
    # the target, not the floor or the ceiling, decided some of the cuts
    assert any(min(m_min, M) < k < M for k in d.kept_all)


def test_dbss_arguments(P):
    prob = make_problem("p", 2, 2, 0, seed=12)
    d = P.DMRG(prob)
    for m_min, target in ((4, 1.0), (4, float("nan")), (0, 1e-3)):
        with pytest.raises(P.DmrgError) as e:
            d.set_dbss(m_min, target)
        assert e.value.code == P.DMRG_EINVAL
    init = initial_mps(prob, 5, 5)
    d.build_blocks(init)
    d.set_dbss(4, 1e-3)
    d.set_dbss(0, 0.0)         # back to a fixed M
    got, _ = d.sweep(8)
    ref = _oracle(prob, init).sweep(8)
    assert [sum(r.kept.values()) for r in ref] == [g["kept"] for g in got]
    assert max(abs(r.energy - g["energy"]) for r, g in zip(ref, got)) < 1e-8


@pytest.mark.parametrize("space,Np,Nn,seed,M0,M,nsweeps",
                         [("p", 2, 2, 12, 5, 8, 3), ("sd", 3, 2, 7, 24, 48, 2)])
def test_two_state_sweeps(P, space, Np, Nn, seed, M0, M, nsweeps):
    """Two lowest states targeted together (averaged density matrix): both energies of
    every step, kept counts, truncation errors and block sectors against the oracle."""
    prob = make_problem(space, Np, Nn, 1 if (Np + Nn) % 2 else 0, seed=seed)
    _compare_sweeps(P, prob, initial_mps(prob, M0, seed + 100), M, nsweeps, n_roots=2)


def test_two_state_full_m_gives_the_two_lowest_exact_states(P):
    from oracle.hamiltonian import ed_lowest
    prob = make_problem("sd", 2, 2, 0, seed=1)
    e0, e1 = ed_lowest(prob, k=2)
    d = P.DMRG(prob)
    d.build_blocks(initial_mps(prob, 8, 5))
    d.set_roots(2)
    d.sweep(400)
    steps, e = d.sweep(400)
    assert abs(steps[-1]["energy"] - e0) < 1e-9 and abs(steps[-1]["energy1"] - e1) < 1e-9
    # the single-state Davidson at the same position agrees on the ground state
    d.set_roots(1)
    e_single, st = d.davidson(1)
    assert abs(e_single - e0) < 1e-9 and np.isnan(st["energy1"])


def test_two_state_arguments(P):
    prob = make_problem("p", 2, 2, 0, seed=12)
    d = P.DMRG(prob)
    for bad in (0, 3):
        with pytest.raises(P.DmrgError) as e:
            d.set_roots(bad)
        assert e.value.code == P.DMRG_EINVAL
    d.set_options(precision=P.MIXED_FP32)
    with pytest.raises(P.DmrgError) as e:
        d.set_roots(2)
    assert e.value.code == P.DMRG_EINVAL
    d.set_options(precision=P.FP64)
    d.set_roots(2)
    with pytest.raises(P.DmrgError) as e:
        d.set_options(precision=P.MIXED_FP32)
    assert e.value.code == P.DMRG_EINVAL
    # dmrg_davidson alone reports both states
    d.build_blocks(initial_mps(prob, 5, 5))
    from oracle.dmrg import davidson_roots
    sb = _oracle(prob, initial_mps(prob, 5, 5)).superblock(1)
    th, _, _, _ = davidson_roots(sb.apply, sb.diagonal(), [np.ones(sb.layout.size)], n_roots=2)
    e, st = d.davidson(1)
    assert abs(e - th[0]) < 1e-8 and abs(st["energy1"] - th[1]) < 1e-8


def test_full_m_reproduces_exact_diagonalization(P):
    from oracle.hamiltonian import ed_lowest
    prob = make_problem("sd", 2, 2, 0, seed=1)
    e0 = ed_lowest(prob)[0]
    d = P.DMRG(prob)
    d.build_blocks(initial_mps(prob, 8, 5))
    steps, e = d.sweep(400)
    assert abs(e - e0) < 1e-9
    assert max(s["trunc_err"] for s in steps) < 1e-12


def test_fused_product_matches_two_stage(P):
    """Superblocks with sectors wider than 32 (chunked path, ring wrap-around), found near
    both ends of the chain after a sweep: the fused H_eff kernel against the independent
    two-stage task-list product (the allocation-free entry point) in FP64, the FP32
    fused product against both, and the energy of the mixed path against FP64 Davidson."""
    prob = make_problem("pf", 4, 4, 0, seed=2)
    d = P.DMRG(prob)
    d.build_blocks(initial_mps(prob, 2048, 2002))
    d.sweep(2048)
    N = prob.n_sites
    rng = np.random.default_rng(19)
    max_dl = max_dr = 0
    checked = 0
    for p in (2, 3, 5, N - 6, N - 4, N - 3):
        lay = d.psi_layout(p)
        x = torch.tensor(rng.standard_normal(lay["size"]), dtype=torch.float64, device="cuda")
        y1 = torch.empty_like(x)
        y2 = torch.empty_like(x)
        d.heff_apply(p, x, y1)
        try:
            d.heff_apply_noalloc(p, x, y2)
        except P.DmrgError:
            continue          # intermediate larger than the fixed scratch
        err = (torch.linalg.norm(y1 - y2) / torch.linalg.norm(y2)).item()
        assert err <= 1e-12, (p, err)
        e64, _ = d.davidson(p, allow_noconv=True)
        d.set_options(precision=P.MIXED_FP32)
        y3 = torch.empty_like(x)
        d.heff_apply(p, x, y3)
        # energy of the mixed path (FP64 Rayleigh quotient) on wide sectors
        e32, _ = d.davidson(p, allow_noconv=True)
        d.set_options(precision=P.FP64)
        err32 = (torch.linalg.norm(y3 - y2) / torch.linalg.norm(y2)).item()
        assert err32 <= 1e-5, (p, err32)
        assert abs(e32 - e64) < 1e-8, (p, e32, e64)
        max_dl = max(max_dl, int(lay["dl"].max()))
        max_dr = max(max_dr, int(lay["dr"].max()))
        checked += 1
    assert checked >= 4
    assert max_dl > 32 and max_dr > 32, (max_dl, max_dr)


def _by_m(prob):
    keys = sorted(range(prob.n_sites),
                  key=lambda s: (int(prob.species[s]), int(prob.two_m[s]), int(prob.orbital[s])))
    return prob.with_order(keys)


@pytest.mark.parametrize("space,Np,Nn,two_M,seed,M0,M,by_m",
                         [("p", 2, 1, 1, 3, 5, 8, True), ("sd", 2, 2, 0, 1, 16, 64, False),
                          ("sd", 3, 2, 3, 7, 24, 48, True)])
def test_dot_rdm_along_a_sweep(P, space, Np, Nn, two_M, seed, M0, M, by_m):
    """Dot-orbital density matrix and entropies after every step of a sweep (both
    directions) against the oracle; chains ordered by m put orbitals of equal (species, m)
    side by side, so the hopping element is exercised."""
    from oracle.dmrg import OracleDMRG
    from oracle.entropy import dot_rdm, entropies
    prob = make_problem(space, Np, Nn, two_M, seed=seed)
    if by_m:
        prob = _by_m(prob)
    init = initial_mps(prob, M0, seed + 100)
    o = OracleDMRG(prob, init, tol=1e-10)
    d = P.DMRG(prob, dav_tol=1e-10)
    d.build_blocks(init)
    with pytest.raises(P.DmrgError):
        d.dot_rdm(1)                       # no wave function held yet
    N = prob.n_sites
    hop = 0.0
    seq = [(p, "L") for p in range(1, N - 2)] + [(p, "R") for p in range(N - 3, 0, -1)]
    for p, dr in seq:
        o.run_step(p, dr, M)
        d.step(p, 0 if dr == "L" else 1, M)
        ref = dot_rdm(o.psi, o.psi_layout, o._prev_L, o._prev_R, o.ch.q[p], o.ch.q[p + 1])
        rho, ent = d.dot_rdm(p)
        assert np.max(np.abs(rho - ref)) < 1e-9, (p, dr, rho, ref)
        assert np.max(np.abs(np.array(ent) - np.array(entropies(ref)))) < 1e-7, (p, dr)
        hop = max(hop, abs(ref[1, 2]))
    assert (hop > 1e-4) == by_m
