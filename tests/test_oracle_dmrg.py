"""Pins of the oracle two-site DMRG."""
import numpy as np
import pytest

from gen import make_problem, initial_mps
from oracle.hamiltonian import ChainHamiltonian, ed_lowest, fock_matrix
from oracle.dmrg import OracleDMRG, enlarge_left, enlarge_right


@pytest.fixture(scope="module")
def ptoy():
    p = make_problem("p", 2, 2, 0, seed=12)
    return p, ed_lowest(p)[0]


def test_full_m_reproduces_exact(ptoy):
    """Large enough M converges to the full CI energy (two-site DMRG, full M)."""
    p, e0 = ptoy
    d = OracleDMRG(p, initial_mps(p, 6, 5))
    res = d.sweep(10 ** 6)
    assert abs(res[-1].energy - e0) < 1e-10
    assert max(r.trunc_err for r in res) < 1e-13
    res = d.sweep(10 ** 6)
    # with complete bases the predicted wave function is already the eigenvector
    assert all(r.n_products == 1 for r in res)
    assert all(abs(r.energy - e0) < 1e-10 for r in res)


def test_full_m_sd_shell():
    p = make_problem("sd", 2, 2, 0, seed=1)
    e0 = ed_lowest(p)[0]
    d = OracleDMRG(p, initial_mps(p, 8, 5))
    res = d.sweep(400)       # >= every bond's full compatible dimension
    assert abs(res[-1].energy - e0) < 1e-10


def test_variational_and_monotone_in_m(ptoy):
    p, e0 = ptoy
    d = OracleDMRG(p, initial_mps(p, 3, 7))
    last = None
    for M in (3, 6, 12):
        for _ in range(2):
            res = d.sweep(M)
        es = [r.energy for r in res]
        assert min(es) >= e0 - 1e-10
        if last is not None:
            assert res[-1].energy <= last + 1e-9
        last = res[-1].energy


def _basis_vectors(d, p):
    """Explicit Fock-space vectors of the enlarged left and right spaces at position p."""
    ch = d.ch
    Lv = {}
    e = enlarge_left(d.left[-1] if False else None, 0, d.mpo, ch) if False else None
    # left blocks 0..p-1
    vec = {(0, 0, 0): np.ones((1, 1))}
    for b in range(0, p):
        blk_prev = None if b == 0 else d.left[b - 1]
        from oracle.dmrg import vacuum
        enl = enlarge_left(vacuum(1, 0) if b == 0 else d.left[b - 1], b, d.mpo, ch)
        ev = {}
        for Q in enl.sectors:
            cols = []
            for (sg, q, off, dd) in enl.pieces[Q]:
                e_s = np.eye(2)[:, sg]
                for i in range(dd):
                    cols.append(np.kron(vec[q][:, i], e_s))
            ev[Q] = np.stack(cols, axis=1)
        vec = {Q: ev[Q] @ d.UL[b][Q] for Q in d.UL[b]}
    Lenl = enlarge_left(d.left[p - 1], p, d.mpo, ch)
    Lv = {}
    for Q in Lenl.sectors:
        cols = []
        for (sg, q, off, dd) in Lenl.pieces[Q]:
            for i in range(dd):
                cols.append(np.kron(vec[q][:, i], np.eye(2)[:, sg]))
        Lv[Q] = np.stack(cols, axis=1)
    N = ch.N
    rvec = {(0, 0, 0): np.ones((1, 1))}
    from oracle.dmrg import vacuum
    for b in range(N - 2, p, -1):
        enl = enlarge_right(vacuum(1, 0) if b == N - 2 else d.right[b + 1], b + 1, d.mpo, ch)
        ev = {}
        for Q in enl.sectors:
            cols = []
            for (sg, q, off, dd) in enl.pieces[Q]:
                for i in range(dd):
                    cols.append(np.kron(np.eye(2)[:, sg], rvec[q][:, i]))
            ev[Q] = np.stack(cols, axis=1)
        rvec = {Q: ev[Q] @ d.UR[b][Q] for Q in d.UR[b]}
    Renl = enlarge_right(d.right[p + 1], p + 1, d.mpo, ch)
    Rv = {}
    for Q in Renl.sectors:
        cols = []
        for (sg, q, off, dd) in Renl.pieces[Q]:
            for i in range(dd):
                cols.append(np.kron(np.eye(2)[:, sg], rvec[q][:, i]))
        Rv[Q] = np.stack(cols, axis=1)
    return Lv, Rv


@pytest.mark.parametrize("p_at", [2, 5, 8])
def test_heff_equals_projected_hamiltonian(p_at):
    """At truncated M, H_eff from renormalized block operators equals P^T H P with P the
    explicit superblock basis in the full Fock space (pins enlargement, Jordan-Wigner
    signs, renormalization and the wave-function layout)."""
    p = make_problem("p", 2, 2, 0, seed=12)
    d = OracleDMRG(p, initial_mps(p, 5, 5))
    d.sweep(5)
    for q in range(1, p_at):
        d.run_step(q, "L", 5)
    sb = d.superblock(p_at)
    Lv, Rv = _basis_vectors(d, p_at)
    cols = []
    for (QL, QR, dL, dR, off) in sb.layout.blocks:
        for i in range(dL):
            for j in range(dR):
                cols.append(np.kron(Lv[QL][:, i], Rv[QR][:, j]))
    P = np.stack(cols, axis=1)
    assert np.allclose(P.T @ P, np.eye(P.shape[1]), atol=1e-12)
    H = fock_matrix(d.ch)
    Hp = P.T @ (H @ P)
    n = sb.layout.size
    He = np.stack([sb.apply(np.eye(n)[:, c]) for c in range(n)], axis=1)
    assert np.max(np.abs(He - Hp)) < 1e-11
    # Hermitian, and Davidson reaches the lowest eigenvalue of the dense H_eff
    assert np.max(np.abs(He - He.T)) < 1e-12
    from oracle.dmrg import davidson
    th, x, _, _ = davidson(sb.apply, sb.diagonal(), np.ones(n), tol=1e-10)
    assert abs(th - np.linalg.eigvalsh(He)[0]) < 1e-10
    assert np.allclose(sb.diagonal(), np.diag(He), atol=1e-12)


# ---------------------------------------------------------------------------------------
# dynamic block state selection (DBSS): kept count set by an a priori truncation error
# ---------------------------------------------------------------------------------------
def _psi_at(p_at=4):
    from oracle.dmrg import davidson
    p = make_problem("p", 2, 2, 0, seed=12)
    d = OracleDMRG(p, initial_mps(p, 6, 5))
    d.sweep(6)
    for q in range(1, p_at):
        d.run_step(q, "L", 6)
    sb = d.superblock(p_at)
    _, x, _, _ = davidson(sb.apply, sb.diagonal(), np.ones(sb.layout.size), tol=1e-10)
    return sb, x


def _schmidt_weights(sb, x):
    """Weights of the enlarged-left states from the singular values of the wave-function
    blocks (one block per left sector), zero-padded to each sector's dimension."""
    w = []
    for (QL, QR, dL, dR, off) in sb.layout.blocks:
        s = np.linalg.svd(x[off:off + dL * dR].reshape(dL, dR), compute_uv=False)
        w.extend(s ** 2)
    n_zero = sum(sb.L.dims.values()) - len(w)
    return np.sort(np.concatenate([w, np.zeros(n_zero)]))[::-1]


@pytest.mark.parametrize("target", [3e-2, 1e-3, 1e-5])
def test_dbss_keeps_the_fewest_states_within_the_target(target):
    from oracle.dmrg import truncate
    sb, x = _psi_at()
    w = _schmidt_weights(sb, x)
    D = len(w)
    for m_min, M in ((1, D), (3, D), (2, 9)):
        # brute force on the definition: discarded weight = the tail sum of the weights
        ok = [k for k in range(min(m_min, M), min(M, D) + 1) if np.sum(w[k:]) <= target]
        k_ref = ok[0] if ok else min(M, D)
        assert w[k_ref - 1] > 1e-10 and w[k_ref - 1] - w[k_ref] > 1e-12   # no tie at the cut
        _, keep, tr, _ = truncate(x, sb.layout, sb.L, "L", M, m_min, target)
        assert sum(keep.values()) == k_ref, (m_min, M, target)
        assert abs(tr - np.sum(w[k_ref:])) < 1e-12
        if k_ref < min(M, D):
            assert tr <= target + 1e-15
        if k_ref > min(m_min, M):
            assert np.sum(w[k_ref - 1:]) > target    # one state fewer misses the target


def test_dbss_special_cases():
    from oracle.dmrg import truncate
    sb, x = _psi_at()
    D = sum(sb.L.dims.values())
    U0, keep0, tr0, _ = truncate(x, sb.layout, sb.L, "L", 7)
    # floor = ceiling: the fixed-M selection
    U1, keep1, tr1, _ = truncate(x, sb.layout, sb.L, "L", 7, 7, 0.5)
    assert keep1 == keep0 and tr1 == tr0
    assert all(np.array_equal(U0[Q], U1[Q]) for Q in U0)
    # a target every count meets: the floor
    _, keep2, _, _ = truncate(x, sb.layout, sb.L, "L", 7, 4, 0.999)
    assert sum(keep2.values()) == 4
    # a target no count meets below the ceiling: the ceiling
    _, keep3, _, _ = truncate(x, sb.layout, sb.L, "L", 7, 2, 1e-300)
    assert keep3 == keep0
    # no more states than the floor: everything is kept
    _, keep4, tr4, _ = truncate(x, sb.layout, sb.L, "L", D + 5, D, 1e-3)
    assert keep4 == dict(sb.L.dims) and tr4 < 1e-13


def test_dbss_sweeps_bound_the_truncation_and_reach_exact():
    """sd shell 2p+2n (m-scheme dimension 640).  From a random start, each DBSS truncation
    below the ceiling discards at most the target and the energies stay variational.  From
    the exact state (one sweep with complete bases), a tight target keeps the full CI
    energy with far fewer states (it drops only the zero weights), and a looser one gives
    an error that shrinks with the target."""
    p = make_problem("sd", 2, 2, 0, seed=1)
    e0 = ed_lowest(p)[0]
    loose = OracleDMRG(p, initial_mps(p, 8, 5), m_min=16, trunc_target=1e-3)
    for _ in range(2):
        res = loose.sweep(64)
        for r in res:
            assert r.energy >= e0 - 1e-10
            if sum(r.kept.values()) < 64:
                assert r.trunc_err <= 1e-3 + 1e-15
    kept = [sum(r.kept.values()) for r in res]
    assert 16 < max(kept) < 64                 # the target, not the ceiling, set the count
    d = OracleDMRG(p, initial_mps(p, 8, 5))
    full = d.sweep(400)
    assert abs(full[-1].energy - e0) < 1e-10
    n_full = sum(sum(r.kept.values()) for r in full)
    errs = []
    for target in (1e-10, 1e-5, 1e-3):        # tightest first: each starts near exact
        d.m_min, d.trunc_target = 4, target
        res = d.sweep(400)
        for r in res:
            assert r.energy >= e0 - 1e-10
            assert r.trunc_err <= target + 1e-15
        errs.append(res[-1].energy - e0)
        n_dbss = sum(sum(r.kept.values()) for r in res)
        assert n_dbss < 0.5 * n_full
    assert abs(errs[0]) < 1e-9
    assert 1e-8 < errs[1] < 1e-3 and errs[2] > errs[1]


# ---------------------------------------------------------------------------------------
# two-state targeting: the two lowest states with the averaged density matrix
# ---------------------------------------------------------------------------------------
def test_two_root_davidson_reduces_to_one_root():
    from oracle.dmrg import davidson, davidson_roots
    sb, _ = _psi_at(3)
    x0 = np.ones(sb.layout.size)
    th, x, npr, rn = davidson(sb.apply, sb.diagonal(), x0, max_sub=6)
    ths, xs, npr2, rns = davidson_roots(sb.apply, sb.diagonal(), [x0], max_sub=6, n_roots=1)
    assert ths == [th] and npr2 == npr and rns == [rn]
    assert np.array_equal(xs[0], x)


@pytest.mark.parametrize("max_sub,second_guess", [(24, False), (5, False), (24, True)])
def test_two_root_davidson_finds_the_two_lowest(max_sub, second_guess):
    """Against the dense H_eff: both Ritz values are its two lowest eigenvalues, the
    vectors are orthonormal eigenvectors (with and without restarts, with a second
    guess entering the subspace)."""
    from oracle.dmrg import davidson_roots
    sb, _ = _psi_at(3)
    n = sb.layout.size
    He = np.stack([sb.apply(np.eye(n)[:, c]) for c in range(n)], axis=1)
    ev, evec = np.linalg.eigh(He)
    assert ev[1] - ev[0] > 1e-3 and ev[2] - ev[1] > 1e-3
    rng = np.random.default_rng(4)
    guesses = [np.ones(n)]
    if second_guess:
        guesses.append(evec[:, 1] + 1e-3 * rng.standard_normal(n))
    ths, xs, npr, rns = davidson_roots(sb.apply, sb.diagonal(), guesses, tol=1e-10,
                                       max_sub=max_sub, n_roots=2)
    assert abs(ths[0] - ev[0]) < 1e-10 and abs(ths[1] - ev[1]) < 1e-10
    assert max(rns) <= 1e-10
    X = np.stack(xs, axis=1)
    assert np.allclose(X.T @ X, np.eye(2), atol=1e-12)
    assert np.linalg.norm(He @ X - X * np.array(ths)) < 1e-9


def test_averaged_density_matrix_truncation():
    """The two-state truncation keeps the largest eigenvalues of (rho_0 + rho_1) / 2,
    obtained independently from the singular values of [P_0 P_1] / sqrt(2) per sector."""
    from oracle.dmrg import davidson_roots, truncate
    sb, _ = _psi_at(4)
    ths, xs, _, _ = davidson_roots(sb.apply, sb.diagonal(), [np.ones(sb.layout.size)],
                                   tol=1e-10, n_roots=2)
    w = []
    for (QL, QR, dL, dR, off) in sb.layout.blocks:
        B = np.hstack([x[off:off + dL * dR].reshape(dL, dR) for x in xs]) / np.sqrt(2.0)
        w.extend(np.linalg.svd(B, compute_uv=False) ** 2)
    w = np.sort(np.concatenate([w, np.zeros(sum(sb.L.dims.values()) - len(w))]))[::-1]
    assert abs(w.sum() - 1.0) < 1e-12
    cuts = [M for M in range(2, len(w)) if w[M - 1] > 1e-10 and w[M - 1] - w[M] > 1e-6 * w[M - 1]]
    assert len(cuts) >= 3
    for M in cuts:
        _, keep, tr, _ = truncate(np.stack(xs), sb.layout, sb.L, "L", M)
        assert sum(keep.values()) == M
        assert abs(tr - w[M:].sum()) < 1e-12


@pytest.mark.parametrize("space,seed,M0", [("p", 12, 6), ("sd", 1, 8)])
def test_two_state_sweeps_reach_the_two_lowest_exact_states(space, seed, M0):
    """Complete bases: the two targeted energies equal the two lowest eigenvalues of the
    sector from exact diagonalization; truncated bases: both stay above them (the
    projected Hamiltonian's eigenvalues interlace the exact ones)."""
    p = make_problem(space, 2, 2, 0, seed=seed)
    e0, e1 = ed_lowest(p, k=2)
    d = OracleDMRG(p, initial_mps(p, M0, 5), n_roots=2)
    res = d.sweep(10 ** 6)
    res = d.sweep(10 ** 6)
    assert abs(res[-1].energy - e0) < 1e-9 and abs(res[-1].energy1 - e1) < 1e-9
    t = OracleDMRG(p, initial_mps(p, M0, 5), n_roots=2)
    for _ in range(2):
        for r in t.sweep(4 if space == "p" else 16):
            assert r.energy >= e0 - 1e-10 and r.energy1 >= e1 - 1e-10


# ---------------------------------------------------------------------------------------
# the truncation's cut rules on wave functions with chosen weights
# ---------------------------------------------------------------------------------------
def _weights_psi(sb, weights):
    """A wave function whose left density matrix has exactly the given eigenvalues: one
    entry per chosen block (the blocks with the largest dims first), value sqrt(w)."""
    x = np.zeros(sb.layout.size)
    blocks = sorted(sb.layout.blocks, key=lambda b: -b[2] * b[3])
    assert len(blocks) >= len(weights)
    for (QL, QR, dL, dR, off), w in zip(blocks, weights):
        x[off] = np.sqrt(w)
    return x


def test_cut_keeps_whole_multiplets_and_drops_zero_weights():
    from oracle.dmrg import truncate
    sb, _ = _psi_at(4)
    # an exact pair at the cut is kept whole (M = 2 keeps 3)
    x = _weights_psi(sb, [0.5, 0.25, 0.25])
    _, keep, tr, _ = truncate(x, sb.layout, sb.L, "L", 2)
    assert sum(keep.values()) == 3 and abs(tr) < 1e-15
    # within the 1e-10 relative tolerance counts as degenerate, beyond it does not
    x = _weights_psi(sb, [0.5, 0.25 * (1 + 2e-11), 0.25 * (1 - 2e-11)])
    assert sum(truncate(x, sb.layout, sb.L, "L", 2)[1].values()) == 3
    x = _weights_psi(sb, [0.5, 0.25 * (1 + 1e-8), 0.25 * (1 - 1e-8)])
    _, keep, tr, _ = truncate(x, sb.layout, sb.L, "L", 2)
    assert sum(keep.values()) == 2 and abs(tr - 0.25 * (1 - 1e-8)) < 1e-15
    # weights at or below 1e-14 are never kept, even below M; all kept when D <= M
    x = _weights_psi(sb, [1.0 - 2e-15, 1e-15, 1e-15])
    D = sum(sb.L.dims.values())
    _, keep, _, _ = truncate(x, sb.layout, sb.L, "L", D - 1)
    assert sum(keep.values()) == 1
    _, keep, _, _ = truncate(x, sb.layout, sb.L, "L", D)
    assert keep == dict(sb.L.dims)


@pytest.mark.parametrize("Np,Nn,two_M", [(0, 3, 1), (0, 2, 0), (1, 0, 1), (6, 1, 1), (5, 5, 0),
                                         (6, 6, 0)])
def test_degenerate_particle_numbers(Np, Nn, two_M):
    """One species absent, a single particle, a full proton shell, the completely filled
    p shell (a one-state sector): complete bases reproduce exact diagonalization."""
    p = make_problem("p", Np, Nn, two_M, seed=4)
    e0 = ed_lowest(p)[0]
    d = OracleDMRG(p, initial_mps(p, 6, 5))
    d.sweep(10 ** 6)
    res = d.sweep(10 ** 6)
    assert abs(res[-1].energy - e0) < 1e-10


def test_filled_shell_closed_form():
    """Every orbital occupied: E = sum_i eps_i + sum_{i<j} vbar[ij, ij]."""
    p = make_problem("p", 6, 6, 0, seed=4)
    v = {tuple(k): x for k, x in zip(p.v_idx.tolist(), p.v_val.tolist())}
    N = p.n_sites
    e = float(np.sum(p.eps)) + sum(v.get((i, j, i, j), 0.0) for i in range(N)
                                   for j in range(i + 1, N))
    d = OracleDMRG(p, initial_mps(p, 6, 5))
    res = d.sweep(10 ** 6)
    assert abs(res[-1].energy - e) < 1e-10 and abs(ed_lowest(p)[0] - e) < 1e-10


@pytest.fixture(scope="module")
def sb_mid():
    p = make_problem("sd", 2, 2, 0, seed=1)
    d = OracleDMRG(p, initial_mps(p, 64, 5))
    for q in range(1, 11):
        d.run_step(q, "L", 64)
    return d.superblock(11)


@pytest.mark.parametrize("max_sub", [4, 7, 24])
def test_davidson_with_restarts_finds_the_lowest_eigenpair(sb_mid, max_sub):
    """A superblock of 169 states (sd 2p+2n, M = 64, mid-chain): Davidson with thick
    restarts every max_sub vectors reaches the lowest eigenvalue of the dense H_eff."""
    from oracle.dmrg import davidson
    sb = sb_mid
    n = sb.layout.size
    assert n > 100
    He = np.stack([sb.apply(np.eye(n)[:, c]) for c in range(n)], axis=1)
    w = np.linalg.eigvalsh(He)
    th, x, nprod, rn = davidson(sb.apply, sb.diagonal(), np.ones(n), tol=1e-9, max_iter=400,
                                max_sub=max_sub)
    assert rn <= 1e-9 and abs(th - w[0]) < 1e-10
    assert np.linalg.norm(He @ x - th * x) < 1e-8
