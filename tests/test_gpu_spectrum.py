"""The library's H_eff against the Hamiltonian itself, independently of the oracle's DMRG:
with full right-block bases (a starting state that keeps every state of every sector,
rotated by seeded orthogonal matrices) the superblock at the first position spans the whole
m-scheme sector, so the matrix of dmrg_heff_apply (applied to every unit vector) must have
the spectrum of the dense Hamiltonian built from the determinant basis by Slater-Condon
rules (oracle.hamiltonian.ed_sector, which shares nothing with the operator partition).
Every eigenvalue is compared, so every term of the partition (normal and complementary
operators of the nine-to-twenty-site right blocks, the dots, the Jordan-Wigner signs of
shuffled chain orders) has to be right, not only those that move the ground state."""
import dataclasses

import numpy as np
import pytest

from gen import make_problem, initial_mps
from gen.shell import mscheme_dimension

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_1507_00161_gb300.build import build
    build()
    import paper_1507_00161_gb300 as P
    assert torch.cuda.is_available()
    return P


@pytest.mark.parametrize("space,Np,Nn,tM,seed,shuffle", [
    ("p", 2, 2, 0, 3, False), ("p", 2, 3, 1, 7, True), ("sd", 2, 1, 3, 4, True),
    ("sd", 2, 2, 0, 1, False)])
def test_full_basis_heff_has_the_exact_spectrum(P, space, Np, Nn, tM, seed, shuffle):
    from oracle.hamiltonian import ed_sector
    prob = make_problem(space, Np, Nn, tM, seed=seed)
    if shuffle:
        order = np.random.default_rng(seed).permutation(prob.n_sites).astype(np.int32)
        prob = dataclasses.replace(prob, order=order)
    dim = mscheme_dimension(space, Np, Nn, tM)
    _, Hd = ed_sector(prob, Np, Nn, tM)
    exact = np.linalg.eigvalsh(Hd)
    init = initial_mps(prob, 10 ** 6, seed + 11)
    for prec, tol in ((P.FP64, 1e-10), (P.MIXED_FP32, 2e-5)):
        d = P.DMRG(prob, precision=prec)
        d.build_blocks(init)
        n = d.psi_layout(1)["size"]
        assert n == dim
        H = np.empty((n, n))
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        for k in range(n):
            x.zero_()
            x[k] = 1.0
            d.heff_apply(1, x, y)
            H[:, k] = y.cpu().numpy()
        d.close()
        scale = np.max(np.abs(exact))
        assert np.max(np.abs(H - H.T)) <= tol * scale
        got = np.linalg.eigvalsh(0.5 * (H + H.T))
        assert np.max(np.abs(got - exact)) <= tol * scale, (prec, np.max(np.abs(got - exact)))
