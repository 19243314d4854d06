"""The learned Davidson preconditioner on the GPU: training-kernel gradients against the
FP64 CPU network, and the trained network inside Davidson (same converged energies as
diagonal Davidson; iteration counts reported)."""
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
    return P


def test_gradients_match_cpu_network(P):
    from oracle import mlp
    rng = np.random.default_rng(7)
    theta = rng.standard_normal(mlp.n_params()) * 0.1
    X = rng.standard_normal((96, 4))
    T = rng.standard_normal(96)
    loss_ref, g_ref = mlp.loss_and_grad(theta, X, T)
    d = P.DMRG(make_problem("p", 2, 2, 0, seed=12))
    loss, g = d.mlp_loss_grad(theta, X, T, precision=P.FP64)
    assert abs(loss - loss_ref) <= 1e-12 * abs(loss_ref)
    assert np.linalg.norm(g - g_ref) <= 1e-10 * np.linalg.norm(g_ref)
    loss32, g32 = d.mlp_loss_grad(theta, X, T, precision=P.MIXED_FP32)
    assert abs(loss32 - loss_ref) <= 1e-5 * abs(loss_ref)
    assert np.linalg.norm(g32 - g_ref) <= 1e-4 * np.linalg.norm(g_ref)


def test_trained_preconditioner_same_energies(P, capsys):
    prob = make_problem("sd", 2, 2, 0, seed=1)
    d = P.DMRG(prob)
    d.build_blocks(initial_mps(prob, 64, 5))
    d.mlp_harvest(True, 1024)
    d.sweep(64)
    d.sweep(64)
    d.mlp_harvest(False)
    d.mlp_reset(3)
    loss0, ns = d.mlp_train(epochs=1, batch=512, lr=1e-3, seed=3)
    loss1, _ = d.mlp_train(epochs=40, batch=512, lr=1e-3, seed=4)
    assert ns > 1000 and loss1 < loss0
    n_diag = n_mlp = 0
    for p in range(2, 12):
        size = d.psi_layout(p)["size"]
        x0 = torch.ones(size, dtype=torch.float64, device="cuda")
        d.set_options(precond=P.PRECOND_DIAG)
        e1, s1 = d.davidson(p, guess=x0)
        d.set_options(precond=P.PRECOND_MLP)
        e2, s2 = d.davidson(p, guess=x0)
        assert abs(e1 - e2) < 1e-8, (p, e1, e2)
        n_diag += s1["n_products"]
        n_mlp += s2["n_products"]
        d.set_options(precond=P.PRECOND_DIAG)
        d.step(p, 0, 64)
    with capsys.disabled():
        print(f"\n[learned preconditioner] sd 2p+2n M=64, positions 2..11 from the uniform guess: "
              f"diagonal {n_diag} products, learned {n_mlp} products (loss {loss0:.3f} -> {loss1:.3f})")
    # what the trained network gains: fewer H_eff products for the same converged energies
    # (the counts vary by a few products between runs: the order of the FP32 gradient sums)
    assert n_mlp < n_diag, (n_mlp, n_diag)


def test_training_after_the_sample_ring_wraps(P):
    # enough harvested iterates to fill the sample ring and wrap around: training must only
    # draw from written samples (loss and parameters finite)
    prob = make_problem("sd", 4, 4, 0, seed=1)
    d = P.DMRG(prob)
    d.build_blocks(initial_mps(prob, 256, 5))
    d.mlp_harvest(True, 2048)
    d.sweep(256)
    d.sweep(256)
    d.mlp_harvest(False)
    d.mlp_reset(3)
    loss, ns = d.mlp_train(epochs=1, batch=1024, lr=1e-3, seed=3)
    assert ns > 200000
    assert np.isfinite(loss)
    assert np.all(np.isfinite(d.mlp_params()))
