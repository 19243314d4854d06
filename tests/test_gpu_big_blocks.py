"""GPU: the wide-block paths of the product and of the renormalization on the pf-shell
workloads, through the C-ABI.

* H_eff psi at the first position of pf 4p+4n (starting state M0 = 1024) and of the
  headline pf 8p+8n (M0 = 4096) against the oracle's product on identical, gauge-free
  inputs (stored by tests/golden/make_heff_pos1.py, which calls only the oracle): the
  layout bit-exact, the sampled elements, the norm and four projections on seeded vectors
  within 1e-12 relative (FP64) and 2e-6 (mixed: split-TF32 tensor cores, FP32 storage).
  These superblocks have right blocks hundreds of states wide, so every term takes the
  grouped GEMM passes.
* A mid-chain superblock of pf 8p+8n after the sweeps 512, 1024 (blocks up to ~100 states
  wide): the grouped GEMM passes against the fused tile kernels (dmrg_set_tuning
  heff_big_edge 0) on the same superblock and inputs, FP64 within 1e-12, the mixed grouped
  passes within 2e-6 of the FP64 result (their K chunks are summed with compensation), the
  mixed fused kernels within 1e-5 (forced onto wide terms they accumulate thousands of
  products in the tensor cores' FP32 accumulators; measured 5e-6 on this superblock).
* Mixed vs FP64 Davidson on identical superblocks along a run of steps: energies within
  1e-8 MeV.
"""
import json
import os

import numpy as np
import pytest

from gen import make_problem, initial_mps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def P():
    from paper_1507_00161_gb300.build import build
    build()
    import paper_1507_00161_gb300 as P
    assert torch.cuda.is_available()
    return P


@pytest.mark.parametrize("case", ["pf4p4n", "pf8p8n"])
def test_heff_first_position_against_oracle(P, case):
    path = os.path.join(GOLDEN, "heff_pos1_%s.json" % case)
    with open(path) as f:
        g = json.load(f)
    prob = make_problem(g["space"], g["Np"], g["Nn"], g["two_Mz"], seed=g["seed"])
    d = P.DMRG(prob)
    d.build_blocks(initial_mps(prob, g["M0"], g["mps_seed"]))
    lay = d.psi_layout(1)
    assert lay["size"] == g["size"]
    got = [[list(map(int, q)), int(a), int(b), int(o)]
           for q, a, b, o in zip(lay["qn_left"], lay["dl"], lay["dr"], lay["off"])]
    assert got == g["blocks"]
    assert max(lay["dr"]) > 32          # wide blocks: the grouped GEMM passes
    x = np.random.default_rng(7).standard_normal(g["size"])
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    yd = torch.empty_like(xd)
    idx = np.array(g["sample_index"])
    ref = np.array(g["sample_value"])
    vs = [np.random.default_rng(100 + j).standard_normal(g["size"]) for j in range(4)]
    for precision, tol in ((P.FP64, 1e-12), (P.MIXED_FP32, 2e-6)):
        d.set_options(precision=precision)
        d.heff_apply(1, xd, yd)
        y = yd.cpu().numpy()
        scale = g["norm"]
        assert abs(np.linalg.norm(y) - scale) <= tol * scale
        assert np.max(np.abs(y[idx] - ref)) <= tol * scale
        for v, pr in zip(vs, g["projections"]):
            assert abs(v @ y - pr) <= tol * scale * np.linalg.norm(v)
    d.close()


def _mid_chain(P, precision=None):
    prob = make_problem("pf", 8, 8, 0, seed=3)
    d = P.DMRG(prob, precision=P.FP64 if precision is None else precision)
    d.build_blocks(initial_mps(prob, 512, 3003))
    d.sweep(512)
    d.sweep(1024)
    for p in range(1, 19):
        d.step(p, 0, 1024)
    return prob, d


def test_grouped_passes_equal_fused_kernels(P):
    prob, d = _mid_chain(P)
    p = 19
    lay = d.psi_layout(p)
    assert max(max(lay["dl"]), max(lay["dr"])) > 32
    x = torch.tensor(np.random.default_rng(3).standard_normal(lay["size"]), dtype=torch.float64,
                     device="cuda")
    out = {}
    for edge in (32, 0):
        d.set_tuning(heff_big_edge=edge)
        for prec in (P.FP64, P.MIXED_FP32):
            d.set_options(precision=prec)
            y = torch.empty_like(x)
            d.heff_apply(p, x, y)
            out[(edge, prec)] = y.cpu().numpy()
    ref = out[(0, P.FP64)]
    nrm = np.linalg.norm(ref)
    assert np.linalg.norm(out[(32, P.FP64)] - ref) <= 1e-12 * nrm
    assert np.linalg.norm(out[(32, P.MIXED_FP32)] - ref) <= 2e-6 * nrm
    assert np.linalg.norm(out[(0, P.MIXED_FP32)] - ref) <= 1e-5 * nrm
    d.close()


def test_mixed_energy_on_identical_superblocks(P):
    """Mixed and FP64 Davidson on the same superblocks along FP64 steps (pf 4p+4n, M = 256):
    the mixed energy (the FP64 Rayleigh quotient of the vector found with split-TF32
    products) within 1e-8 MeV of the FP64 energy."""
    prob = make_problem("pf", 4, 4, 0, seed=2)
    d = P.DMRG(prob)
    d.build_blocks(initial_mps(prob, 256, 2002))
    for p in range(1, 16):
        if p % 5 == 0:
            d.set_options(precision=P.MIXED_FP32)
            e_m, st_m = d.davidson(p)
            d.set_options(precision=P.FP64)
            e_d, st_d = d.davidson(p)
            assert st_m["converged"] and st_d["converged"]
            assert abs(e_m - e_d) <= 1e-8, (p, e_m, e_d)
        d.step(p, 0, 256)
    d.close()


def test_tuning_rejects_bad_values(P):
    prob = make_problem("p", 2, 2, 0, seed=12)
    d = P.DMRG(prob)
    with pytest.raises(P.DmrgError):
        d.set_tuning(heff_big_edge=-1)
    with pytest.raises(P.DmrgError):
        d.set_tuning(svd_cluster=3)
    with pytest.raises(P.DmrgError):
        d.set_tuning(heff_graph=2)
    assert d.tuning() == {"heff_big_edge": 128, "svd_cluster": 0, "heff_graph": 1}
    d.set_tuning(heff_big_edge=48, svd_cluster=8, heff_graph=0)
    assert d.tuning() == {"heff_big_edge": 48, "svd_cluster": 8, "heff_graph": 0}
    d.close()


def test_autotune_picks_a_candidate_and_products_agree(P):
    """The autotuner times the work splits on a mid-chain superblock, keeps one of the
    candidates, and the product with the chosen split equals the FP64 product within 1e-5
    (the bar of the fused kernels, which keep the blocks up to the chosen edge)."""
    prob, d = _mid_chain(P, precision=P.MIXED_FP32)
    p = 19
    chosen, times = d.autotune(p, reps=2)
    assert chosen in (0, 32, 64, 128, 256)
    assert set(times) == {0, 32, 64, 128, 256} and all(t > 0 for t in times.values())
    assert d.tuning()["heff_big_edge"] == chosen
    n = d.psi_layout(p)["size"]
    x = torch.tensor(np.random.default_rng(5).standard_normal(n), dtype=torch.float64,
                     device="cuda")
    y = torch.empty_like(x)
    d.heff_apply(p, x, y)
    d.set_options(precision=P.FP64)
    ref = torch.empty_like(x)
    d.heff_apply(p, x, ref)
    err = float(torch.linalg.norm(y - ref) / torch.linalg.norm(ref))
    assert err <= 1e-5, (chosen, err)
    print("[autotune] chosen edge %d, times (ms) %s" % (chosen, times))
    d.close()


def test_graph_replay_is_bit_exact(P):
    """The product replayed from its CUDA graph (dmrg_tuning.heff_graph = 1: eager first
    product, captured at the second) equals the eagerly launched product bit for bit, in
    both precisions, on a superblock with fused tiles and grouped passes (pf 4p+4n, first
    position of the M0 = 1024 starting state, grouped passes above 32 states); a sweep with
    graphs gives the same energies, bit for bit, as one without."""
    prob = make_problem("pf", 4, 4, 0, seed=2)
    init = initial_mps(prob, 1024, 2002)
    out = {}
    for graph in (0, 1):
        d = P.DMRG(prob)
        d.build_blocks(init)
        d.set_tuning(heff_big_edge=32, heff_graph=graph)
        n = d.psi_layout(1)["size"]
        x = torch.tensor(np.random.default_rng(3).standard_normal(n), dtype=torch.float64,
                         device="cuda")
        for prec in (P.FP64, P.MIXED_FP32):
            d.set_options(precision=prec)
            r0 = d.counters()["t_detail"][22]
            ys = []
            for _ in range(3):
                y = torch.full_like(x, float("nan"))
                d.heff_apply(1, x, y)
                ys.append(y.cpu().numpy())
            replays = d.counters()["t_detail"][22] - r0
            assert replays == (2 if graph else 0), (graph, prec, replays)
            out[(graph, prec)] = ys
        d.close()
    for prec in (P.FP64, P.MIXED_FP32):
        ref = out[(0, prec)][0]
        assert np.all(np.isfinite(ref))
        for y in out[(0, prec)] + out[(1, prec)]:
            assert np.array_equal(y, ref), prec
    prob = make_problem("sd", 3, 3, 0, seed=1)
    init = initial_mps(prob, 64, 9)
    energies = {}
    for graph in (0, 1):
        d = P.DMRG(prob, precision=P.MIXED_FP32)
        d.set_tuning(heff_graph=graph)
        d.build_blocks(init)
        steps, e = d.sweep(64)
        energies[graph] = [s["energy"] for s in steps]
        if graph:
            assert d.counters()["t_detail"][22] > 0
        d.close()
    assert energies[0] == energies[1]
