"""The allocation-free H_eff entry point, for callers that cannot allocate device memory
during a product (a process whose GPU memory another allocator owns, code that must not
trigger the synchronisation of cudaMalloc / cudaFree).  Through the C-ABI it must give
the same product as dmrg_heff_apply (same 1e-12 relative tolerance as the other H_eff
tests) on two calls in a row, leave device memory untouched, and fully overwrite its
output.  Collected last on purpose."""
import numpy as np
import pytest

from gen import make_problem, initial_mps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("space,Np,Nn,seed,M0", [("p", 2, 2, 12, 5), ("sd", 2, 2, 1, 16)])
def test_noalloc_matches_heff_apply(space, Np, Nn, seed, M0):
    from paper_1507_00161_gb300.build import build
    build()
    import paper_1507_00161_gb300 as P
    prob = make_problem(space, Np, Nn, 0, seed=seed)
    d = P.DMRG(prob)
    d.build_blocks(initial_mps(prob, M0, seed + 100))
    rng = np.random.default_rng(seed)
    for p in (1, 2):
        if p == 2:
            d.step(1, 0, M0)           # makes the left block of bond 1
        size = d.psi_layout(p)["size"]   # sets up the superblock (this call allocates)
        x = torch.tensor(rng.standard_normal(size), dtype=torch.float64, device="cuda")
        ref = torch.empty_like(x)
        d.heff_apply(p, x, ref)
        ref_h = ref.cpu().numpy()
        ys = [torch.empty_like(x) for _ in range(3)]
        torch.cuda.synchronize()
        free0 = mallocs0 = None
        for i, y in enumerate(ys):        # calls in a row, output pre-filled with NaN
            if i == 1:
                # the first call on a device is the documented set-up (address lookup;
                # the driver may load the code holding the array then): memory is
                # checked over the calls after it
                torch.cuda.synchronize()
                free0 = torch.cuda.mem_get_info()[0]
                mallocs0 = d.counters()["pool_mallocs"]
            y.fill_(float("nan"))
            d.heff_apply_noalloc(p, x, y)
            yh = y.cpu().numpy()
            err = np.linalg.norm(yh - ref_h) / np.linalg.norm(ref_h)
            assert err <= 1e-12, err
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert d.counters()["pool_mallocs"] == mallocs0   # no allocation by the library


def test_noalloc_rejects_products_above_its_limit():
    """A product whose intermediate exceeds the 2,097,152-double array is rejected with
    DMRG_EINVAL and leaves the output untouched (pf 8p+8n mid-chain after sweeps at 512
    and 1024 states)."""
    from paper_1507_00161_gb300.build import build
    build()
    import paper_1507_00161_gb300 as P
    prob = make_problem("pf", 8, 8, 0, seed=3)
    d = P.DMRG(prob, precision=P.MIXED_FP32)
    d.build_blocks(initial_mps(prob, 512, 3003))
    d.sweep(512)
    d.sweep(1024)
    for p in range(1, 19):
        d.step(p, 0, 1024)
    d.set_options(precision=P.FP64)
    size = d.psi_layout(19)["size"]
    x = torch.ones(size, dtype=torch.float64, device="cuda")
    y = torch.full_like(x, float("nan"))
    with pytest.raises(P.DmrgError) as e:
        d.heff_apply_noalloc(19, x, y)
    assert e.value.code == P.DMRG_EINVAL
    assert "2097152" in str(e.value)
    assert torch.isnan(y).all()
    d.close()


def test_noalloc_requires_set_up_superblock():
    from paper_1507_00161_gb300.build import build
    build()
    import paper_1507_00161_gb300 as P
    prob = make_problem("p", 2, 2, 0, seed=12)
    d = P.DMRG(prob)
    d.build_blocks(initial_mps(prob, 5, 112))
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(P.DmrgError) as e:
        d.heff_apply_noalloc(1, x, y)
    assert e.value.code == P.DMRG_EINVAL
