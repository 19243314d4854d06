"""Host logic of bench.py's side measurements, on CPU, against a stand-in for the device
library (every call the sections make, returning plausible shapes): the sections run to the
end without an error entry and report the keys the design document quotes.  The numbers
are the stand-in's; the real ones come from the GPU."""
import os
import sys
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


class _Event:
    def __init__(self, enable_timing=False):
        pass

    def record(self, *a):
        pass

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return 1.0


class _FakeDMRG:
    """Stand-in context: the calls and return shapes of paper_1507_00161_gb300.DMRG."""

    def __init__(self, prob, precision=0, dav_tol=1e-8, **kw):
        self.N = prob.n_sites
        self.theta = None

    def build_blocks(self, init):
        pass

    def _steps(self, n):
        return [{"p": 1, "dir": 0, "n_products": 3, "kept": 8, "energy": -1.0, "residual": 1e-9,
                 "trunc_err": 1e-6, "seconds": 0.01, "heff_seconds": 0.001, "heff_flops": 1e6,
                 "heff_bytes": 1e5, "energy1": -0.5} for _ in range(n)]

    def sweep(self, M):
        return self._steps(2 * (self.N - 3)), -1.0

    def step(self, p, direction, M):
        return self._steps(1)[0]

    def set_dbss(self, *a):
        pass

    def set_roots(self, *a):
        pass

    def set_options(self, **kw):
        pass

    def psi_layout(self, p):
        return {"size": 16}

    def davidson(self, p, guess=None, out=None, allow_noconv=False):
        return -1.0, {"n_products": 4, "converged": 1}

    def mlp_harvest(self, *a):
        pass

    def mlp_reset(self, *a):
        pass

    def mlp_train(self, **kw):
        return 0.5, 1000

    def mlp_params(self):
        return np.zeros(10)

    def mlp_set_params(self, theta):
        self.theta = theta

    def mutual_information(self, M):
        rng = np.random.default_rng(0)
        A = rng.random((self.N, self.N))
        I = A + A.T
        np.fill_diagonal(I, 0.0)
        return I, np.full(self.N, 0.5), self._steps(self.N - 3)

    def close(self):
        pass


@pytest.fixture
def fake(monkeypatch):
    torch = pytest.importorskip("torch")
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda *a: (1 << 30, 1 << 31))
    monkeypatch.setattr(torch, "ones", lambda n, **kw: np.ones(n))
    import paper_1507_00161_gb300 as P0
    return types.SimpleNamespace(DMRG=_FakeDMRG, FP64=0, MIXED_FP32=1, PRECOND_DIAG=0,
                                 PRECOND_MLP=1, fiedler_order=P0.fiedler_order)


def test_next_rows_section(fake):
    import bench
    from gen import initial_mps, make_problem
    prob = make_problem("p", 2, 2, 0, seed=1)
    out = bench.run_next_rows(fake, prob, initial_mps(prob, 8, 1), 8, None)
    assert set(out) == {"dbss", "two_state", "mutual_information"}
    for k, v in out.items():
        assert "error" not in v, (k, v)
    mi = out["mutual_information"]
    assert sorted(mi["fiedler_order"]) == list(range(40))
    assert len(mi["top_pairs"]) == 5


def test_pfg_section(fake, monkeypatch):
    import bench
    import gen
    # the starting state of the 60-site workload is not needed by the stand-in
    monkeypatch.setattr(gen, "initial_mps", lambda prob, M, seed: None)
    out = bench.run_pfg(fake, 2048)
    for tmz in (0, 4):
        r = out["two_Mz_%d" % tmz]
        assert [s["M"] for s in r["sweeps"]] == [512, 1024, 1024, 2048]
    assert "mlp" in out["two_Mz_0"]
    h = out["two_Mz_4"]["precond_held_out"]
    for k in ("products_diagonal", "products_learned", "sweep_s_diagonal", "sweep_s_learned",
              "max_step_dE"):
        assert k in h
