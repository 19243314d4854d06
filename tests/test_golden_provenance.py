"""Stored oracle values are what their committed scripts compute from oracle/ and gen/
alone, recomputed here:
* the pf+g9/2 sweep (tests/golden/pfg_2p2n_M4.json): every step's energy and truncation
  error to 1e-10, the kept states per sector exactly;
* the oracle's H_eff psi at the first position of pf 4p+4n (heff_pos1_pf4p4n.json): the
  layout exactly, the norm and the sampled elements to 1e-12 |y|, the projections on
  seeded vectors (norm ~ sqrt(size)) to 1e-9 |y|."""
import importlib.util
import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def test_pfg_golden_is_reproduced_by_its_script():
    spec = importlib.util.spec_from_file_location(
        "make_pfg_sweep", os.path.join(HERE, "golden", "make_pfg_sweep.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    with open(mod.OUT) as f:
        stored = json.load(f)
    new = mod.compute()
    assert len(new["steps"]) == len(stored["steps"])
    for a, b in zip(new["steps"], stored["steps"]):
        assert (a["p"], a["dir"]) == (b["p"], b["dir"])
        assert abs(a["energy"] - b["energy"]) <= 1e-10
        assert abs(a["trunc_err"] - b["trunc_err"]) <= 1e-10
        assert a["kept"] == b["kept"]


def test_pf4p4n_product_golden_is_reproduced_by_its_script():
    spec = importlib.util.spec_from_file_location(
        "make_heff_pos1", os.path.join(HERE, "golden", "make_heff_pos1.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    with open(os.path.join(HERE, "golden", "heff_pos1_pf4p4n.json")) as f:
        stored = json.load(f)
    new = mod.compute("pf4p4n")
    assert new["blocks"] == stored["blocks"] and new["size"] == stored["size"]
    assert new["sample_index"] == stored["sample_index"]
    scale = stored["norm"]
    assert abs(new["norm"] - scale) <= 1e-12 * scale
    assert max(abs(a - b) for a, b in zip(new["sample_value"], stored["sample_value"])) <= 1e-12 * scale
    assert max(abs(a - b) for a, b in zip(new["projections"], stored["projections"])) <= 1e-9 * scale
