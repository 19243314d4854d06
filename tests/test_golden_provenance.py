"""The stored pf+g9/2 oracle sweep (tests/golden/pfg_2p2n_M4.json) is what its committed
script computes from oracle/ and gen/ alone: recomputed here, every step's energy and
truncation error agree to 1e-10 and the kept states per sector exactly."""
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
