"""The stored full-length oracle results (tests/golden/oracle_*.json) are
what the committed script computes from the oracle: their layout is
checked, and the cheapest records (the smallest lattice of each ensemble
file) are recomputed here from the oracle alone."""
import importlib.util
import json
import os

import numpy as np

import oracle
from paper_1804_07981_b300.inputs import ensemble_params

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _script():
    spec = importlib.util.spec_from_file_location(
        "make_oracle_refs", os.path.join(GOLDEN, "make_oracle_refs.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_golden_files_cover_the_workloads():
    runs = _load("oracle_4096_runs.json")
    assert sorted((r["rho"], r["seed"]) for r in runs["runs"]) == \
        [(rho, s) for rho in (0.20, 0.35, 0.50) for s in (1, 2, 3)]
    win = _load("oracle_32768_windows.json")
    t, c, M = win["steps"], win["centre"], win["M"]
    assert (t, c, win["window"]) == (1024, 33, 2 * 1024 + 33) and len(win["windows"]) == 8
    w0 = win["windows"][0]
    # the first window's centre crosses both wrap seams
    assert w0["i0"] + t < M <= w0["i0"] + t + c - 1 and w0["j0"] + t < M <= w0["j0"] + t + c - 1
    for w in win["windows"]:
        assert len(w["centre_rows"]) == c and all(len(r) == c for r in w["centre_rows"])
    w4 = _load("oracle_32768_windows_4096.json")
    t4 = w4["steps"]
    assert (t4, w4["centre"], w4["window"]) == (4096, 33, 2 * 4096 + 33)
    assert len(w4["windows"]) == 4
    v0 = w4["windows"][0]
    assert v0["i0"] + t4 < M <= v0["i0"] + t4 + c - 1 and v0["j0"] + t4 < M <= v0["j0"] + t4 + c - 1
    ens = _load("oracle_ensemble_subset.json")
    mod = _script()
    p = ensemble_params(4096, seed=1)
    assert [r["index"] for r in ens["lattices"]] == mod.ensemble_subset_indices(p)
    all512 = _load("oracle_ensemble_all_512.json")
    assert all512["steps"] == 512 and len(all512["digests"]) == 4096
    assert all(len(d) == 32 and int(d, 16) >= 0 for d in all512["digests"])
    e256 = _load("oracle_ensemble_256.json")
    assert e256["steps"] == 10000
    assert [r["index"] for r in e256["lattices"]] == list(range(0, 4096, 16))
    assert all((r["M"], r["N"]) == (int(p["M"][r["index"]]), int(p["N"][r["index"]]))
               for r in e256["lattices"])


def test_smallest_ensemble_record_recomputes_from_the_oracle():
    mod = _script()
    ens = _load("oracle_ensemble_subset.json")
    rec = min(ens["lattices"], key=lambda r: r["M"] * r["N"])
    p = ensemble_params(4096, seed=1)
    l = rec["index"]
    g0 = oracle.init(rec["M"], rec["N"], int(p["seed"][l]), float(p["p_lr"][l]),
                     float(p["p_tb"][l]))
    g, lr, tb = oracle.run(g0, ens["steps"], threads=os.cpu_count() or 1)
    got = mod.record(g, lr, tb)
    for key, val in got.items():
        assert rec[key] == val, key
    assert isinstance(rec["first_zero_step"], int) and np.all(lr >= 0)


def test_smallest_record_of_the_256_lattice_file_recomputes():
    """The smallest lattice of the seeded 256-lattice subset (10^4 steps),
    recomputed from the oracle."""
    mod = _script()
    e256 = _load("oracle_ensemble_256.json")
    rec = min(e256["lattices"], key=lambda r: r["M"] * r["N"])
    p = ensemble_params(4096, seed=1)
    l = rec["index"]
    g0 = oracle.init(rec["M"], rec["N"], int(p["seed"][l]), float(p["p_lr"][l]),
                     float(p["p_tb"][l]))
    g, lr, tb = oracle.run(g0, e256["steps"], threads=os.cpu_count() or 1)
    got = mod.record(g, lr, tb)
    for key, val in got.items():
        assert rec[key] == val, key


def test_smallest_records_of_the_whole_ensemble_files_recompute():
    """The three smallest lattices of the 512-step file, recomputed from the
    oracle."""
    mod = _script()
    p = ensemble_params(4096, seed=1)
    cells = p["M"].astype(np.int64) * p["N"].astype(np.int64)
    all512 = _load("oracle_ensemble_all_512.json")
    for l in np.argsort(cells, kind="stable")[:3]:
        l = int(l)
        g0 = oracle.init(int(p["M"][l]), int(p["N"][l]), int(p["seed"][l]),
                         float(p["p_lr"][l]), float(p["p_tb"][l]))
        g, lr, tb = oracle.run(g0, 512)
        assert mod.lattice_digest(g, lr, tb) == all512["digests"][l], l
