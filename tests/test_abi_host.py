"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports every symbol the
header declares, and validates formulas on the host before any device work."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2603_28796_b300 import _abi, build, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "gs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", text)))


def test_library_loads_and_exports_every_declared_symbol():
    L = ctypes.CDLL(build.LIB)
    declared = header_functions()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(L, name), name
    assert set(declared) == set(_abi.EXPORTED)


def test_debug_library_exports_the_same_symbols():
    L = ctypes.CDLL(build.LIB_DEBUG)
    for name in header_functions():
        assert hasattr(L, name), name


def test_status_strings():
    assert _abi.gs_status_str(0) == "ok"
    assert "timed out" in _abi.gs_status_str(6)
    assert _abi.gs_status_str(99) == "unknown status"


def test_adam_defaults_follow_the_paper():
    a = _abi.gs_adam_default()
    # lr 0.5 on each of the two logits == lr 1.0 on their difference; tau = 1.0
    assert (a.lr, a.beta1, a.beta2, a.eps, a.tau) == (1.0, 0.9, 0.999, 1e-8, 1.0)


def test_inspect_statistics():
    clauses = [[], [3], [-7, 7], [5, 5, -2], [1, 2, 3]]
    cp = np.cumsum([0] + [len(c) for c in clauses]).astype(np.int64)
    lits = np.array([l for c in clauses for l in c], dtype=np.int32)
    info = _abi.gs_inspect_cnf(8, cp, lits)
    assert info["n_vars"] == 8 and info["n_clauses"] == 5 and info["nnz"] == 9
    assert info["n_empty"] == 1 and info["n_unit"] == 1 and info["n_taut"] == 1 and info["n_dup"] == 1
    assert info["max_k"] == 3
    # occurrence codes: one per other literal of each occurrence, one for each unit clause
    assert info["n_occ_codes"] == 1 + 2 * 1 + 3 * 2 + 3 * 2


def test_inspect_splits_hub_variables():
    n, m = 50, 400
    rng = np.random.default_rng(1)
    clauses = [[1] + list(rng.choice(np.arange(2, n + 1), 2, replace=False)) for _ in range(m)]
    cp = np.cumsum([0] + [3] * m).astype(np.int64)
    lits = np.array(clauses, dtype=np.int32).ravel()
    info = _abi.gs_inspect_cnf(n, cp, lits)
    assert info["n_split"] >= 1   # variable 1 has 400 occurrences * 2 codes > one tile


@pytest.mark.parametrize(
    "n,cp,lits,status",
    [
        (3, [0, 2], [1, 4], 1),              # literal beyond n
        (3, [0, 2], [1, 0], 1),              # literal 0
        (3, [0, 2, 1], [1, 2], 1),           # decreasing clause_ptr
        (3, [1, 2], [1, 2], 1),              # clause_ptr[0] != 0
        (-1, [0], [], 1),                    # negative n
        (3, [0, 300], list(range(1, 4)) * 100, 5),   # clause wider than 256
        (2 ** 28, [0], [], 5),               # too many variables
    ],
)
def test_inspect_rejects_bad_input(n, cp, lits, status):
    with pytest.raises(_abi.GSError) as ei:
        _abi.gs_inspect_cnf(n, np.array(cp, dtype=np.int64), np.array(lits, dtype=np.int32))
    assert ei.value.status == status
    assert _abi.gs_last_error() != ""


def test_load_rejects_bad_input_before_device_work():
    # argument validation happens on the host, synchronously, before any CUDA call
    with pytest.raises(_abi.GSError) as ei:
        _abi.gs_load_cnf(3, np.array([0, 2], dtype=np.int64), np.array([1, -9], dtype=np.int32), stream=0)
    assert ei.value.status == 1


def test_dimacs_parse_errors(tmp_path):
    bad = {
        "no_header.cnf": "1 2 0\n",
        "bad_token.cnf": "p cnf 3 1\n1 x 0\n",
        "unterminated.cnf": "p cnf 3 1\n1 2\n",
        "count.cnf": "p cnf 3 2\n1 2 0\n",
        "range.cnf": "p cnf 3 1\n1 5 0\n",
    }
    for name, text in bad.items():
        p = tmp_path / name
        p.write_text(text)
        with pytest.raises(_abi.GSError) as ei:
            _abi.gs_load_dimacs(str(p), stream=0)
        assert ei.value.status == 2, name


def test_workload_catalogue_sizes():
    w = synth.WORKLOADS
    assert (w["differentiation"]["n"], w["differentiation"]["m"], w["differentiation"]["B"]) == (100_000, 426_000, 1024)
    assert (w["plain"]["n"], w["plain"]["m"], w["plain"]["B"]) == (200, 852, 64)
    assert (w["precision"]["n"], w["precision"]["m"], w["precision"]["B"]) == (2_000_000, 8_000_000, 256)
    assert (w["structured"]["n"], w["structured"]["m"], w["structured"]["B"]) == (10_000_000, 42_000_000, 32)


@pytest.mark.parametrize("seed", range(6))
def test_inspect_statistics_random(seed):
    """Loader statistics against a direct Python count on random formulas with empty, unit,
    duplicated-literal and tautological clauses (the multi-threaded tile builder must see every
    clause exactly once)."""
    from tests import _brute
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 3000))
    clauses = _brute.random_clauses(rng, n, int(rng.integers(1, 20000)), 0, 9, distinct=bool(seed % 2))
    cp, lits = _brute.csr_of(clauses)
    info = _abi.gs_inspect_cnf(n, cp, lits)
    widths = np.array([len(c) for c in clauses])
    assert info["n_clauses"] == len(clauses) and info["nnz"] == widths.sum() and info["max_k"] == widths.max()
    assert info["n_empty"] == (widths == 0).sum() and info["n_unit"] == (widths == 1).sum()
    assert info["n_dup"] == sum(len(set(c)) < len(c) for c in clauses)
    assert info["n_taut"] == sum(any(-l in c for l in c) for c in clauses)
    assert info["n_occ_codes"] == int((widths * np.maximum(widths - 1, 1)).sum())
    assert info["n_fwd_tiles"] >= -(-widths.sum() // 512)
    used = np.unique(np.abs(lits))
    assert info["n_var_tiles"] >= -(-len(used) // 64)


def test_load_with_tile_caps_out_of_range_is_refused_on_the_host():
    cnf = synth.planted_ksat(100, 400, 3, seed=4)
    for bad in (dict(fwd_tile_codes=16), dict(fwd_tile_codes=1024), dict(var_tile_codes=400),
                dict(own_item_codes=100), dict(own_item_codes=70000)):
        with pytest.raises(_abi.GSError) as ei:
            _abi.gs_load_batch_opts([cnf.n_vars], [cnf.n_clauses], cnf.clause_ptr, cnf.lits, stream=0, **bad)
        assert ei.value.status == 1 and "tile caps" in str(ei.value)


def test_inspect_reports_default_tile_caps():
    cnf = synth.planted_ksat(100, 400, 3, seed=4)
    info = _abi.gs_inspect_cnf(cnf.n_vars, cnf.clause_ptr, cnf.lits)
    assert (info["fwd_tile_codes"], info["var_tile_codes"], info["own_item_codes"]) == (512, 384, 4096)


def test_tuning_cache_key_and_round_trip(tmp_path, monkeypatch):
    from paper_2603_28796_b300 import tuning

    a = synth.planted_ksat(300, 1200, 3, seed=1)
    b = synth.planted_ksat(300, 1200, 4, seed=1)       # same sizes, other clause widths
    sa = tuning.signature(a, 64, "f32", device="dev0")
    sb = tuning.signature(b, 64, "f32", device="dev0")
    assert sa["n"] == 300 and sa["m"] == 1200 and sa["nnz"] == 3600 and sa["n_inst"] == 1
    assert sa["khist"] != sb["khist"]
    assert tuning.signature(a, 128, "f32", device="dev0") != sa
    batch = synth.concat([a, b])
    sc = tuning.signature(batch, 64, "f32", device="dev0")
    assert sc["n_inst"] == 2 and sc["n"] == 600 and sc["nnz"] == 3600 + 4800
    path = str(tmp_path / "cache.json")
    monkeypatch.setenv("GS_TUNING_CACHE", path)
    assert tuning.lookup(sa) is None
    entry = {"plan": {"fwd_tile_codes": 256, "var_tile_codes": 192, "own_item_codes": 2048},
             "tuning": {"var_lanes": 16, "fwd_lanes": 32, "var_gather": 1, "loss_mode": 1, "var_split": 2},
             "ms_per_step": 1.0}
    tuning.save_entry(sa, entry)
    hit = tuning.lookup(sa)
    assert hit["plan"] == entry["plan"] and hit["tuning"] == entry["tuning"] and hit["key"] == sa
    assert tuning.lookup(sb) is None
