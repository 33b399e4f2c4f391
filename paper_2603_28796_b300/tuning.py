"""Autotuner over the kernels' work-item shapes, with a persistent cache.

Two kinds of knobs shape the work of the variable-major pass, the forward pass and the check:

- load-time tile sizes (``gs_plan_opts``): literal codes per clause tile, occurrence codes per
  occurrence tile, codes per owned-variable item. They fix the index structures, so each setting
  is a separate load of the formula;
- run-time settings (``gs_tuning``): candidates per warp (lanes per candidate chunk) of the
  variable pass and of the forward pass, the gather form, the loss mode, shared or owned
  variables. ``gs_autotune`` searches these on a loaded problem.

``tuned_problem`` loads the formula with each tile setting of a small grid, lets ``gs_autotune``
pick the run-time settings, times the whole step (fused step + check) and keeps the fastest. The
choice is cached in a JSON file keyed by the device name and the problem's shape: variables,
clauses, literals, instances, the clause-width histogram, B and the storage dtype. A later call
with the same key loads the formula once with the cached tile sizes and applies the cached
run-time settings without searching. Lookups read the user's cache
(``~/.cache/galoissat/tuning_cache.json``) and then the cache the package ships with entries
measured on B300 for its benchmark workloads (``tuning_cache.json`` beside this file); new
entries go to the user's cache. ``GS_TUNING_CACHE`` names one file to use instead of both.
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics
import time
from typing import Optional, Tuple

import numpy as np

from . import _abi

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(HERE, "tuning_cache.json")

# Tile-size grid searched at load time (0 = the library default: 512 / 384 / 4096 codes).
TILE_GRID = (
    {"fwd_tile_codes": 0, "var_tile_codes": 0, "own_item_codes": 0},
    {"fwd_tile_codes": 256, "var_tile_codes": 192, "own_item_codes": 2048},
    {"fwd_tile_codes": 512, "var_tile_codes": 384, "own_item_codes": 8192},
)


USER_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "galoissat", "tuning_cache.json")


def cache_path() -> str:
    """The file new entries are written to."""
    return os.environ.get("GS_TUNING_CACHE", USER_CACHE)


def lookup_paths():
    env = os.environ.get("GS_TUNING_CACHE")
    return [env] if env else [USER_CACHE, DEFAULT_CACHE]


def _arrays(cnf):
    """(n_vars [n_inst], n_clauses [n_inst], clause_ptr, lits) of a CNF or a Batch."""
    if hasattr(cnf, "n_inst"):
        return (np.asarray(cnf.n_vars, dtype=np.int64), np.asarray(cnf.n_clauses, dtype=np.int64),
                cnf.clause_ptr, cnf.lits)
    return (np.array([cnf.n_vars], dtype=np.int64), np.array([cnf.n_clauses], dtype=np.int64),
            cnf.clause_ptr, cnf.lits)


def signature(cnf, B: int, dtype: str, device: Optional[str] = None) -> dict:
    """The cache key of a formula (or batch) stepped with B candidates stored as dtype."""
    nv, nc, cp, lits = _arrays(cnf)
    widths = np.diff(np.asarray(cp, dtype=np.int64))
    hist = np.bincount(widths) if widths.size else np.zeros(1, dtype=np.int64)
    if device is None:
        import torch

        device = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return {"device": device, "n": int(nv.sum()), "m": int(nc.sum()), "nnz": int(cp[-1]) if len(cp) else 0,
            "n_inst": int(nv.size), "B": int(B), "dtype": str(dtype),
            "khist": hashlib.sha1(np.ascontiguousarray(hist, dtype=np.int64).tobytes()).hexdigest()[:16]}


def _key(sig: dict) -> str:
    return "|".join("%s=%s" % (k, sig[k]) for k in ("device", "n", "m", "nnz", "n_inst", "B", "dtype", "khist"))


def load_cache(path: Optional[str] = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def lookup(sig: dict) -> Optional[dict]:
    for path in lookup_paths():
        hit = load_cache(path).get(_key(sig))
        if hit is not None:
            return hit
    return None


def save_entry(sig: dict, entry: dict, path: Optional[str] = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    data = load_cache(path)
    data[_key(sig)] = dict(entry, key=sig)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def load_problem(cnf, opts: Optional[dict] = None) -> _abi.Problem:
    nv, nc, cp, lits = _arrays(cnf)
    o = opts or {}
    return _abi.gs_load_batch_opts(nv, nc, cp, lits, fwd_tile_codes=o.get("fwd_tile_codes", 0),
                                   var_tile_codes=o.get("var_tile_codes", 0),
                                   own_item_codes=o.get("own_item_codes", 0))


def time_step(prob: _abi.Problem, B: int, dtype: str, steps: int = 6) -> float:
    """Mean ms of the whole step (fused step with loss and bits, then the check) on the
    problem's current tuning, after two warm-up steps."""
    import torch

    from .engine import Engine

    eng = Engine(prob, B, dtype, seed=1)
    for _ in range(2):
        eng.step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        a.record()
        eng.step()
        b.record()
    torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    del eng
    torch.cuda.empty_cache()
    return ms


def tuned_problem(cnf, B: int, dtype: str, search_tiles: bool = True, use_cache: bool = True,
                  write_cache: bool = True) -> Tuple[_abi.Problem, dict]:
    """A loaded problem with its tile sizes and run-time settings tuned for B candidates stored as
    dtype. Returns (problem, record); record holds the tile sizes, the run-time settings, the
    timed ms per step of each tile setting tried (empty on a cache hit) and where the choice came
    from ("cache" or "search")."""
    sig = signature(cnf, B, dtype)
    if use_cache:
        hit = lookup(sig)
        if hit is not None:
            prob = load_problem(cnf, hit["plan"])
            t = hit["tuning"]
            _abi.gs_set_tuning(prob, var_lanes=t["var_lanes"], fwd_lanes=t["fwd_lanes"], var_gather=t["var_gather"],
                               loss_mode=t["loss_mode"], var_split=t["var_split"])
            _abi.gs_reserve(prob, B, dtype)
            return prob, {"plan": hit["plan"], "tuning": t, "source": "cache", "tried": []}
    grid = TILE_GRID if search_tiles else TILE_GRID[:1]
    best = None
    tried = []
    t0 = time.perf_counter()
    for opts in grid:
        prob = load_problem(cnf, opts)
        tuning = _abi.gs_autotune(prob, B, dtype)
        ms = time_step(prob, B, dtype)
        info = prob.info()
        plan = {"fwd_tile_codes": info["fwd_tile_codes"], "var_tile_codes": info["var_tile_codes"],
                "own_item_codes": info["own_item_codes"]}
        tried.append({"plan": plan, "tuning": tuning, "ms_per_step": ms})
        if best is None or ms < best[0]:
            if best is not None:
                best[1].close()
            best = (ms, prob, plan, tuning)
        else:
            prob.close()
    ms, prob, plan, tuning = best
    rec = {"plan": plan, "tuning": tuning, "ms_per_step": ms, "source": "search", "tried": tried,
           "search_s": time.perf_counter() - t0}
    if write_cache:
        try:
            save_entry(sig, {"plan": plan, "tuning": tuning, "ms_per_step": ms})
        except OSError:
            pass
    return prob, rec
