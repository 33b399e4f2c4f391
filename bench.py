#!/usr/bin/env python
"""Benchmark of the differentiable solving stage (fwd+bwd clause-literal evals/s).

One step = one pass of the whole hot path over one batch of candidates: relaxed values,
forward clause products + loss, backward leave-one-out gradient, Adam update, rounding (all in
the fused gs_step) and the exact bit-packed check (gs_check_bits). Workload: planted uniform
random 3-SAT, n = 100,000, m = 426,000, B = 1024 candidates, float32 (the differentiation
workload). One clause-literal eval = one (literal occurrence, candidate) pair taken through
forward and backward in a step, so a step is nnz * B evals.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Under torchrun (N > 1) every rank optimises its own batch of candidates of the same formula
(weak scaling, no data-path collective); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "differentiation"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--dtype", default=None, help="override the storage dtype (f32, bf16, f16)")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink the workload's formula (n and m) by this factor, for profiling small cases")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--launch", choices=["graph", "eager"], default="graph",
                    help="graph: the K timed steps are captured once in a CUDA graph and replayed once in the "
                         "timed region (the engine's own run loop); eager: one host call per kernel launch")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-autotune", action="store_true", help="skip gs_autotune (use defaults / --var-* flags)")
    ap.add_argument("--legs", default="st,pool,precision,tseitin,plain,structured,batching",
                    help="extra single-GPU measurements added to the line under 'legs' (comma list of st, pool, "
                         "precision, tseitin, plain, structured, batching; 'none' for none)")
    ap.add_argument("--leg-steps", type=int, default=50, help="timed steps of each extra leg")
    ap.add_argument("--var-lanes", type=int, default=0, help="cap on lanes per candidate chunk (gs_set_tuning)")
    ap.add_argument("--var-gather", type=int, default=0, help="0: automatic, 1: register loads, 2: TMA gather4 ring (gs_set_tuning)")
    ap.add_argument("--var-split", type=int, default=0,
                    help="0: automatic, 1: lane groups share each variable, 2: lane groups own whole variables (gs_set_tuning)")
    ap.add_argument("--loss-mode", type=int, default=0,
                    help="0: automatic, 1: loss credited in the variable pass, 2: separate forward pass (gs_set_tuning)")
    return ap.parse_args()


# ---------------------------------------------------------------------------------------------
def workload_setup(name, dtype_override=None, scale=1.0):
    from paper_2603_28796_b300 import synth

    w = synth.WORKLOADS[name]
    cnf = synth.workload_cnf(name, seed=0, scale=scale)
    dtype = dtype_override or w["dtype"]
    return cnf, int(w["B"]), dtype, w["desc"]


def kernel_source_hash():
    """sha256 of the sources the variable-major pass is compiled from: a traffic figure taken
    by ncu is only reported while these are unchanged."""
    import hashlib

    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2603_28796_b300", "csrc")
    for name in ("gs_kernels.cu", "gs_var.cuh", "gs_device.cuh", "gs_internal.h"):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


def recorded_traffic(workload, B, dtype):
    """DRAM read+write bytes of one launch of the variable pass from the committed ncu summary,
    or None when it was taken on another workload or an older kernel source."""
    try:
        with open(os.path.join(ROOT, "profiles", "var_pass_traffic.json")) as f:
            tr = json.load(f)
    except Exception:
        return None, None
    if tr.get("workload") != workload or tr.get("B") != B or tr.get("dtype") != dtype:
        return None, "recorded for another workload"
    if tr.get("source_sha256") != kernel_source_hash():
        return None, "recorded on an older kernel source"
    return tr.get("bytes_per_launch"), "ncu capture (profiles/var_pass_traffic.json)"


def gather_probe(torch, x, row_bytes, n_gathers, reps=5, seed=0):
    """Random row-gather rate (GB/s) of the memory hierarchy for rows of row_bytes at the row
    stride of x (a [n, ldB] tensor), the rows being drawn uniformly from all n rows: the working
    set of one candidate chunk of the variable pass. Uses the library's probe kernel."""
    from paper_2603_28796_b300 import _abi

    n = x.shape[0]
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    idx = torch.randint(0, n, (n_gathers,), generator=g, dtype=torch.int32).to(x.device)
    base = x.as_strided((n, x.stride(0)), (x.stride(0), 1))
    sink = torch.zeros(1, dtype=torch.int32, device=x.device)
    for _ in range(2):
        _abi.gs_gather_probe(base, row_bytes, idx, sink)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        _abi.gs_gather_probe(base, row_bytes, idx, sink)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    return n_gathers * row_bytes / (ms / 1000.0) / 1e9, ms


def load_tuned(cnf, B, dtype, search_tiles=True):
    """The workload's problem, loaded with its tuned tile sizes and run-time settings (the
    package's tuning cache, else a search that is then cached); returns (problem, record)."""
    from paper_2603_28796_b300 import tuning

    prob, rec = tuning.tuned_problem(cnf, B, dtype, search_tiles=search_tiles)
    out = {"plan": rec["plan"], "tuning": rec["tuning"], "source": rec["source"]}
    if rec.get("tried"):
        out["tried"] = [{"plan": t["plan"], "ms_per_step": t["ms_per_step"]} for t in rec["tried"]]
    return prob, out


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", "gs_clocks_%d_%d.csv" % (os.getpid(), gpu_index))

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        rows = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()
            try:
                with open(self.path) as f:
                    rows = [r.strip().split(", ") for r in f if r.strip()]
                os.remove(self.path)
            except Exception:
                rows = []
        if not rows:
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=10)
                rows = [r.strip().split(", ") for r in out.stdout.splitlines() if r.strip()]
            except Exception:
                return None
        sm = [float(r[1]) for r in rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) > 8:
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------------------------------------
def cpu_oracle_sample(cnf, B_sample, seed, target_s, max_steps=None):
    """Times the FP64 oracle (as it stands) on B_sample candidates of the workload.
    Returns (evals_per_s, seconds, steps, threads)."""
    import oracle
    from paper_2603_28796_b300 import synth

    if hasattr(cnf, "n_inst"):       # a batch: the oracle runs its first instance
        cnf = cnf.instance(0)
    n = cnf.n_vars
    d = synth.init_delta(n, B_sample, seed).astype(np.float64)
    m = np.zeros_like(d)
    v = np.zeros_like(d)
    x = oracle.relax(d)

    def one(t, d, m, v, x):
        oracle.forward(n, cnf.clause_ptr, cnf.lits, x)
        g, _ = oracle.backward(n, cnf.clause_ptr, cnf.lits, x)
        d, m, v, x = oracle.adam(d, m, v, g, t)
        oracle.round_check(n, cnf.clause_ptr, cnf.lits, d)
        return d, m, v, x

    t0 = time.perf_counter()
    d, m, v, x = one(1, d, m, v, x)
    t1 = time.perf_counter() - t0
    steps = 1
    if max_steps is None:
        want = max(1, int(target_s / max(t1, 1e-3)))
        extra = min(want - 1, 50)
    else:
        extra = max_steps - 1
    t0 = time.perf_counter()
    for t in range(2, 2 + extra):
        d, m, v, x = one(t, d, m, v, x)
    total = t1 + (time.perf_counter() - t0)
    steps += extra
    return cnf.nnz * B_sample * steps / total, total, steps, oracle.threads()


# ---------------------------------------------------------------------------------------------
# Extra single-GPU legs: the other workloads, each timed on its own problem after the headline.
def _timed_steps(torch, eng, K, W):
    """Mean ms per step (fused step + check) over K eager steps after W warm-up steps, and the
    mean ms of the gs_step calls alone."""
    from paper_2603_28796_b300 import _abi

    for _ in range(max(3, W)):
        eng.step()
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for k in range(K):
        eng.t += 1
        ev[k][0].record()
        _abi.gs_step(eng.prob, eng.delta, eng.m, eng.v, eng.t, x_in=eng.x[eng.cur], x_out=eng.x[eng.cur ^ 1],
                     loss=eng.loss, bits=eng.bits)
        ev[k][1].record()
        eng.cur ^= 1
        _abi.gs_check_bits(eng.prob, eng.bits, eng.B, eng.unsat, eng.best)
    t1.record()
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / K, statistics.mean(e[0].elapsed_time(e[1]) for e in ev)


def _gather_model_bytes(nnz, n, B, s):
    return nnz * B * 2 * s + n * B * (24 + s)


def _row_read_stats(prob, B, s, step_ms):
    """Actual row reads of one variable pass: every occurrence code (one other literal of one
    occurrence, sum over clauses of k(k-1)) reads one candidate row slice of B*s bytes, which
    for clauses wider than 3 is more than the gather model's two reads per literal."""
    rr = prob.info()["n_occ_codes"] * B * s
    return {"row_read_bytes": rr, "row_read_GBps": rr / (step_ms / 1000.0) / 1e9}


def _compulsory_bytes(n, B, s):
    """Strict DRAM floor of one fused step: delta, m, v read and written, x read once and
    written once, the bit rows written (index data excluded)."""
    return n * B * (24 + 2 * s) + n * ((B + 63) // 64) * 8


def leg_precision(torch, args, peak):
    """Mixed-width power-law workload: BF16 storage (the batched form) vs FP32 (the plain form)
    on the same GPU, and the gradient error of the BF16 storage against the FP32 one at the same
    logits (relative L2 norm over all coordinates and worst coordinate relative to the RMS)."""
    from paper_2603_28796_b300 import _abi, synth
    from paper_2603_28796_b300.engine import Engine, candidates

    cnf, B, _, desc = workload_setup("precision")
    n, nnz = cnf.n_vars, cnf.nnz
    out = {"workload": desc, "n": n, "m": cnf.n_clauses, "nnz": nnz, "B": B}
    for dtype, s in (("bf16", 2), ("f32", 4)):
        prob, tuning = load_tuned(cnf, B, dtype)
        eng = Engine(prob, B, dtype, seed=11)
        ms, step_ms = _timed_steps(torch, eng, args.leg_steps, args.warmup)
        gm = _gather_model_bytes(nnz, B=B, n=n, s=s)
        cb = _compulsory_bytes(n, B, s)
        out[dtype] = {"ms_per_step": ms, "steps_per_s": 1000.0 / ms, "evals_per_s": nnz * B / (ms / 1000.0),
                      "gs_step_ms": step_ms, "gather_model_GBps": gm / (step_ms / 1000.0) / 1e9,
                      "gather_model_frac": gm / (step_ms / 1000.0) / 1e9 / peak,
                      "compulsory_frac": cb / (step_ms / 1000.0) / 1e9 / peak, "tuning": tuning,
                      **_row_read_stats(prob, B, s, step_ms)}
        del eng
        if dtype == "bf16":
            prob.close()
        torch.cuda.empty_cache()
    out["bf16_speedup"] = out["f32"]["ms_per_step"] / out["bf16"]["ms_per_step"]
    delta = candidates(n, B)
    delta.copy_(torch.from_numpy(synth.init_delta(n, B, seed=12)).cuda()[:, :B])
    x32, x16 = candidates(n, B), candidates(n, B, torch.bfloat16)
    _abi.gs_relax(prob, delta, x32)
    _abi.gs_relax(prob, delta, x16)
    g32 = _abi.gs_backward(prob, x32).double()
    g16 = _abi.gs_backward(prob, x16).double()
    diff = g16 - g32
    rms = float(g32.pow(2).mean().sqrt())
    out["grad_error_bf16_vs_f32"] = {
        "rel_l2": float(diff.norm() / g32.norm()), "max_abs_over_rms": float(diff.abs().max()) / rms,
        "sign_agreement": float(((g16 > 0) == (g32 > 0)).double().mean()),
        "note": "gradients at the same float32 logits; x stored as BF16 (round to nearest even) vs FP32",
    }
    prob.close()
    return out


def leg_plain(torch, args):
    """Plain method: n=200, m=852, B=64, 1000 steps captured in one CUDA graph (the whole
    problem and state fit in L2, so this is launch- and latency-bound, not HBM-bound)."""
    from paper_2603_28796_b300 import _abi
    from paper_2603_28796_b300.engine import Engine

    cnf, B, dtype, desc = workload_setup("plain")
    prob, tuning = load_tuned(cnf, B, dtype)
    eng = Engine(prob, B, dtype, seed=5)
    steps = 1000
    eng.run(steps, graph=True)           # warm-up replay (capture included)
    torch.cuda.synchronize()
    g = eng.capture(steps)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    g.replay()
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    unsat = eng.unsat.cpu().numpy()[0]
    out = {"workload": desc, "steps": steps, "graph": True, "ms_total": ms, "us_per_step": 1000.0 * ms / steps,
           "steps_per_s": 1000.0 * steps / ms, "evals_per_s": cnf.nnz * B * steps / (ms / 1000.0),
           "solved_candidates": int((unsat == 0).sum()), "tuning": tuning,
           "l2": "whole problem and state are L2-resident (1.7 MB); no flush"}
    del g, eng
    prob.close()
    return out


def leg_structured(torch, args, peak):
    """Community-structured workload: n=10,000,000, m=42,000,000, k uniform 2..8, B=32, BF16."""
    from paper_2603_28796_b300 import _abi
    from paper_2603_28796_b300.engine import Engine

    cnf, B, dtype, desc = workload_setup("structured")
    prob, tuning = load_tuned(cnf, B, dtype)
    eng = Engine(prob, B, dtype, seed=21)
    ms, step_ms = _timed_steps(torch, eng, args.leg_steps, args.warmup)
    s = 2
    gm = _gather_model_bytes(cnf.nnz, cnf.n_vars, B, s)
    cb = _compulsory_bytes(cnf.n_vars, B, s)
    out = {"workload": desc, "n": cnf.n_vars, "m": cnf.n_clauses, "nnz": cnf.nnz, "B": B, "dtype": dtype,
           "ms_per_step": ms, "steps_per_s": 1000.0 / ms, "evals_per_s": cnf.nnz * B / (ms / 1000.0),
           "gs_step_ms": step_ms, "gather_model_GBps": gm / (step_ms / 1000.0) / 1e9,
           "gather_model_frac": gm / (step_ms / 1000.0) / 1e9 / peak,
           "compulsory_frac": cb / (step_ms / 1000.0) / 1e9 / peak, "tuning": tuning,
           **_row_read_stats(prob, B, s, step_ms)}
    del eng
    prob.close()
    torch.cuda.empty_cache()
    return out


def leg_batching(torch, args, peak):
    """512 uneven instances, B=64 each: one batched problem stepped by one persistent launch
    per kernel, vs a loop over 512 separately loaded problems stepping the same state rows; then
    the same batch with BF16 storage (steps/s against FP32 and the gradient error of BF16
    storage)."""
    from paper_2603_28796_b300 import _abi
    from paper_2603_28796_b300.engine import Engine

    bt = workload_setup("batching")
    batch, B, dtype, desc = bt
    prob, tuning = load_tuned(batch, B, dtype, search_tiles=False)
    eng = Engine(prob, B, dtype, seed=31)
    nnz, n = int(batch.clause_ptr[-1]), int(sum(batch.n_vars))
    ms, step_ms = _timed_steps(torch, eng, max(5, args.leg_steps // 5), args.warmup)
    gm = _gather_model_bytes(nnz, n, B, 4)
    cb = _compulsory_bytes(n, B, 4)
    # the whole iteration loop captured in one CUDA graph
    Kg = max(4, (args.leg_steps // 5) // 2 * 2)
    graph = eng.capture(Kg)
    torch.cuda.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record()
    graph.replay()
    g1.record()
    torch.cuda.synchronize()
    ms_graph = g0.elapsed_time(g1) / Kg
    del graph
    out = {"workload": desc, "n": n, "m": int(sum(batch.n_clauses)), "nnz": nnz, "B": B, "dtype": dtype,
           "batched": {"ms_per_step": ms, "steps_per_s": 1000.0 / ms, "evals_per_s": nnz * B / (ms / 1000.0),
                       "gs_step_ms": step_ms, "gather_model_frac": gm / (step_ms / 1000.0) / 1e9 / peak,
                       "compulsory_frac": cb / (step_ms / 1000.0) / 1e9 / peak, "tuning": tuning,
                       **_row_read_stats(prob, B, 4, step_ms)},
           "batched_graph": {"ms_per_step": ms_graph, "steps_per_s": 1000.0 / ms_graph,
                             "evals_per_s": nnz * B / (ms_graph / 1000.0), "steps": Kg}}
    # per-instance loop over the same state rows
    vo = np.concatenate([[0], np.cumsum(batch.n_vars)]).astype(np.int64)
    co = np.concatenate([[0], np.cumsum(batch.n_clauses)]).astype(np.int64)
    probs = []
    for i in range(batch.n_inst):
        a, b = batch.clause_ptr[co[i]], batch.clause_ptr[co[i + 1]]
        probs.append(_abi.gs_load_cnf(int(batch.n_vars[i]), batch.clause_ptr[co[i]:co[i + 1] + 1] - a,
                                      batch.lits[a:b]))
        _abi.gs_reserve(probs[-1], B, dtype)
    views = []
    for i in range(batch.n_inst):
        r0, r1 = vo[i], vo[i + 1]
        # state rows are views of the batched buffers (256-byte rows); bit rows (8 bytes) of an
        # instance need not start on a 16-byte boundary, so each instance gets its own
        bits_i = torch.zeros((max(int(r1 - r0), 1), eng.nwd), dtype=torch.int64, device=eng.delta.device)
        views.append((eng.delta[r0:r1], eng.m[r0:r1], eng.v[r0:r1], eng.x[0][r0:r1], eng.x[1][r0:r1],
                      eng.loss[i:i + 1], bits_i, eng.unsat[i:i + 1], eng.best[i:i + 1]))

    def loop_step():
        eng.t += 1
        for p, (d, mm, vv, x0, x1, lo, bi, un, be) in zip(probs, views):
            xi, xo = (x0, x1) if eng.cur == 0 else (x1, x0)
            _abi.gs_step(p, d, mm, vv, eng.t, x_in=xi, x_out=xo, loss=lo, bits=bi)
            _abi.gs_check_bits(p, bi, B, un, be)
        eng.cur ^= 1

    for _ in range(3):
        loop_step()
    torch.cuda.synchronize()
    K = max(5, args.leg_steps // 5)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(K):
        loop_step()
    t1.record()
    torch.cuda.synchronize()
    ms_loop = t0.elapsed_time(t1) / K
    out["per_instance_loop"] = {"ms_per_step": ms_loop, "steps_per_s": 1000.0 / ms_loop,
                                "evals_per_s": nnz * B / (ms_loop / 1000.0), "launch": "eager"}
    out["batched_speedup"] = ms_loop / ms
    for p in probs:
        p.close()
    del eng
    prob.close()
    torch.cuda.empty_cache()

    # The same batch with BF16 storage of the relaxed values (FP32 accumulation and Adam state),
    # its steps/s against the FP32 batch above, and the gradient error of BF16 storage against
    # FP32 storage at the same logits (seeded normal logits, scale 2).
    from paper_2603_28796_b300.engine import candidates
    prob16, tuning16 = load_tuned(batch, B, "bf16", search_tiles=False)
    eng16 = Engine(prob16, B, "bf16", seed=31)
    ms16, step16 = _timed_steps(torch, eng16, max(5, args.leg_steps // 5), args.warmup)
    gm16 = _gather_model_bytes(nnz, n, B, 2)
    cb16 = _compulsory_bytes(n, B, 2)
    out["batched_bf16"] = {"ms_per_step": ms16, "steps_per_s": 1000.0 / ms16, "evals_per_s": nnz * B / (ms16 / 1000.0),
                           "gs_step_ms": step16, "gather_model_frac": gm16 / (step16 / 1000.0) / 1e9 / peak,
                           "compulsory_frac": cb16 / (step16 / 1000.0) / 1e9 / peak, "tuning": tuning16,
                           **_row_read_stats(prob16, B, 2, step16)}
    out["bf16_speedup"] = ms / ms16
    del eng16
    torch.cuda.empty_cache()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(37)
    delta = candidates(n, B)
    delta.normal_(0.0, 2.0, generator=gen)
    x32, x16 = candidates(n, B), candidates(n, B, torch.bfloat16)
    _abi.gs_relax(prob16, delta, x32)
    _abi.gs_relax(prob16, delta, x16)
    del delta
    g32 = _abi.gs_backward(prob16, x32)
    del x32
    g16 = _abi.gs_backward(prob16, x16)
    del x16
    sq_d = sq_r = 0.0
    max_d = 0.0
    agree = 0
    for r0 in range(0, n, 1 << 20):
        a32 = g32[r0:r0 + (1 << 20)].double()
        d = g16[r0:r0 + (1 << 20)].double() - a32
        sq_d += float(d.pow(2).sum())
        sq_r += float(a32.pow(2).sum())
        max_d = max(max_d, float(d.abs().max()))
        agree += int(((a32 + d > 0) == (a32 > 0)).sum())
    rms = (sq_r / (n * B)) ** 0.5
    out["grad_error_bf16_vs_f32"] = {
        "rel_l2": (sq_d / sq_r) ** 0.5, "max_abs_over_rms": max_d / rms, "sign_agreement": agree / (n * B),
        "note": "gradients at the same float32 logits; x stored as BF16 (round to nearest even) vs FP32"}
    del g32, g16
    prob16.close()
    torch.cuda.empty_cache()
    return out


def leg_tseitin(torch, args, peak):
    """The paper's formulation vs the native one on the mixed-width power-law formula (FP32,
    B = 256): the width-3 chain normalisation of Eq. 6-8 (gs_tseitin3: more variables and
    clauses, every clause of width 3) against the formula with its own clause widths."""
    from paper_2603_28796_b300 import _abi, synth
    from paper_2603_28796_b300.engine import Engine

    cnf, B, _, desc = workload_setup("precision")
    n3, cp3, lits3 = _abi.gs_tseitin3(cnf.n_vars, cnf.clause_ptr, cnf.lits)
    out = {"workload": desc.replace("BF16 storage vs FP32", "FP32") + "; native widths vs width-3 chains (Eq. 6-8)",
           "B": B}
    for name, (n, cp, lits) in (("native", (cnf.n_vars, cnf.clause_ptr, cnf.lits)), ("width3", (n3, cp3, lits3))):
        prob, tuning = load_tuned(synth.CNF(n, cp, lits), B, "f32", search_tiles=False)
        eng = Engine(prob, B, "f32", seed=13)
        ms, step_ms = _timed_steps(torch, eng, args.leg_steps, args.warmup)
        nnz = int(cp[-1])
        out[name] = {"n": n, "m": int(cp.size - 1), "nnz": nnz, "ms_per_step": ms, "steps_per_s": 1000.0 / ms,
                     "evals_per_s": nnz * B / (ms / 1000.0), "gs_step_ms": step_ms, "tuning": tuning}
        del eng
        prob.close()
        torch.cuda.empty_cache()
    out["native_speedup"] = out["width3"]["ms_per_step"] / out["native"]["ms_per_step"]
    return out


def leg_pool(torch, args, peak):
    """Candidate pool and branching variables (Eq. 9, Lemma 1) on the differentiation workload after
    a few straight-through steps: N = 100 noisy samples of the highest-loss candidate with the top
    0.05 % most confident variables of each, and the d = 7 least confident variables."""
    from paper_2603_28796_b300 import _abi, pool
    from paper_2603_28796_b300.engine import STEngine

    cnf, B, _, desc = workload_setup("differentiation")
    prob = _abi.gs_load_cnf(cnf.n_vars, cnf.clause_ptr, cnf.lits)
    eng = STEngine(prob, B, seed=51, noise_seed=53)
    eng.run(20, graph=False)
    torch.cuda.synchronize()
    b_sel = pool.select_candidate(eng.unsat.cpu().numpy()[0], "max")
    N, S, d = pool.DEFAULT_N, pool.selection_size(cnf.n_vars), pool.DEFAULT_D

    def timed(fn, k=10):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(k):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    ms_pool = timed(lambda: _abi.gs_pool_sample(prob, eng.delta, b_sel, N, S, seed=7))
    ms_branch = timed(lambda: _abi.gs_branch_vars(prob, eng.delta, b_sel, d))
    out = {"workload": desc + ", straight-through state after 20 steps", "N": N, "S": S, "d": d,
           "pool_ms": ms_pool, "pool_keys_per_s": cnf.n_vars * N / (ms_pool / 1000.0),
           "branch_ms": ms_branch, "b_sel": b_sel,
           "method": "4-pass radix select of unique 64-bit keys, in-kernel Philox noise"}
    del eng
    prob.close()
    torch.cuda.empty_cache()
    return out


def leg_st(torch, args, peak):
    """The paper's own training forward on the differentiation workload: straight-through Gumbel
    (hard assignment in the forward pass, soft chain in the backward pass, noise drawn in the
    kernel). One step = gs_check_bits on the hard assignment (the loss) + gs_st_step."""
    from paper_2603_28796_b300 import _abi
    from paper_2603_28796_b300.engine import STEngine

    cnf, B, _, desc = workload_setup("differentiation")
    prob = _abi.gs_load_cnf(cnf.n_vars, cnf.clause_ptr, cnf.lits)
    eng = STEngine(prob, B, seed=41, noise_seed=43)
    for _ in range(max(3, args.warmup)):
        eng.step()
    torch.cuda.synchronize()
    K = max(args.leg_steps, 20)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for k in range(K):
        eng.t += 1
        _abi.gs_check_bits(prob, eng.bits[eng.cur], B, eng.unsat, eng.best)
        ev[k][0].record()
        _abi.gs_st_step(prob, eng.delta, eng.m, eng.v, eng.bits[eng.cur], eng.bits[eng.cur ^ 1], eng.t,
                        seed=eng.noise_seed, noise=eng.noise[eng.cur], noise_next_out=eng.noise[eng.cur ^ 1])
        ev[k][1].record()
        eng.cur ^= 1
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / K
    st_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
    n, nnz = cnf.n_vars, cnf.nnz
    compulsory = n * B * (24 + 8) + n * ((B + 63) // 64) * 8     # delta, m, v + noise ring + bits
    out = {"workload": desc + ", straight-through Gumbel", "ms_per_step": ms, "steps_per_s": 1000.0 / ms,
           "evals_per_s": nnz * B / (ms / 1000.0), "st_step_ms": st_ms,
           "compulsory_bytes": compulsory, "compulsory_GBps": compulsory / (st_ms / 1000.0) / 1e9,
           "compulsory_frac": compulsory / (st_ms / 1000.0) / 1e9 / peak,
           "median_unsat": float(np.median(eng.unsat.cpu().numpy()[0]))}
    del eng
    prob.close()
    torch.cuda.empty_cache()
    return out


def run_legs(torch, args, peak):
    names = [x for x in args.legs.split(",") if x and x != "none"]
    legs = {}
    for name in names:
        t0 = time.perf_counter()
        try:
            if name == "precision":
                legs[name] = leg_precision(torch, args, peak)
            elif name == "plain":
                legs[name] = leg_plain(torch, args)
            elif name == "structured":
                legs[name] = leg_structured(torch, args, peak)
            elif name == "st":
                legs[name] = leg_st(torch, args, peak)
            elif name == "tseitin":
                legs[name] = leg_tseitin(torch, args, peak)
            elif name == "pool":
                legs[name] = leg_pool(torch, args, peak)
            elif name == "batching":
                legs[name] = leg_batching(torch, args, peak)
            else:
                legs[name] = {"error": "unknown leg"}
                continue
        except Exception as e:   # a leg that cannot run (e.g. out of memory) is reported, not fatal
            legs[name] = {"error": "%s: %s" % (type(e).__name__, e)}
        legs[name]["wall_s"] = time.perf_counter() - t0
    return legs


# ---------------------------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cnf, B, dtype, desc = workload_setup(args.workload, args.dtype, args.scale)
    if hasattr(cnf, "n_inst"):       # a batch: the oracle runs its first instance
        desc += "; oracle sample: instance 0"
        cnf = cnf.instance(0)
    B_sample = 16
    import oracle

    oracle.build()
    # warm-up steps (untimed), then K timed oracle steps on the bounded sample
    cpu_oracle_sample(cnf, B_sample, 1, 0, max_steps=max(1, args.warmup))
    t0 = time.perf_counter()
    evs, secs, steps, cores = cpu_oracle_sample(cnf, B_sample, 2, 0, max_steps=max(1, args.steps))
    wall = time.perf_counter() - t0
    sample = "%d of %d candidates per step, %d steps, FP64 oracle (forward, backward, Adam, round+check)" % (
        B_sample, B, steps)
    line = {
        "impl": "reference", "metric": "fwd+bwd clause-literal evals/s", "value": evs, "unit": "evals/s",
        "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup, "ms_per_step": 1000.0 * secs / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "B_sample": B_sample, "nnz": cnf.nnz, "n": cnf.n_vars, "m": cnf.n_clauses},
        "cpu_baseline": {"value": evs, "unit": "evals/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": evs, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_native(args):
    import torch
    import torch.distributed as dist

    from paper_2603_28796_b300 import _abi, synth
    from paper_2603_28796_b300.engine import Engine, candidates

    from paper_2603_28796_b300 import shard

    rank, world, local = shard.init_from_env("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    cnf, B, dtype, desc = workload_setup(args.workload, args.dtype, args.scale)
    full = cnf
    inst_ids = None
    if hasattr(cnf, "n_inst"):
        # a batch of instances: under torchrun each rank takes a share of whole instances,
        # balanced by literal count (the job's total work is fixed: strong scaling)
        if world > 1:
            c_off = np.concatenate([[0], np.cumsum(cnf.n_clauses)]).astype(np.int64)
            inst_nnz = np.diff(cnf.clause_ptr[c_off])
            inst_ids = shard.partition_instances(inst_nnz, world)[rank]
            nv, nc, cp, lt = shard.sub_batch(cnf.n_vars, cnf.n_clauses, cnf.clause_ptr, cnf.lits, inst_ids)
            cnf = synth.Batch(nv, nc, cp, lt, np.zeros(int(nv.sum()), np.uint8), cnf.name)
        n, nnz, m = int(np.sum(cnf.n_vars)), int(cnf.clause_ptr[-1]), int(np.sum(cnf.n_clauses))
    else:
        n, nnz, m = cnf.n_vars, cnf.nnz, cnf.n_clauses
    if args.scale != 1.0:
        desc += " (formula scaled by %g: n=%d, m=%d)" % (args.scale, n, m)
    tune_rec = None
    if args.var_lanes or args.var_gather or args.var_split or args.loss_mode or args.no_autotune:
        if hasattr(cnf, "n_inst"):
            prob = _abi.gs_load_batch(cnf.n_vars, cnf.n_clauses, cnf.clause_ptr, cnf.lits)
        else:
            prob = _abi.gs_load_cnf(cnf.n_vars, cnf.clause_ptr, cnf.lits)
        _abi.gs_set_tuning(prob, var_lanes=args.var_lanes, var_gather=args.var_gather, var_split=args.var_split,
                           loss_mode=args.loss_mode)
    else:
        prob, tune_rec = load_tuned(cnf, B, dtype)
    tuning = _abi.gs_get_tuning(prob)
    info = prob.info()
    eng = Engine(prob, B, dtype, seed=shard.rank_seed(1, rank))
    evals_per_step = nnz * B
    s_bytes = {"f32": 4, "bf16": 2, "f16": 2}[dtype]

    for _ in range(max(3, args.warmup)):
        eng.step()
    torch.cuda.synchronize()

    K = args.steps

    def record_steps(ev):
        for k in range(K):
            e0, e1, e2 = ev[k]
            eng.t += 1
            e0.record()
            _abi.gs_step(prob, eng.delta, eng.m, eng.v, eng.t, x_in=eng.x[eng.cur], x_out=eng.x[eng.cur ^ 1],
                         loss=eng.loss, bits=eng.bits)
            e1.record()
            eng.cur ^= 1
            _abi.gs_check_bits(prob, eng.bits, B, eng.unsat, eng.best)
            e2.record()

    graph = None
    if args.launch == "graph":
        # The K timed steps (each: gs_step, then gs_check_bits), with the per-step timing events
        # as event-record nodes, are captured before the timed region; capture runs nothing.
        ev = [[torch.cuda.Event(enable_timing=True, external=True) for _ in range(3)] for _ in range(K)]
        t0, cur0 = eng.t, eng.cur
        graph = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream()
        cap.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(cap):
            with torch.cuda.graph(graph, stream=cap):
                record_steps(ev)
        torch.cuda.current_stream().wait_stream(cap)
        eng_after = (eng.t, eng.cur)
        eng.t, eng.cur = t0, cur0
    else:
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record()
    if graph is not None:
        graph.replay()
    else:
        record_steps(ev)
    t_end.record()
    torch.cuda.synchronize()
    if graph is not None:
        eng.t, eng.cur = eng_after
        del graph
    clocks = sampler.stop()
    if world > 1:
        dist.barrier()
    total_ms = t_start.elapsed_time(t_end)
    step_ms = [ev[k][0].elapsed_time(ev[k][1]) for k in range(K)]
    check_ms = [ev[k][1].elapsed_time(ev[k][2]) for k in range(K)]
    total_ms = shard.max_over_ranks(total_ms, device=dev)
    _abi.gs_sync_status(prob)
    # the run's one cross-rank exchange (outside the timed region): the best candidate over all
    # ranks and its rounded assignment
    if hasattr(full, "n_inst"):
        table = shard.global_best_instances(inst_ids if inst_ids is not None else range(prob.n_inst), eng.unsat,
                                            eng.best, full.n_inst)
        best = {"instances": int(full.n_inst), "solved_instances": int((table[:, 0] == 0).sum()),
                "sum_of_best_unsat": int(table[:, 0].clamp(min=0).sum())}
    else:
        b_rank, b_cand, b_unsat, _ = shard.global_best(eng.unsat, eng.best, eng.bits, n=n)
        best = {"unsat": b_unsat, "rank": b_rank, "candidate": b_cand, "of": B * world}

    # evals of the whole job: every rank's literals x candidates (ranks hold equal formulas under
    # the candidate split, shares of the batch under the instance split)
    job_evals = evals_per_step * world
    if world > 1 and inst_ids is not None:
        t = torch.tensor([float(evals_per_step)], dtype=torch.float64, device=dev)
        dist.all_reduce(t)
        job_evals = float(t.item())
    value = job_evals * K / (total_ms / 1000.0)
    # launches per step: the variable pass and its two loss-reduction kernels, the check and its
    # two count-reduction kernels (+ the bit-row compaction for B <= 32, + the forward pass and
    # its two reduction kernels when the loss comes from a separate pass)
    launches_per_step = 6 + (1 if B <= 32 else 0) + (3 if tuning["loss_mode"] == 2 else 0)
    # Roofline of the dominant kernel (the fused variable-major pass inside gs_step). The HBM
    # fraction counts the compulsory bytes of a launch (state streams, the relaxed values read
    # once and written once, the bit rows, the index data once per candidate chunk): the bytes
    # that must cross HBM whatever the gather strategy. The gather model (each literal value
    # read twice per step) counts row reads that L2 serves; it is reported under its own key and,
    # as actual row reads, against the random-row gather rate the probe kernel measures on the
    # same rows.
    peak, peak_kind = measured_peaks()
    lanes = tuning["var_lanes"]
    vec = 16 // s_bytes
    n_chunks = -(-B // (min(lanes, max(4, -(-B // vec))) * vec))
    index_bytes = n_chunks * 4 * (info["n_occ_codes"] + info["n_var_tiles"] * 16)
    compulsory = _compulsory_bytes(n, B, s_bytes) + index_bytes
    gather_model = _gather_model_bytes(nnz, n, B, s_bytes)
    mean_step_s = statistics.mean(step_ms) / 1000.0
    achieved = compulsory / mean_step_s / 1e9
    traffic, traffic_src = recorded_traffic(args.workload, B, dtype)
    row_reads = info["n_occ_codes"] * B * s_bytes          # every occurrence code reads one row slice
    l2 = None
    if rank == 0:
        row_bytes = min(512, -(-B // vec) * 16) if B * s_bytes >= 16 else 16
        row_bytes = 1 << (int(row_bytes) - 1).bit_length()
        probe_gbs, probe_ms = gather_probe(torch, eng.x[eng.cur], row_bytes, int(info["n_occ_codes"]))
        kern_gbs = row_reads / mean_step_s / 1e9
        l2 = {"row_read_bytes": row_reads, "GBps": kern_gbs, "probe_GBps": probe_gbs,
              "frac": kern_gbs / probe_gbs, "row_bytes": row_bytes,
              "probe": "gs_gather_probe: %d random %d-byte row reads over all %d rows at the pass's row stride "
                       "(one candidate chunk's working set), 8 in flight per lane" % (
                           int(info["n_occ_codes"]), row_bytes, n)}
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_source": peak_kind,
                "kernel": "k_var_pass (fused gradient + Adam + relax + round + loss credit), timed as the gs_step call",
                "model": "compulsory bytes per launch: n*B*(24+2s) state and value streams + bit rows + index data "
                         "once per candidate chunk",
                "bytes_per_launch": compulsory,
                "dram_measured": None if traffic is None else {
                    "bytes_per_launch": traffic, "GBps": traffic / mean_step_s / 1e9,
                    "frac": traffic / mean_step_s / 1e9 / peak, "over_compulsory": traffic / compulsory,
                    "source": traffic_src},
                "traffic_note": traffic_src,
                "gather_model": {"bytes_per_launch": gather_model, "GBps": gather_model / mean_step_s / 1e9,
                                 "frac_of_hbm_peak": gather_model / mean_step_s / 1e9 / peak,
                                 "note": "each literal value read once in forward and once in backward; most of "
                                         "these row reads are L2 hits, so this exceeds 1 of HBM"},
                "l2_gather": l2,
                "gs_step_ms": statistics.mean(step_ms), "check_ms": statistics.mean(check_ms)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        evs, secs, steps, cores = cpu_oracle_sample(cnf, 16, 7, args.cpu_seconds)
        cpu = {"value": evs, "unit": "evals/s", "cores": cores, "kind": "oracle",
               "sample": "16 of %d candidates, %d oracle steps (forward, backward, Adam, round+check), %.1f s" % (
                   B, steps, secs)}

    e2e = None
    if not args.no_e2e:
        # End to end through the public API with host buffers: every step copies that step's
        # candidate logits delta from pinned host memory to the device, relaxes them to the
        # step's input values x = sigma(delta) (gs_relax), runs the fused step on them (gradient
        # at x, Adam on the copied delta) and the check, and reads back the per-candidate loss
        # and unsat counts into pinned host memory. The copy of step k + 1's logits runs on a
        # second stream into a second buffer while step k computes (the copy waits only for the
        # step that last used that buffer).
        Ke = max(3, min(K, 20))
        host_delta = torch.from_numpy(synth.init_delta(n, B, seed=77 + rank)).pin_memory()
        host_loss = torch.empty((1, B), dtype=torch.float64).pin_memory()
        host_unsat = torch.empty((1, B), dtype=torch.int32).pin_memory()
        dbuf = [eng.delta, candidates(n, B)]
        copy_stream = torch.cuda.Stream()
        main = torch.cuda.current_stream()
        copied = [torch.cuda.Event() for _ in range(2)]
        used = [torch.cuda.Event() for _ in range(2)]
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record()
        copy_stream.wait_stream(main)
        with torch.cuda.stream(copy_stream):
            dbuf[0].copy_(host_delta[:, :B], non_blocking=True)
            copied[0].record(copy_stream)
        for k in range(Ke):
            cur = k % 2
            if k + 1 < Ke:
                with torch.cuda.stream(copy_stream):
                    if k >= 1:
                        copy_stream.wait_event(used[cur ^ 1])
                    dbuf[cur ^ 1].copy_(host_delta[:, :B], non_blocking=True)
                    copied[cur ^ 1].record(copy_stream)
            main.wait_event(copied[cur])
            eng.delta = dbuf[cur]
            _abi.gs_relax(prob, eng.delta, eng.x[eng.cur])
            eng.step()
            used[cur].record(main)
            host_loss.copy_(eng.loss, non_blocking=True)
            host_unsat.copy_(eng.unsat, non_blocking=True)
        a1.record()
        torch.cuda.synchronize()
        eng.delta = dbuf[0]
        e_ms = a0.elapsed_time(a1)
        e_ms = shard.max_over_ranks(e_ms, device=dev)
        e2e = {"value": evals_per_step * Ke * world / (e_ms / 1000.0), "unit": "evals/s",
               "h2d_bytes_per_step": n * B * 4, "d2h_bytes_per_step": B * 8 + B * 4, "steps": Ke,
               "h2d_GBps": n * B * 4 * Ke / (e_ms / 1000.0) / 1e9,
               "inputs": "each step's logits delta [n, B] float32 copied in, relaxed on the device, stepped; "
                         "loss [B] float64 and unsat [B] int32 copied out",
               "overlap": "copy of step k+1's inputs on a second stream during step k"}

    legs = None
    if rank == 0 and world == 1 and args.legs not in ("", "none"):
        del eng
        prob.close()
        torch.cuda.empty_cache()
        legs = run_legs(torch, args, peak)

    line = {
        "metric": "fwd+bwd clause-literal evals/s", "value": value, "unit": "evals/s", "n_gpus": world, "steps": K,
        "warmup": max(3, args.warmup), "ms_per_step": total_ms / K, "higher_is_better": True,
        "scaling": "strong" if inst_ids is not None else "weak",
        "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": {"workload": desc, "n": n, "m": m, "nnz": nnz, "B": B, "global_batch": B * world,
                   "parallelism": ("dp%d (instances split over ranks by literal count)" % world) if inst_ids is not None
                   else "dp%d (independent candidate batches)" % world,
                   "l2": "inputs larger than L2: x %.0f MB + delta/m/v %.0f MB per step" % (
                       n * B * s_bytes / 1e6, n * B * 12 / 1e6),
                   "steps_per_s": 1000.0 * K / total_ms, "tuning": tuning,
                   "launch": ("cuda_graph: the K steps captured once, replayed once in the timed region"
                              if args.launch == "graph" else "eager: one host call per kernel launch"),
                   "plan": {k: info[k] for k in ("fwd_tile_codes", "var_tile_codes", "own_item_codes")},
                   "tuning_source": tune_rec["source"] if tune_rec else "flags", "best_after_run": best},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": launches_per_step * K,
        "legs": legs,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
