"""Whole-run behaviour of the plain method (planted 3-SAT, n = 200, m = 852, B = 64, 1000 steps)
against an FP64 oracle run from the same initial logits.

The float32 and float64 trajectories of a chaotic optimisation separate after enough steps, so
the whole run is compared in two ways:
- lockstep: every K = 50 steps the GPU's state (logits, moments, relaxed values) is fed into one
  oracle step and the GPU's next step must match it within the single-step bars (loss 1e-5,
  Adam within the propagated bound, rounded bits = [delta' > 0], unsat counts bit-exact); this
  catches drift that a single-step test on fresh inputs cannot;
- statistics: the fraction of identical rounded bits between the two final states, and the two
  distributions of final unsatisfied-clause counts (printed; their medians must agree within a
  few clauses and the solved fractions within a few candidates).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2603_28796_b300 import _abi, synth  # noqa: E402
from paper_2603_28796_b300.engine import Engine  # noqa: E402
from tests import _gpu_helpers as H  # noqa: E402

pytestmark = pytest.mark.gpu

STEPS, K, B, SEED = 1000, 50, 64, 7


def test_plain_workload_lockstep_and_trajectory_statistics():
    cnf = synth.workload_cnf("plain", seed=0)
    n, cp, lits = cnf.n_vars, cnf.clause_ptr, cnf.lits
    prob = H.load(cnf)
    eng = Engine(prob, B, "f32", seed=SEED)
    # the oracle's own trajectory from the same float32 initial logits
    d = synth.init_delta(n, B, seed=SEED)[:, :B].astype(np.float64)
    m, v = np.zeros_like(d), np.zeros_like(d)
    x = oracle.relax(d)
    checked = 0
    for t in range(1, STEPS + 1):
        lock = (t - 1) % K == 0 or t == STEPS
        if lock:
            torch.cuda.synchronize()
            gd, gm, gv, gx = (H.host64(a) for a in (eng.delta, eng.m, eng.v, eng.x_cur))
        eng.step()
        if lock:
            torch.cuda.synchronize()
            ref = oracle.step(n, cp, lits, gd, gm, gv, gx, t)
            H.assert_loss(eng.loss.cpu().numpy()[0], ref["loss"], "step %d loss" % t)
            tol = H.adam_tolerances(gd, gm, gv, ref["grad"], ref["scale"], t)
            d1 = H.host64(eng.delta)
            H.check_adam(dict(delta=d1, m=H.host64(eng.m), v=H.host64(eng.v)),
                         dict(delta=ref["delta"], m=ref["m"], v=ref["v"]), tol, "step %d" % t)
            assert np.array_equal(H.unpack_bits(eng.bits, n, B), (d1 > 0).astype(np.uint8)), "step %d bits" % t
            _, u_ref, b_ref = oracle.round_check(n, cp, lits, d1)
            assert np.array_equal(eng.unsat.cpu().numpy()[0], u_ref), "step %d unsat" % t
            assert int(eng.best.cpu().numpy()[0]) == b_ref
            checked += 1
        o = oracle.step(n, cp, lits, d, m, v, x, t)
        d, m, v, x = o["delta"], o["m"], o["v"], o["x"]
    assert checked == STEPS // K + 1
    torch.cuda.synchronize()
    u_gpu = eng.unsat.cpu().numpy()[0]
    _, u_or, _ = oracle.round_check(n, cp, lits, d)
    same = float(((H.host64(eng.delta) > 0) == (d > 0)).mean())
    stats = {"same_bits": same, "gpu_median": float(np.median(u_gpu)), "oracle_median": float(np.median(u_or)),
             "gpu_solved": int((u_gpu == 0).sum()), "oracle_solved": int((u_or == 0).sum()),
             "gpu_hist": np.bincount(u_gpu).tolist(), "oracle_hist": np.bincount(u_or).tolist()}
    print("plain-workload trajectory statistics:", stats)
    assert abs(stats["gpu_median"] - stats["oracle_median"]) <= 3.0
    assert abs(stats["gpu_solved"] - stats["oracle_solved"]) <= 4
    prob.close()
