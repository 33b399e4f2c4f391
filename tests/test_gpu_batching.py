"""The batched form at the scale of the uneven-batch workload: many CNF instances of very
different size in one problem, stepped by one launch per kernel, the iteration loop captured in
a CUDA graph.

The batch mixes planted 3-SAT (clause/variable ratio uniform in [4.0, 4.26]) and planted 4-SAT
(ratio 9.5) with n from 1,000 to 200,000, B = 64 candidates per instance. Checks:
- four steps replayed from one captured CUDA graph equal four eager steps bitwise (logits,
  moments, relaxed values, per-instance losses, unsat counts, best candidates), for lane groups
  sharing each variable and owning whole variables;
- one fused step, per instance, on sampled candidate columns against the FP64 oracle (candidates
  are independent, so a column sample is exact): the per-instance loss within 1e-5, Adam within
  the propagated bound, the rounded bits equal to [delta' > 0], and the unsat counts bit-exact.
Both run with FP32 and with BF16 storage of the relaxed values.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2603_28796_b300 import _abi, synth  # noqa: E402
from paper_2603_28796_b300.engine import Engine  # noqa: E402
from tests import _gpu_helpers as H  # noqa: E402

pytestmark = pytest.mark.gpu

B = 64
N_VARS = [1000, 200000, 1500, 150000, 2500, 120000, 4000, 90000, 6000, 65000, 9000, 45000, 14000, 30000,
          20000, 180000]


@pytest.fixture(scope="module")
def batch_prob():
    rng = np.random.default_rng(2024)
    parts = []
    for i, n in enumerate(N_VARS):
        k = 3 if i % 2 == 0 else 4
        ratio = float(rng.uniform(4.0, 4.26)) if k == 3 else 9.5
        parts.append(synth.planted_ksat(n, int(round(ratio * n)), k, seed=8100 + i))
    batch = synth.concat(parts, name="uneven batch of %d" % len(parts))
    prob = _abi.gs_load_batch(batch.n_vars, batch.n_clauses, batch.clause_ptr, batch.lits)
    assert prob.n_inst == len(parts)
    yield parts, batch, prob
    prob.close()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("split", [1, 2])
def test_uneven_batch_graph_replay_equals_eager(batch_prob, split, dtype):
    parts, batch, prob = batch_prob
    _abi.gs_set_tuning(prob, var_split=split, loss_mode=1)
    e1, e2 = Engine(prob, B, dtype, seed=81), Engine(prob, B, dtype, seed=81)
    for _ in range(4):
        e1.step()
    g = e2.capture(4)
    g.replay()
    torch.cuda.synchronize()
    for a, b in ((e1.delta, e2.delta), (e1.m, e2.m), (e1.v, e2.v), (e1.x_cur, e2.x_cur), (e1.loss, e2.loss),
                 (e1.unsat, e2.unsat), (e1.best, e2.best), (e1.bits, e2.bits)):
        assert torch.equal(a, b)
    assert e1.loss.shape == (len(parts), B)
    _abi.gs_sync_status(prob)
    _abi.gs_set_tuning(prob)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_uneven_batch_step_matches_oracle_per_instance(batch_prob, dtype):
    """With BF16 storage the oracle runs at the stored (rounded) values, so the bars are the
    FP32-accumulation ones."""
    parts, batch, prob = batch_prob
    eng = Engine(prob, B, dtype, seed=82)
    for _ in range(2):
        eng.step()
    torch.cuda.synchronize()
    cols = np.array([0, 17, 38, 63])
    d0 = H.host64(eng.delta)[:, cols]
    m0 = H.host64(eng.m)[:, cols]
    v0 = H.host64(eng.v)[:, cols]
    x0 = H.host64(eng.x_cur)[:, cols]
    t = eng.t + 1
    eng.step()
    torch.cuda.synchronize()
    d1 = H.host64(eng.delta)
    m1, v1 = H.host64(eng.m)[:, cols], H.host64(eng.v)[:, cols]
    loss = eng.loss.cpu().numpy()
    unsat = eng.unsat.cpu().numpy()
    best = eng.best.cpu().numpy()
    assert np.array_equal(H.unpack_bits(eng.bits, eng.n, B), (d1 > 0).astype(np.uint8))
    off = 0
    for i, p in enumerate(parts):
        rows = slice(off, off + p.n_vars)
        lu, _ = oracle.forward(p.n_vars, p.clause_ptr, p.lits, x0[rows])
        H.assert_loss(loss[i, cols], lu, "instance %d (n=%d) loss" % (i, p.n_vars))
        g_ref, scale = oracle.backward(p.n_vars, p.clause_ptr, p.lits, x0[rows])
        d_ref, m_ref, v_ref, _ = oracle.adam(d0[rows], m0[rows], v0[rows], g_ref, t)
        tol = H.adam_tolerances(d0[rows], m0[rows], v0[rows], g_ref, scale, t)
        H.check_adam(dict(delta=d1[rows][:, cols], m=m1[rows], v=v1[rows]), dict(delta=d_ref, m=m_ref, v=v_ref),
                     tol, "instance %d (n=%d)" % (i, p.n_vars))
        _, u_ref, _ = oracle.round_check(p.n_vars, p.clause_ptr, p.lits, d1[rows][:, cols])
        assert np.array_equal(unsat[i, cols], u_ref), "instance %d unsat counts" % i
        lo = np.flatnonzero(unsat[i] == unsat[i].min())[0]
        assert best[i] == lo
        off += p.n_vars
    _abi.gs_sync_status(prob)
