"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

Every input comes from the seeded generators; the oracle sees the same values in float64
(16-bit inputs are generated already rounded to their dtype). Bars: rounded assignments, unsat
counts and best candidates bit-exact; loss within 1e-5 relative; gradient within
1e-5 * max(|g|, A) with A = sum |leave-one-out|; Adam outputs within the bound propagated from
those through float32 arithmetic (tests/_gpu_helpers.adam_tolerances).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2603_28796_b300 import _abi, synth  # noqa: E402
from paper_2603_28796_b300.engine import Engine, candidates  # noqa: E402
from tests import _gpu_helpers as H  # noqa: E402

pytestmark = pytest.mark.gpu


def edge_cnf():
    """Empty, unit, duplicate-literal and tautological clauses, a variable with no occurrence,
    and a hub variable whose occurrence list is split over several tiles."""
    rng = np.random.default_rng(9)
    n = 40
    clauses = [[], [3], [-7], [5, 5, -2], [4, -4, 9], [], [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12]]
    for _ in range(300):                       # hub: variable 20 in 300 clauses (> one tile)
        others = rng.choice([v for v in range(1, n + 1) if v not in (20, 40)], size=2, replace=False)
        s = rng.integers(0, 2, size=3)
        clauses.append([20 if s[0] else -20] + [int(o) if si else -int(o) for o, si in zip(others, s[1:])])
    for _ in range(60):
        k = int(rng.integers(1, 6))
        vs = rng.choice(np.arange(1, 40), size=k, replace=False)
        clauses.append([int(v) if rng.integers(0, 2) else -int(v) for v in vs])
    cp = np.zeros(len(clauses) + 1, dtype=np.int64)
    for t, c in enumerate(clauses):
        cp[t + 1] = cp[t] + len(c)
    lits = np.array([l for c in clauses for l in c], dtype=np.int32)
    return synth.CNF(n, cp, lits, None, "edge cases")   # variable 40 never occurs


CNFS = {
    "3sat": lambda: synth.planted_ksat(1500, 6390, 3, seed=21),
    "mixed": lambda: synth.mixed_powerlaw(3000, 10000, seed=22),      # power-law hubs -> split tiles
    "community": lambda: synth.community(8 * 400, 4 * 8 * 400, 8, seed=23),
    "edge": edge_cnf,
}
_cache = {}


def get(name):
    if name not in _cache:
        cnf = CNFS[name]()
        _cache[name] = (cnf, H.load(cnf))
    return _cache[name]


# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("B", [1, 7, 64, 100, 300])
@pytest.mark.parametrize("name", ["3sat", "mixed", "edge"])
def test_forward_and_backward(name, B, dtype):
    cnf, prob = get(name)
    x = H.device_cands(synth.uniform_values(cnf.n_vars, B, seed=B), B, dtype)
    xh = H.host64(x)
    loss = _abi.gs_forward(prob, x)
    grad = _abi.gs_backward(prob, x)
    torch.cuda.synchronize()
    lu, _ = oracle.forward(cnf.n_vars, cnf.clause_ptr, cnf.lits, xh)
    g_ref, scale = oracle.backward(cnf.n_vars, cnf.clause_ptr, cnf.lits, xh)
    H.assert_loss(loss.cpu().numpy()[0], lu)
    H.assert_grad(H.host64(grad), g_ref, scale)


@pytest.mark.parametrize("gather", [1, 2])
@pytest.mark.parametrize("B", [33, 1024 + 40])
def test_forward_backward_many_chunks(B, gather):
    cnf, prob = get("3sat")
    _abi.gs_set_tuning(prob, var_gather=gather)
    x = H.device_cands(synth.uniform_values(cnf.n_vars, B, seed=3), B, "f32")
    xh = H.host64(x)
    dl = torch.from_numpy(synth.normal_values(1, B, seed=4)[0].astype(np.float64)).cuda().reshape(1, B)
    loss = _abi.gs_forward(prob, x)
    grad = _abi.gs_backward(prob, x, dloss=dl)
    torch.cuda.synchronize()
    lu, _ = oracle.forward(cnf.n_vars, cnf.clause_ptr, cnf.lits, xh)
    g_ref, scale = oracle.backward(cnf.n_vars, cnf.clause_ptr, cnf.lits, xh)
    w = dl.cpu().numpy()[0].astype(np.float32).astype(np.float64)
    H.assert_loss(loss.cpu().numpy()[0], lu)
    H.assert_grad(H.host64(grad), g_ref * w, scale * np.abs(w))
    _abi.gs_set_tuning(prob)


def test_boolean_points_exact():
    # At Boolean x the loss is the unsat count and the gradient an integer (exact at zeros).
    cnf, prob = get("mixed")
    B = 96
    xb = (synth.uniform_values(cnf.n_vars, B, seed=5) > 0.5).astype(np.float32)
    x = H.device_cands(xb, B)
    loss = _abi.gs_forward(prob, x)
    grad = _abi.gs_backward(prob, x)
    torch.cuda.synchronize()
    lu, _ = oracle.forward(cnf.n_vars, cnf.clause_ptr, cnf.lits, xb.astype(np.float64))
    g_ref, _ = oracle.backward(cnf.n_vars, cnf.clause_ptr, cnf.lits, xb.astype(np.float64))
    assert np.array_equal(loss.cpu().numpy()[0], lu)
    assert np.array_equal(H.host64(grad), g_ref)
    unsat, best = _abi.gs_round_check(prob, H.device_cands(2 * xb - 1, B))
    assert np.array_equal(unsat.cpu().numpy()[0], lu.astype(np.int32))


@pytest.mark.parametrize("gather", [1, 2])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("B", [5, 64, 200])
@pytest.mark.parametrize("name", ["3sat", "mixed", "edge", "community"])
def test_fused_step(name, B, dtype, gather):
    """gather 1: register loads, 2: TMA gather4 ring where a chunk spans 32 lanes (B = 200)."""
    if gather == 2 and B != 200:
        pytest.skip("register loads are the only path below 32 lanes per chunk")
    check_fused_step(name, B, dtype, var_gather=gather)


@pytest.mark.parametrize("B", [200, 300])
@pytest.mark.parametrize("name", ["3sat", "mixed", "edge", "community"])
def test_fused_step_f16_wide_chunks(name, B):
    """FP16 storage with 32-lane chunks (the variable's loss credits kept in shared memory; one
    partial chunk at B = 200, a full and a partial one at B = 300)."""
    check_fused_step(name, B, "f16")


@pytest.mark.parametrize("split", [1, 2])
@pytest.mark.parametrize("lanes", [4, 8])
@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("B", [5, 100])
@pytest.mark.parametrize("name", ["3sat", "mixed", "edge", "community"])
def test_fused_step_narrow_chunks(name, B, dtype, lanes, split):
    """Chunks of 4 or 8 lanes (several lane groups per warp, several chunks at B = 100) with the
    groups sharing each variable (split 1) or owning whole variables (split 2); the rounded bits
    of chunks narrower than a 32-bit word go to the right word."""
    check_fused_step(name, B, dtype, var_lanes=lanes, var_split=split)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("name", ["3sat", "mixed", "community"])
def test_backward_owned_variables(name, dtype):
    """Gradient pass (gs_backward with per-candidate loss weights) with variable-owning groups."""
    cnf, prob = get(name)
    B = 40
    _abi.gs_set_tuning(prob, var_lanes=8, var_split=2)
    x = H.device_cands(synth.uniform_values(cnf.n_vars, B, seed=21), B, dtype)
    xh = H.host64(x)
    dl = torch.from_numpy(synth.normal_values(1, B, seed=22)[0].astype(np.float64)).cuda().reshape(1, B)
    grad = _abi.gs_backward(prob, x, dloss=dl)
    torch.cuda.synchronize()
    g_ref, scale = oracle.backward(cnf.n_vars, cnf.clause_ptr, cnf.lits, xh)
    w = dl.cpu().numpy()[0].astype(np.float32).astype(np.float64)
    H.assert_grad(H.host64(grad), g_ref * w, scale * np.abs(w))
    _abi.gs_set_tuning(prob)


def check_fused_step(name, B, dtype, **tuning):
    cnf, prob = get(name)
    _abi.gs_set_tuning(prob, **tuning)
    n = cnf.n_vars
    t = 3
    d0 = synth.init_delta(n, B, seed=11)
    m0 = synth.normal_values(n, B, seed=12, scale=0.05)
    v0 = np.abs(synth.normal_values(n, B, seed=13, scale=0.01))
    xin = H.device_cands(synth.uniform_values(n, B, seed=14), B, dtype)
    delta, m, v = (H.device_cands(a, B) for a in (d0, m0, v0))
    xout = candidates(n, B, H.TORCH_DT[dtype], fill=-1.0)
    bits = torch.zeros((n, (B + 63) // 64), dtype=torch.int64, device="cuda")
    loss = torch.zeros((1, B), dtype=torch.float64, device="cuda")
    _abi.gs_step(prob, delta, m, v, t, x_in=xin, x_out=xout, loss=loss, bits=bits)
    torch.cuda.synchronize()
    xh = H.host64(xin)
    lu, _ = oracle.forward(n, cnf.clause_ptr, cnf.lits, xh)
    g_ref, scale = oracle.backward(n, cnf.clause_ptr, cnf.lits, xh)
    d_ref, m_ref, v_ref, x_ref = oracle.adam(d0[:, :B], m0[:, :B], v0[:, :B], g_ref, t)
    H.assert_loss(loss.cpu().numpy()[0], lu, "fused loss")
    tol = H.adam_tolerances(d0[:, :B], m0[:, :B], v0[:, :B], g_ref, scale, t)
    out = dict(delta=H.host64(delta), m=H.host64(m), v=H.host64(v))
    H.check_adam(out, dict(delta=d_ref, m=m_ref, v=v_ref), tol, "fused %s B=%d %s" % (name, B, dtype))
    # x_out = sigma(delta') rounded to dtype; bits = [delta' > 0] (properties of the outputs)
    dg = out["delta"]
    sig = 1.0 / (1.0 + np.exp(-dg))
    xo = H.host64(xout)
    rel = {"f32": 10 * H.U32, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}[dtype]
    assert np.all(np.abs(xo - sig) <= rel * sig + 1e-38 + (2.0 ** -24 if dtype == "f16" else 0.0))
    assert np.array_equal(H.unpack_bits(bits, n, B), (dg > 0).astype(np.uint8))
    assert H.padding_bits_zero(bits, n, B)
    # where the oracle's delta' is clear of zero by more than the bound, the rounding agrees
    clear = np.abs(d_ref) > tol["delta"]
    assert np.array_equal(((dg > 0) == (d_ref > 0))[clear], np.ones(clear.sum(), bool))
    _abi.gs_set_tuning(prob)


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_step_with_external_gradient(dtype):
    cnf, prob = get("3sat")
    n, B, t = cnf.n_vars, 96, 1
    d0 = synth.init_delta(n, B, seed=31)
    g = synth.normal_values(n, B, seed=32, scale=2.0)
    z = np.zeros((n, B), np.float32)
    delta, m, v, grad = (H.device_cands(a, B) for a in (d0, z, z, g))
    xout = candidates(n, B, H.TORCH_DT[dtype])
    _abi.gs_step(prob, delta, m, v, t, grad=grad, x_out=xout)
    torch.cuda.synchronize()
    d_ref, m_ref, v_ref, _ = oracle.adam(d0, z, z, g, t)
    tol = H.adam_tolerances(d0, z, z, g, None, t, g_rel=0.0)
    H.check_adam(dict(delta=H.host64(delta), m=H.host64(m), v=H.host64(v)), dict(delta=d_ref, m=m_ref, v=v_ref), tol)


@pytest.mark.parametrize("B", [1, 17, 32, 33, 63, 64, 65, 130, 1000])
@pytest.mark.parametrize("name", ["3sat", "mixed", "edge", "community"])
def test_round_check_bit_exact(name, B):
    cnf, prob = get(name)
    n = cnf.n_vars
    d = synth.normal_values(n, B, seed=41 + B)
    d[::7, ::3] = 0.0                        # ties go to state 0
    d[1::11, ::5] = -0.0
    delta = H.device_cands(d, B)
    bits = torch.zeros((n, (B + 63) // 64), dtype=torch.int64, device="cuda")
    unsat, best = _abi.gs_round_check(prob, delta, bits=bits)
    torch.cuda.synchronize()
    xh, u_ref, b_ref = oracle.round_check(n, cnf.clause_ptr, cnf.lits, d.astype(np.float64))
    assert np.array_equal(H.unpack_bits(bits, n, B), xh)
    assert H.padding_bits_zero(bits, n, B)
    assert np.array_equal(unsat.cpu().numpy()[0], u_ref)
    assert int(best.cpu().numpy()[0]) == b_ref
    # the same through the bits-only entry point
    u2, b2 = _abi.gs_check_bits(prob, bits, B)
    assert np.array_equal(u2.cpu().numpy()[0], u_ref) and int(b2[0]) == b_ref


def test_planted_assignment_has_no_unsat_clause():
    cnf, prob = get("community")
    B = 70
    d = np.repeat((2.0 * cnf.xstar.astype(np.float32) - 1.0)[:, None], B, axis=1)
    d[:, 1::2] = -d[:, 1::2]                 # odd candidates: the complement
    unsat, best = _abi.gs_round_check(prob, H.device_cands(d, B))
    u = unsat.cpu().numpy()[0]
    assert np.all(u[0::2] == 0) and int(best[0]) == 0
    _, u_ref, _ = oracle.round_check(cnf.n_vars, cnf.clause_ptr, cnf.lits, d.astype(np.float64))
    assert np.array_equal(u, u_ref)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
def test_relax(dtype):
    cnf, prob = get("3sat")
    n, B = cnf.n_vars, 40
    d = synth.normal_values(n, B, seed=51, scale=6.0)
    delta = H.device_cands(d, B)
    x = candidates(n, B, H.TORCH_DT[dtype])
    _abi.gs_relax(prob, delta, x, tau=1.0)
    torch.cuda.synchronize()
    ref = oracle.relax(d.astype(np.float64))
    rel = {"f32": 10 * H.U32, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}[dtype]
    assert np.all(np.abs(H.host64(x) - ref) <= rel * ref + (2.0 ** -24 if dtype == "f16" else 1e-38))


def test_batch_instances():
    parts = [synth.planted_ksat(300 + 50 * i, int(4.2 * (300 + 50 * i)), 3 + (i % 2), seed=60 + i) for i in range(5)]
    parts.append(edge_cnf())
    batch = synth.concat(parts)
    prob = _abi.gs_load_batch(batch.n_vars, batch.n_clauses, batch.clause_ptr, batch.lits)
    assert prob.n_inst == 6
    n, B = int(batch.n_vars.sum()), 72
    x = H.device_cands(synth.uniform_values(n, B, seed=61), B)
    d = synth.normal_values(n, B, seed=62)
    loss = _abi.gs_forward(prob, x)
    grad = _abi.gs_backward(prob, x)
    unsat, best = _abi.gs_round_check(prob, H.device_cands(d, B))
    torch.cuda.synchronize()
    xh = H.host64(x)
    off = 0
    for i, p in enumerate(parts):
        rows = slice(off, off + p.n_vars)
        lu, _ = oracle.forward(p.n_vars, p.clause_ptr, p.lits, xh[rows])
        g_ref, scale = oracle.backward(p.n_vars, p.clause_ptr, p.lits, xh[rows])
        _, u_ref, b_ref = oracle.round_check(p.n_vars, p.clause_ptr, p.lits, d[rows].astype(np.float64))
        H.assert_loss(loss.cpu().numpy()[i], lu, "instance %d loss" % i)
        H.assert_grad(H.host64(grad)[rows], g_ref, scale, "instance %d grad" % i)
        assert np.array_equal(unsat.cpu().numpy()[i], u_ref)
        assert int(best.cpu().numpy()[i]) == b_ref
        off += p.n_vars


@pytest.mark.parametrize("split", [1, 2])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_batch_instances_fused_step(dtype, split):
    """Fused step on a batch of instances (per-instance credited losses), with lane groups sharing
    each variable (split 1) or owning whole variables (split 2): owned-variable items never span
    two instances and their loss partials are reduced per instance."""
    parts = [synth.planted_ksat(300 + 50 * i, int(4.2 * (300 + 50 * i)), 3 + (i % 2), seed=70 + i) for i in range(4)]
    parts.append(edge_cnf())
    parts.append(synth.mixed_powerlaw(600, 2000, seed=75))
    batch = synth.concat(parts)
    prob = _abi.gs_load_batch(batch.n_vars, batch.n_clauses, batch.clause_ptr, batch.lits)
    _abi.gs_set_tuning(prob, var_lanes=8, var_split=split, loss_mode=1)
    n, B, t = int(batch.n_vars.sum()), 40, 2
    d0 = synth.init_delta(n, B, seed=71)
    m0 = synth.normal_values(n, B, seed=72, scale=0.05)
    v0 = np.abs(synth.normal_values(n, B, seed=73, scale=0.01))
    xin = H.device_cands(synth.uniform_values(n, B, seed=74), B, dtype)
    delta, m, v = (H.device_cands(a, B) for a in (d0, m0, v0))
    xout = candidates(n, B, H.TORCH_DT[dtype])
    loss = torch.zeros((len(parts), B), dtype=torch.float64, device="cuda")
    bits = torch.zeros((n, 1), dtype=torch.int64, device="cuda")
    _abi.gs_step(prob, delta, m, v, t, x_in=xin, x_out=xout, loss=loss, bits=bits)
    torch.cuda.synchronize()
    xh, dg = H.host64(xin), H.host64(delta)
    off = 0
    for i, p in enumerate(parts):
        rows = slice(off, off + p.n_vars)
        lu, _ = oracle.forward(p.n_vars, p.clause_ptr, p.lits, xh[rows])
        H.assert_loss(loss.cpu().numpy()[i], lu, "instance %d loss" % i)
        g_ref, scale = oracle.backward(p.n_vars, p.clause_ptr, p.lits, xh[rows])
        d_ref, m_ref, v_ref, _ = oracle.adam(d0[rows, :B], m0[rows, :B], v0[rows, :B], g_ref, t)
        tol = H.adam_tolerances(d0[rows, :B], m0[rows, :B], v0[rows, :B], g_ref, scale, t)
        out = dict(delta=dg[rows], m=H.host64(m)[rows], v=H.host64(v)[rows])
        H.check_adam(out, dict(delta=d_ref, m=m_ref, v=v_ref), tol, "instance %d" % i)
        off += p.n_vars
    assert np.array_equal(H.unpack_bits(bits, n, B), (dg > 0).astype(np.uint8))
    prob.close()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_autotune_on_batch(dtype):
    """gs_autotune on a batch of many instances: its timed steps write one loss row per instance
    into its own temporaries. It returns valid settings, the problem stays usable, and a step
    with the chosen settings matches the oracle per instance."""
    parts = [synth.planted_ksat(200 + 10 * i, int(4.2 * (200 + 10 * i)), 3 + (i % 2), seed=400 + i)
             for i in range(40)]
    batch = synth.concat(parts)
    prob = _abi.gs_load_batch(batch.n_vars, batch.n_clauses, batch.clause_ptr, batch.lits)
    B = 64
    tuned = _abi.gs_autotune(prob, B, dtype)
    assert tuned["var_lanes"] in (4, 8, 16, 32) and tuned["var_split"] in (1, 2)
    assert tuned["loss_mode"] in (1, 2) and tuned["var_gather"] in (1, 2)
    _abi.gs_sync_status(prob)
    n = int(batch.n_vars.sum())
    eng = Engine(prob, B, dtype, seed=401)
    x0 = H.host64(eng.x_cur)
    eng.step()
    torch.cuda.synchronize()
    loss = eng.loss.cpu().numpy()
    assert loss.shape == (len(parts), B)
    off = 0
    for i, p in enumerate(parts):
        lu, _ = oracle.forward(p.n_vars, p.clause_ptr, p.lits, x0[off:off + p.n_vars])
        H.assert_loss(loss[i], lu, "instance %d loss after autotune" % i)
        off += p.n_vars
    assert off == n
    _abi.gs_sync_status(prob)
    del eng
    prob.close()


def test_deterministic_bitwise():
    cnf, prob = get("mixed")
    B = 128
    outs = []
    for _ in range(2):
        e = Engine(prob, B, "f32", seed=5)
        for _ in range(3):
            e.step()
        torch.cuda.synchronize()
        outs.append((e.delta.cpu().clone(), e.loss.cpu().clone(), e.unsat.cpu().clone()))
    for a, b in zip(*outs):
        assert torch.equal(a, b)


def test_engine_graph_equals_eager():
    cnf, prob = get("3sat")
    B = 64
    e1, e2 = Engine(prob, B, seed=2), Engine(prob, B, seed=2)
    for _ in range(6):
        e1.step()
    e2.run(6, graph=True)
    torch.cuda.synchronize()
    assert torch.equal(e1.delta, e2.delta) and torch.equal(e1.loss, e2.loss) and torch.equal(e1.unsat, e2.unsat)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_engine_graph_equals_eager_owned_variables(dtype):
    """The owned-variable pass and the 32-bit-word check (B = 32) inside a captured CUDA graph
    reproduce the eager steps bitwise (their grids and workspaces are set up by gs_reserve)."""
    cnf, prob = get("community")
    B = 32
    _abi.gs_set_tuning(prob, var_split=2, loss_mode=1)
    e1, e2 = Engine(prob, B, dtype, seed=3), Engine(prob, B, dtype, seed=3)
    for _ in range(5):
        e1.step()
    e2.run(5, graph=True)
    torch.cuda.synchronize()
    assert torch.equal(e1.delta, e2.delta) and torch.equal(e1.loss, e2.loss) and torch.equal(e1.unsat, e2.unsat)
    _abi.gs_set_tuning(prob)


def test_columns_beyond_B_untouched():
    cnf, prob = get("edge")
    n, B = cnf.n_vars, 13
    full = torch.full((n, 16), 7.0, device="cuda")
    delta = full[:, :B]
    delta.copy_(H.device_cands(synth.init_delta(n, B, seed=1), B))
    mfull, vfull = torch.full((n, 16), 7.0, device="cuda"), torch.full((n, 16), 7.0, device="cuda")
    m, v = mfull[:, :B], vfull[:, :B]
    m.zero_()
    v.zero_()
    xin = H.device_cands(synth.uniform_values(n, B, seed=2), B)
    xfull = torch.full((n, 16), 7.0, device="cuda")
    _abi.gs_step(prob, delta, m, v, 1, x_in=xin, x_out=xfull[:, :B])
    g = torch.full((n, 16), 7.0, device="cuda")
    _abi.gs_backward(prob, xin, grad=g[:, :B])
    torch.cuda.synchronize()
    for t in (full, mfull, vfull, xfull, g):
        assert torch.all(t[:, B:] == 7.0)


def test_wait_timeout_is_reported_and_context_survives():
    cnf, prob = get("edge")
    _abi.gs_wait_selftest(prob, limit_us=2000)
    with pytest.raises(_abi.GSError) as ei:
        _abi.gs_sync_status(prob)
    assert ei.value.status == 6
    _abi.gs_sync_status(prob)                 # cleared
    x = H.device_cands(synth.uniform_values(cnf.n_vars, 8, seed=1), 8)
    loss = _abi.gs_forward(prob, x)           # the context is still usable
    torch.cuda.synchronize()
    lu, _ = oracle.forward(cnf.n_vars, cnf.clause_ptr, cnf.lits, H.host64(x))
    H.assert_loss(loss.cpu().numpy()[0], lu)


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")
def test_capture_without_reserve_is_refused():
    cnf = synth.planted_ksat(200, 800, 3, seed=77)
    prob = H.load(cnf)
    x = H.device_cands(synth.uniform_values(200, 48, seed=1), 48)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with pytest.raises(_abi.GSError) as ei:
        with torch.cuda.graph(g, stream=s):
            _abi.gs_forward(prob, x)
    assert ei.value.status == 7


def test_autotune_picks_a_valid_tuning_and_keeps_results():
    cnf, prob = get("3sat")
    B = 200
    t = _abi.gs_autotune(prob, B, "f32")
    assert t["var_lanes"] in (4, 8, 16, 32) and t["fwd_lanes"] in (4, 8, 16, 32) and t["var_gather"] in (1, 2)
    assert t["loss_mode"] in (1, 2) and t["var_split"] in (1, 2)
    assert _abi.gs_get_tuning(prob) == t
    x = H.device_cands(synth.uniform_values(cnf.n_vars, B, seed=9), B)
    loss = _abi.gs_forward(prob, x)
    grad = _abi.gs_backward(prob, x)
    torch.cuda.synchronize()
    lu, _ = oracle.forward(cnf.n_vars, cnf.clause_ptr, cnf.lits, H.host64(x))
    g_ref, scale = oracle.backward(cnf.n_vars, cnf.clause_ptr, cnf.lits, H.host64(x))
    H.assert_loss(loss.cpu().numpy()[0], lu)
    H.assert_grad(H.host64(grad), g_ref, scale)
    _abi.gs_set_tuning(prob)


@pytest.mark.parametrize("name", ["mixed", "edge", "community"])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_loss_modes_agree(name, dtype):
    """The fused step's loss credited in the variable pass (loss_mode 1) or from a separate
    forward pass (loss_mode 2): identical updates and rounded bits, both losses at the oracle's."""
    cnf, prob = get(name)
    n, B, t = cnf.n_vars, 100, 3
    x0 = synth.uniform_values(n, B, seed=31)
    d0 = synth.init_delta(n, B, seed=32)
    outs = []
    for mode in (1, 2):
        _abi.gs_set_tuning(prob, loss_mode=mode)
        xin = H.device_cands(x0, B, dtype)
        delta, m, v = H.device_cands(d0, B), candidates(n, B), candidates(n, B)
        xout = candidates(n, B, H.TORCH_DT[dtype])
        bits = torch.zeros((n, 2), dtype=torch.int64, device="cuda")
        loss = torch.zeros((1, B), dtype=torch.float64, device="cuda")
        _abi.gs_step(prob, delta, m, v, t, x_in=xin, x_out=xout, loss=loss, bits=bits)
        torch.cuda.synchronize()
        outs.append((delta, m, v, xout, bits, loss))
    _abi.gs_set_tuning(prob)
    for a, b in zip(outs[0][:5], outs[1][:5]):
        assert torch.equal(a, b)
    lu, _ = oracle.forward(n, cnf.clause_ptr, cnf.lits, H.host64(H.device_cands(x0, B, dtype)))
    for o in outs:
        H.assert_loss(o[5].cpu().numpy()[0], lu)


def test_checkpoint_resume_is_bitwise():
    """N steps == k steps, state_dict() through torch.save / torch.load, a fresh engine, N - k steps."""
    import io
    cnf, prob = get("mixed")
    B = 96
    ref = Engine(prob, B, "bf16", seed=4)
    for _ in range(7):
        ref.step()
    a = Engine(prob, B, "bf16", seed=4)
    for _ in range(3):
        a.step()
    buf = io.BytesIO()
    torch.save(a.state_dict(), buf)
    buf.seek(0)
    b = Engine(prob, B, "bf16", seed=99)
    b.load_state_dict(torch.load(buf))
    for _ in range(4):
        b.step()
    torch.cuda.synchronize()
    for x, y in ((ref.delta, b.delta), (ref.m, b.m), (ref.v, b.v), (ref.x_cur, b.x_cur), (ref.bits, b.bits),
                 (ref.loss, b.loss), (ref.unsat, b.unsat)):
        assert torch.equal(x, y)


def test_hub_variable_with_100k_occurrences():
    """One variable in every one of 100,000 clauses: its occurrence list is split into hundreds
    of tile parts combined by the last part to finish."""
    rng = np.random.default_rng(12)
    n, m = 5000, 100_000
    others = rng.integers(2, n + 1, size=(m, 2))
    others[:, 1] = np.where(others[:, 1] == others[:, 0], (others[:, 0] % (n - 1)) + 2, others[:, 1])
    signs = np.where(rng.random((m, 3)) < 0.5, 1, -1)
    lits = (np.concatenate([np.ones((m, 1), dtype=np.int64), others], axis=1) * signs).astype(np.int32).ravel()
    cp = np.arange(0, 3 * m + 1, 3, dtype=np.int64)
    cnf = synth.CNF(n, cp, lits)
    prob = H.load(cnf)
    assert prob.info()["n_split"] >= 1
    B = 64
    x = synth.uniform_values(n, B, seed=13)
    g = _abi.gs_backward(prob, H.device_cands(x, B))
    torch.cuda.synchronize()
    g_ref, scale = oracle.backward(n, cp, lits, x.astype(np.float64))
    H.assert_grad(H.host64(g), g_ref, scale)


def test_allocation_failure_is_reported():
    """A workspace request far beyond the device's memory (thousands of tiles x 2^27 candidates,
    terabytes of loss partials) fails cleanly with GS_ERR_OOM at its first allocation, and the
    problem stays usable."""
    cnf = synth.planted_ksat(5000, 40000, 8, seed=3)
    prob = H.load(cnf)
    assert prob.info()["n_var_tiles"] * (1 << 27) * 4 > 2 * 10 ** 12
    try:
        with pytest.raises(_abi.GSError) as ei:
            _abi.gs_reserve(prob, 1 << 27, "f32")
        assert ei.value.status == 3          # GS_ERR_OOM
        B = 64
        x = H.device_cands(synth.uniform_values(cnf.n_vars, B, seed=1), B)
        loss = _abi.gs_forward(prob, x)
        torch.cuda.synchronize()
        lu, _ = oracle.forward(cnf.n_vars, cnf.clause_ptr, cnf.lits, H.host64(x))
        H.assert_loss(loss.cpu().numpy()[0], lu)
    finally:
        prob.close()


@pytest.mark.parametrize("caps", [dict(fwd_tile_codes=32, var_tile_codes=32, own_item_codes=256),
                                  dict(fwd_tile_codes=256, var_tile_codes=192, own_item_codes=2048),
                                  dict(fwd_tile_codes=512, var_tile_codes=384, own_item_codes=65536)])
@pytest.mark.parametrize("name", ["3sat", "mixed", "edge", "community"])
def test_tile_caps(name, caps):
    """Tile sizes chosen at load time (gs_plan_opts): small caps make many tiles and split every
    variable with more than 32 codes; forward, backward, the fused step in both variable-pass
    forms and the check keep their parity with the oracle."""
    cnf = CNFS[name]()
    prob = _abi.gs_load_batch_opts([cnf.n_vars], [cnf.n_clauses], cnf.clause_ptr, cnf.lits, **caps)
    info = prob.info()
    assert (info["fwd_tile_codes"], info["var_tile_codes"], info["own_item_codes"]) == (
        caps["fwd_tile_codes"], caps["var_tile_codes"], caps["own_item_codes"])
    n = cnf.n_vars
    for B, dtype, tuning in ((200, "f32", {}), (40, "bf16", dict(var_lanes=4, var_split=2))):
        _abi.gs_set_tuning(prob, **tuning)
        x = H.device_cands(synth.uniform_values(n, B, seed=41), B, dtype)
        xh = H.host64(x)
        loss = _abi.gs_forward(prob, x)
        grad = _abi.gs_backward(prob, x)
        d0 = synth.init_delta(n, B, seed=42)
        delta = H.device_cands(d0, B)
        m, v = H.device_cands(np.zeros((n, B), np.float32), B), H.device_cands(np.zeros((n, B), np.float32), B)
        xout = candidates(n, B, H.TORCH_DT[dtype])
        lstep = torch.zeros((1, B), dtype=torch.float64, device="cuda")
        bits = torch.zeros((n, (B + 63) // 64), dtype=torch.int64, device="cuda")
        _abi.gs_step(prob, delta, m, v, 1, x_in=x, x_out=xout, loss=lstep, bits=bits)
        unsat, best = _abi.gs_check_bits(prob, bits, B)
        torch.cuda.synchronize()
        lu, _ = oracle.forward(n, cnf.clause_ptr, cnf.lits, xh)
        g_ref, scale = oracle.backward(n, cnf.clause_ptr, cnf.lits, xh)
        H.assert_loss(loss.cpu().numpy()[0], lu, "forward")
        H.assert_loss(lstep.cpu().numpy()[0], lu, "fused loss")
        H.assert_grad(H.host64(grad), g_ref, scale)
        d_ref, m_ref, v_ref, _ = oracle.adam(d0[:, :B], np.zeros((n, B)), np.zeros((n, B)), g_ref, 1)
        tol = H.adam_tolerances(d0[:, :B], np.zeros((n, B)), np.zeros((n, B)), g_ref, scale, 1)
        dg = H.host64(delta)
        H.check_adam(dict(delta=dg, m=H.host64(m), v=H.host64(v)), dict(delta=d_ref, m=m_ref, v=v_ref), tol, name)
        _, u_ref, b_ref = oracle.round_check(n, cnf.clause_ptr, cnf.lits, dg)
        assert np.array_equal(unsat.cpu().numpy()[0], u_ref) and int(best.cpu().numpy()[0]) == b_ref
    _abi.gs_sync_status(prob)
    prob.close()
