"""GPU parity of the straight-through Gumbel path (Eq. 3 with noise, Eq. 4 in the forward pass)
against the FP64 oracle: the Philox logistic noise, the hard sampling, one training step from
given noise (bit-exact hard assignments and integer gradients, Adam within the derived bound),
and the in-kernel noise path against the explicit one."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2603_28796_b300 import _abi, synth  # noqa: E402
from paper_2603_28796_b300.engine import STEngine, candidates  # noqa: E402
from tests import _brute  # noqa: E402
from tests import _gpu_helpers as H  # noqa: E402

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


def formula(kind, seed=0):
    rng = np.random.default_rng(seed)
    if kind == "3sat":
        return synth.planted_ksat(300, 1200, 3, seed=seed)
    if kind == "mixed":     # widths 1..7, duplicates, tautologies, an empty clause
        cl = _brute.random_clauses(rng, 150, 700, 1, 7, distinct=False) + [[]]
        cp, lits = _brute.csr_of(cl)
        return (150, cp, lits)
    if kind == "hubs":      # variable 1 in every clause: split over many tiles
        cl = [[1 if rng.random() < 0.5 else -1] + [int(x) * (1 if rng.random() < 0.5 else -1)
                                                   for x in rng.choice(np.arange(2, 90), 2, replace=False)]
              for _ in range(1500)]
        cp, lits = _brute.csr_of(cl)
        return (89, cp, lits)
    raise KeyError(kind)


def unpack(f):
    if isinstance(f, tuple):
        return f
    return f.n_vars, f.clause_ptr, f.lits


_probs = {}


def problem(kind):
    if kind not in _probs:
        n, cp, lits = unpack(formula(kind))
        _probs[kind] = (n, cp, lits, _abi.gs_load_cnf(n, cp, lits))
    return _probs[kind]


def noise_bound(k23):
    """|l_kernel - l| for l = log(u / (1 - u)): the correctly rounded quotient (2^-24 relative, so
    2^-24 in l) and the fast log's documented error (2^-21.41 absolute near 1, 3 ulp elsewhere),
    plus the final rounding."""
    u = (k23.astype(np.float64) + 0.5) / 2 ** 23
    l = np.abs(np.log(u) - np.log1p(-u))
    return 2.0 ** -21.41 + 2.0 ** -24 + 4 * 2 * U * l + 1e-12


@pytest.mark.parametrize("B", [1, 37, 64, 200])
def test_noise_matches_oracle_philox(B):
    n, cp, lits, prob = problem("3sat")
    for seed, step in ((1, 1), (2 ** 63 + 5, 7), (12345, 0)):
        dev = candidates(n, B)
        _abi.gs_st_noise(prob, seed, step, dev)
        torch.cuda.synchronize()
        ref, k23 = oracle.logistic_noise(n, B, seed, step)
        err = np.abs(H.host64(dev) - ref)
        assert np.all(err <= noise_bound(k23)), float(err.max())


@pytest.mark.parametrize("B", [1, 64, 130, 1024])
def test_sample_bit_exact_with_given_noise(B):
    n, cp, lits, prob = problem("3sat")
    rng = np.random.default_rng(B)
    d = synth.init_delta(n, B, seed=3)
    l32 = oracle.logistic_noise(n, B, 9, 2)[0].astype(np.float32)
    d[rng.random((n, B)) < 0.05] = 0.0                # exact ties go to state 0
    l32[rng.random((n, B)) < 0.02] = 0.0
    bits = torch.full((n, (B + 63) // 64), -1, dtype=torch.int64, device="cuda")
    _abi.gs_st_sample(prob, H.device_cands(d, B), bits, noise=H.device_cands(l32, B))
    torch.cuda.synchronize()
    ref = (d[:, :B].astype(np.float64) + l32[:, :B].astype(np.float64) > 0).astype(np.uint8)
    assert np.array_equal(H.unpack_bits(bits, n, B), ref)
    assert H.padding_bits_zero(bits, n, B)


def test_sample_generated_noise_agrees_off_ties():
    n, cp, lits, prob = problem("3sat")
    B = 256
    d = synth.init_delta(n, B, seed=4)
    bits = torch.zeros((n, B // 64), dtype=torch.int64, device="cuda")
    _abi.gs_st_sample(prob, H.device_cands(d, B), bits, seed=21, step=5)
    torch.cuda.synchronize()
    lref, k23 = oracle.logistic_noise(n, B, 21, 5)
    z = d.astype(np.float64) + lref
    ref = (z > 0).astype(np.uint8)
    got = H.unpack_bits(bits, n, B)
    tie = np.abs(z) <= noise_bound(k23)
    assert np.array_equal(got[~tie], ref[~tie])
    assert tie.sum() <= 2


def run_step(kind, B, t, seed=0, noise_arrays=True, eps=1e-8):
    n, cp, lits, prob = problem(kind)
    d0 = synth.init_delta(n, B, seed=10 + seed)
    m0 = synth.normal_values(n, B, seed=11 + seed, scale=0.02) if t > 1 else np.zeros((n, B), np.float32)
    v0 = np.abs(synth.normal_values(n, B, seed=12 + seed, scale=0.005)) if t > 1 else np.zeros((n, B), np.float32)
    l0 = oracle.logistic_noise(n, B, 77, t)[0].astype(np.float32)
    l1 = oracle.logistic_noise(n, B, 77, t + 1)[0].astype(np.float32)
    delta, m, v = (H.device_cands(a, B) for a in (d0, m0, v0))
    nw = (B + 63) // 64
    bits_in = torch.zeros((n, nw), dtype=torch.int64, device="cuda")
    bits_out = torch.full((n, nw), -1, dtype=torch.int64, device="cuda")
    _abi.gs_st_sample(prob, delta, bits_in, noise=H.device_cands(l0, B))
    unsat = torch.zeros((1, B), dtype=torch.int32, device="cuda")
    _abi.gs_check_bits(prob, bits_in, B, unsat)
    adam = dict(eps=eps)
    if noise_arrays:
        _abi.gs_st_step(prob, delta, m, v, bits_in, bits_out, t, noise=H.device_cands(l0, B),
                        noise_next=H.device_cands(l1, B), adam=adam)
    else:
        _abi.gs_st_step(prob, delta, m, v, bits_in, bits_out, t, seed=77, adam=adam)
    torch.cuda.synchronize()
    ref = oracle.st_step(n, cp, lits, d0, m0, v0, l0, l1, t, eps=eps)
    return dict(n=n, B=B, d0=d0, m0=m0, v0=v0, l0=l0, l1=l1, ref=ref, bits_in=bits_in, bits_out=bits_out,
                unsat=unsat, delta=delta, m=m, v=v)


@pytest.mark.parametrize("kind", ["3sat", "mixed", "hubs"])
@pytest.mark.parametrize("B", [1, 37, 64, 200, 1024, 1500])
@pytest.mark.parametrize("t", [1, 5])
def test_st_step_matches_oracle(kind, B, t):
    r = run_step(kind, B, t)
    n, ref = r["n"], r["ref"]
    # forward at the hard point: the sampled assignment and its exact loss
    assert np.array_equal(H.unpack_bits(r["bits_in"], n, B), ref["x_hat"])
    assert np.array_equal(r["unsat"].cpu().numpy()[0], ref["unsat"])
    # Adam through the soft chain from an exact integer gradient
    z = r["d0"].astype(np.float64) + r["l0"].astype(np.float64)
    z_err = 2 * U * (np.abs(r["d0"]) + np.abs(r["l0"]))          # float32 sum, then the scaling
    tol = H.adam_tolerances(r["d0"], r["m0"], r["v0"], ref["grad"], 0.0, t, g_rel=0.0, z=z, z_err=z_err)
    out = dict(delta=H.host64(r["delta"]), m=H.host64(r["m"]), v=H.host64(r["v"]))
    H.check_adam(out, ref, tol, "st step %s B=%d t=%d" % (kind, B, t))
    # next hard assignment: exact wherever the decision is not within the update's error of a tie
    got = H.unpack_bits(r["bits_out"], n, B)
    zn = ref["delta"] + r["l1"].astype(np.float64)
    tie = np.abs(zn) <= tol["delta"] + 1e-30
    assert np.array_equal(got[~tie], ref["x_hat_next"][~tie])
    assert H.padding_bits_zero(r["bits_out"], n, B)


def test_generated_noise_equals_explicit_generated_arrays():
    """In-kernel noise == the same step fed the arrays gs_st_noise writes (bitwise)."""
    n, cp, lits, prob = problem("mixed")
    B = 200
    outs = []
    for explicit in (False, True):
        d = H.device_cands(synth.init_delta(n, B, seed=5), B)
        m, v = candidates(n, B), candidates(n, B)
        bi = torch.zeros((n, 4), dtype=torch.int64, device="cuda")
        bo = torch.zeros((n, 4), dtype=torch.int64, device="cuda")
        _abi.gs_st_sample(prob, d, bi, seed=3, step=1)
        if explicit:
            l0, l1 = candidates(n, B), candidates(n, B)
            _abi.gs_st_noise(prob, 3, 1, l0)
            _abi.gs_st_noise(prob, 3, 2, l1)
            _abi.gs_st_step(prob, d, m, v, bi, bo, 1, noise=l0, noise_next=l1)
        else:
            _abi.gs_st_step(prob, d, m, v, bi, bo, 1, seed=3)
        torch.cuda.synchronize()
        outs.append([x.clone() for x in (d, m, v, bo)])
    for a, b in zip(*outs):
        assert torch.equal(a, b)


def test_st_engine_trains_and_counts_exactly():
    """Plain workload, 400 graph-captured straight-through steps: the reported unsat counts are
    the exact Boolean counts of the assignments they belong to, and training reduces them."""
    cnf = synth.workload_cnf("plain", seed=0)
    prob = H.load(cnf)
    B = 64
    eng = STEngine(prob, B, seed=3, noise_seed=11)
    eng.step()
    torch.cuda.synchronize()
    u0 = eng.unsat.cpu().numpy()[0].copy()
    eng.run(398, graph=True)
    bits_before = eng.bits_cur.clone()
    eng.step()
    torch.cuda.synchronize()
    u = eng.unsat.cpu().numpy()[0]
    xh = H.unpack_bits(bits_before, cnf.n_vars, B)
    lits = cnf.lits.astype(np.int64)
    vv = np.abs(lits) - 1
    for b in range(B):
        true = np.where(lits > 0, xh[vv, b] == 1, xh[vv, b] == 0)
        assert int((~np.logical_or.reduceat(true, cnf.clause_ptr[:-1])).sum()) == u[b]
    assert np.median(u) < 0.5 * np.median(u0)


def test_st_step_rejects_aliased_bits():
    n, cp, lits, prob = problem("3sat")
    d = candidates(n, 64)
    b = torch.zeros((n, 1), dtype=torch.int64, device="cuda")
    with pytest.raises(_abi.GSError):
        _abi.gs_st_step(prob, d, candidates(n, 64), candidates(n, 64), b, b, 1)


def test_noise_ring_equals_generated_noise():
    """The two-buffer noise ring (each step stores the next step's draw) gives bitwise the same
    trajectory as drawing every value in the kernel twice."""
    n, cp, lits, prob = problem("mixed")
    B = 100
    engines = [STEngine(prob, B, seed=2, noise_seed=9, noise_ring=r) for r in (True, False)]
    for e in engines:
        for _ in range(6):
            e.step()
    torch.cuda.synchronize()
    a, b = engines
    for x, y in ((a.delta, b.delta), (a.m, b.m), (a.v, b.v), (a.bits_cur, b.bits_cur), (a.unsat, b.unsat)):
        assert torch.equal(x, y)


def test_st_checkpoint_resume_is_bitwise():
    import io
    n, cp, lits, prob = problem("mixed")
    B = 70
    ref = STEngine(prob, B, seed=1, noise_seed=5)
    for _ in range(6):
        ref.step()
    a = STEngine(prob, B, seed=1, noise_seed=5)
    for _ in range(2):
        a.step()
    buf = io.BytesIO()
    torch.save(a.state_dict(), buf)
    buf.seek(0)
    b = STEngine(prob, B, seed=8, noise_seed=77)
    b.load_state_dict(torch.load(buf))
    for _ in range(4):
        b.step()
    torch.cuda.synchronize()
    for x, y in ((ref.delta, b.delta), (ref.m, b.m), (ref.v, b.v), (ref.bits_cur, b.bits_cur),
                 (ref.unsat, b.unsat)):
        assert torch.equal(x, y)


def test_st_step_on_a_batch_of_instances():
    """A batch of uneven instances loaded as one problem: rows are instance-concatenated, each
    instance's literals local to it; the step equals the oracle run on each instance alone."""
    batch = synth.uneven_batch(5, n_min=60, n_max=400, seed=3)
    prob = _abi.gs_load_batch(batch.n_vars, batch.n_clauses, batch.clause_ptr, batch.lits)
    n = int(sum(batch.n_vars))
    B, t = 70, 2
    d0 = synth.init_delta(n, B, seed=4)
    l0 = oracle.logistic_noise(n, B, 8, t)[0].astype(np.float32)
    l1 = oracle.logistic_noise(n, B, 8, t + 1)[0].astype(np.float32)
    delta, m, v = H.device_cands(d0, B), candidates(n, B), candidates(n, B)
    bits_in = torch.zeros((n, 2), dtype=torch.int64, device="cuda")
    bits_out = torch.zeros((n, 2), dtype=torch.int64, device="cuda")
    _abi.gs_st_sample(prob, delta, bits_in, noise=H.device_cands(l0, B))
    unsat = torch.zeros((5, B), dtype=torch.int32, device="cuda")
    _abi.gs_check_bits(prob, bits_in, B, unsat)
    _abi.gs_st_step(prob, delta, m, v, bits_in, bits_out, t, noise=H.device_cands(l0, B),
                    noise_next=H.device_cands(l1, B))
    torch.cuda.synchronize()
    got_d = H.host64(delta)
    got_bits = H.unpack_bits(bits_out, n, B)
    u = unsat.cpu().numpy()
    r0 = 0
    z = np.zeros((n, B))
    for i in range(5):
        inst = batch.instance(i)
        ni = inst.n_vars
        rows = slice(r0, r0 + ni)
        ref = oracle.st_step(ni, inst.clause_ptr, inst.lits, d0[rows], z[rows], z[rows], l0[rows], l1[rows], t)
        assert np.array_equal(u[i], ref["unsat"])
        zi = d0[rows].astype(np.float64) + l0[rows].astype(np.float64)
        zerr = 2 * U * (np.abs(d0[rows]) + np.abs(l0[rows]))
        tol = H.adam_tolerances(d0[rows], z[rows], z[rows], ref["grad"], 0.0, t, g_rel=0.0, z=zi, z_err=zerr)
        assert np.all(np.abs(got_d[rows] - ref["delta"]) <= tol["delta"] + 1e-38)
        tie = np.abs(ref["delta"] + l1[rows].astype(np.float64)) <= tol["delta"] + 1e-30
        assert np.array_equal(got_bits[rows][~tie], ref["x_hat_next"][~tie])
        r0 += ni
