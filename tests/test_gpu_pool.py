"""GPU parity of the candidate pool and the branching-variable choice (Sec. "Partial Assignment
Extraction for SAT Instances", Eq. 9; Sec. "Guided Branching for UNSAT Instances") against the
oracle's plain sorts: bit-exact samples and selected rows from given noise, including ties, and
the in-kernel noise against the same noise written out by gs_st_noise."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2603_28796_b300 import _abi, pool, synth  # noqa: E402
from paper_2603_28796_b300.engine import candidates  # noqa: E402
from tests import _gpu_helpers as H  # noqa: E402

pytestmark = pytest.mark.gpu

_cache = {}


def problem(n):
    if n not in _cache:
        cnf = synth.planted_ksat(n, 4 * n, 3, seed=n)
        _cache[n] = (cnf, H.load(cnf))
    return _cache[n]


@pytest.mark.parametrize("n,B,N,S", [(300, 16, 1, 1), (300, 16, 37, 5), (2000, 64, 64, 40), (2000, 8, 130, 2000),
                                     (5000, 32, 100, 3)])
def test_pool_matches_oracle_with_given_noise(n, B, N, S):
    cnf, prob = problem(n)
    rng = np.random.default_rng(n + N)
    d = synth.init_delta(n, B, seed=N)
    b = int(rng.integers(0, B))
    l = oracle.logistic_noise(n, N, 5, 0)[0].astype(np.float32)
    # planted ties: equal |z| in every sample for two rows, and exact zeros
    d[7, b] = d[3, b]
    l[7, :] = l[3, :]
    d[11, b] = 0.0
    l[11, : N // 2] = 0.0
    delta = H.device_cands(d, B)
    noise = H.device_cands(l, N)
    bits, sel = _abi.gs_pool_sample(prob, delta, b, N, S, noise=noise)
    torch.cuda.synchronize()
    x_ref, sel_ref = oracle.pool_select(d[:, b], l, S)
    assert np.array_equal(sel.cpu().numpy(), sel_ref)
    assert np.array_equal(H.unpack_bits(bits, n, N).T, x_ref)
    assert H.padding_bits_zero(bits, n, N)


def test_pool_generated_noise_equals_written_noise():
    cnf, prob = problem(2000)
    n, B, N, S = 2000, 64, 100, 25
    delta = H.device_cands(synth.init_delta(n, B, seed=1), B)
    noise = candidates(n, N)
    _abi.gs_st_noise(prob, 123, 0, noise)
    b1, s1 = _abi.gs_pool_sample(prob, delta, 17, N, S, seed=123)
    b2, s2 = _abi.gs_pool_sample(prob, delta, 17, N, S, noise=noise)
    torch.cuda.synchronize()
    assert torch.equal(b1, b2) and torch.equal(s1, s2)


@pytest.mark.parametrize("d_count", [1, 7, 20])
def test_branch_vars_match_oracle(d_count):
    cnf, prob = problem(5000)
    n, B = 5000, 16
    d = synth.init_delta(n, B, seed=d_count)
    d[100, 3] = -d[40, 3]                         # a tie in |delta|, lower row first
    d[200, 3] = 0.0
    got = _abi.gs_branch_vars(prob, H.device_cands(d, B), 3, d_count).cpu().numpy()
    assert np.array_equal(got, oracle.branch_select(d[:, 3], d_count))


def test_pool_restricted_rows_and_formulas():
    """Only the formula's own rows take part when chain variables follow them; the augmented
    formulas carry the sample's values for the selected rows."""
    cnf, prob = problem(2000)
    n, B, N, S = 2000, 16, 10, 20
    d = synth.init_delta(n, B, seed=9)
    l = oracle.logistic_noise(1500, N, 6, 0)[0].astype(np.float32)
    samples, sel = pool.sample_pool(prob, H.device_cands(d, B), 4, N=N, S=S, n_vars=1500,
                                    noise=H.device_cands(l, N))
    x_ref, sel_ref = oracle.pool_select(d[:1500, 4], l, S)
    assert np.array_equal(sel, sel_ref) and np.array_equal(samples, x_ref)
    forms = pool.augmented_formulas(cnf.n_vars, cnf.clause_ptr, cnf.lits, samples, sel)
    for k in (0, N - 1):
        units = [int(line.split()[0]) for line in forms[k].strip().split("\n")[-S:]]
        assert units == [(v + 1) if samples[k, v] else -(v + 1) for v in sel[k]]


def test_pool_rejects_bad_sizes():
    cnf, prob = problem(300)
    delta = candidates(300, 16)
    with pytest.raises(_abi.GSError):
        _abi.gs_pool_sample(prob, delta, 0, 4, 301)            # S > n_rows
    with pytest.raises(_abi.GSError):
        _abi.gs_pool_sample(prob, delta, 0, 0, 1)              # N < 1
    with pytest.raises(_abi.GSError):
        _abi.gs_branch_vars(prob, delta, 0, 0)


def test_dimacs_writer_round_trip(tmp_path):
    """An augmented formula written by pool.dimacs loads back through gs_load_dimacs with the
    formula's clauses plus one unit clause per selected variable."""
    cnf, prob = problem(300)
    units = [5, -17, 300]
    path = tmp_path / "aug.cnf"
    path.write_text(pool.dimacs(cnf.n_vars, cnf.clause_ptr, cnf.lits, units, comment="round trip"))
    p2 = _abi.gs_load_dimacs(str(path))
    info = p2.info()
    assert info["n_vars"] == cnf.n_vars and info["n_clauses"] == cnf.n_clauses + 3
    assert info["nnz"] == cnf.nnz + 3 and info["n_unit"] == 3
    # the planted assignment with the units' values forced: unsat counts agree with a host count
    x = cnf.xstar.copy()
    x[4], x[16], x[299] = 1, 0, 1
    B = 1
    d = np.where(x[:, None] == 1, 1.0, -1.0).astype(np.float32)
    unsat, _ = _abi.gs_round_check(p2, H.device_cands(d, B))
    torch.cuda.synchronize()
    lits = cnf.lits.astype(np.int64)
    true = np.where(lits > 0, x[np.abs(lits) - 1] == 1, x[np.abs(lits) - 1] == 0)
    want = int((~np.logical_or.reduceat(true, cnf.clause_ptr[:-1])).sum())
    assert int(unsat.cpu().numpy()[0, 0]) == want
