"""Properties of the seeded input generators (host only)."""
import numpy as np
import pytest

from paper_2603_28796_b300 import synth


def satisfied_by(cnf, x):
    lits = cnf.lits.astype(np.int64)
    v = np.abs(lits) - 1
    true = np.where(lits > 0, x[v] == 1, x[v] == 0)
    per_clause = np.logical_or.reduceat(true, cnf.clause_ptr[:-1]) if cnf.nnz else np.zeros(0, bool)
    widths = np.diff(cnf.clause_ptr)
    per_clause = np.where(widths > 0, per_clause, False)
    return per_clause


def distinct_vars(cnf):
    for t in range(min(cnf.n_clauses, 2000)):
        c = np.abs(cnf.clause(t))
        if len(np.unique(c)) != len(c):
            return False
    return True


@pytest.mark.parametrize("k", [3, 4])
def test_planted_ksat(k):
    cnf = synth.planted_ksat(500, 2000, k, seed=1)
    assert cnf.n_clauses == 2000 and cnf.nnz == 2000 * k
    assert np.all(np.diff(cnf.clause_ptr) == k)
    assert satisfied_by(cnf, cnf.xstar).all()
    assert distinct_vars(cnf)
    assert np.all((np.abs(cnf.lits) >= 1) & (np.abs(cnf.lits) <= 500))
    # signs uniform over the 2^k - 1 satisfying patterns: true-literal count ~ k 2^(k-1) / (2^k - 1)
    lits = cnf.lits.astype(np.int64)
    v = np.abs(lits) - 1
    true = np.where(lits > 0, cnf.xstar[v] == 1, cnf.xstar[v] == 0)
    expect = k * 2 ** (k - 1) / (2 ** k - 1) / k
    assert abs(true.mean() - expect) < 0.02


def test_determinism():
    a = synth.planted_ksat(300, 900, 3, seed=7)
    b = synth.planted_ksat(300, 900, 3, seed=7)
    c = synth.planted_ksat(300, 900, 3, seed=8)
    assert np.array_equal(a.lits, b.lits) and np.array_equal(a.xstar, b.xstar)
    assert not np.array_equal(a.lits, c.lits)
    d1 = synth.init_delta(10, 6, seed=3, ldB=8)
    d2 = synth.init_delta(10, 6, seed=3, ldB=8)
    assert np.array_equal(d1, d2) and np.all(d1[:, 6:] == 0)


def test_mixed_powerlaw():
    cnf = synth.mixed_powerlaw(20000, 60000, seed=2)
    w = np.diff(cnf.clause_ptr)
    assert w.min() >= 2 and w.max() <= 12
    q = 0.6
    pk = np.array([q ** (k - 2) for k in range(2, 13)])
    pk /= pk.sum()
    assert abs(w.mean() - (pk * np.arange(2, 13)).sum()) < 0.05     # E[k] = 3.46
    assert satisfied_by(cnf, cnf.xstar).all()
    assert distinct_vars(cnf)
    occ = np.bincount(np.abs(cnf.lits) - 1, minlength=cnf.n_vars)
    # heavy tail: the busiest variable has far more occurrences than the mean
    assert occ.max() > 50 * occ.mean()


def test_community():
    n_comm, block = 20, 500
    cnf = synth.community(n_comm * block, 4 * n_comm * block, n_comm, seed=3)
    w = np.diff(cnf.clause_ptr)
    assert w.min() >= 2 and w.max() <= 8 and abs(w.mean() - 5.0) < 0.05
    assert satisfied_by(cnf, cnf.xstar).all()
    assert distinct_vars(cnf)
    # fraction of literals in the clause's majority block ~ 0.9 + 0.1 / n_comm
    same = []
    for t in range(2000):
        blocks = (np.abs(cnf.clause(t)) - 1) // block
        same.append(np.bincount(blocks).max() / len(blocks))
    assert np.mean(same) > 0.85


def test_uneven_batch():
    b = synth.uneven_batch(6, n_min=100, n_max=400, seed=4)
    assert b.n_inst == 6
    widths = []
    for i in range(6):
        inst = b.instance(i)
        assert satisfied_by(inst, inst.xstar).all()
        assert 100 <= inst.n_vars <= 400
        widths.append(int(np.diff(inst.clause_ptr)[0]))
        ratio = inst.n_clauses / inst.n_vars
        assert (4.0 - 0.01 <= ratio <= 4.27) if widths[-1] == 3 else abs(ratio - 9.5) < 0.01
    assert sorted(widths) == [3, 3, 3, 4, 4, 4]


def test_dimacs_text_roundtrip_format():
    cnf = synth.planted_ksat(5, 3, 3, seed=0)
    text = cnf.to_dimacs()
    lines = text.strip().split("\n")
    assert lines[0] == "p cnf 5 3" and all(l.endswith(" 0") for l in lines[1:])
