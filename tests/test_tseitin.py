"""The width-3 chain normalisation (Sec. "Clause Normalization for Vectorization", Eq. 6-8) of the
C library, host only: the appendix's worked example, sizes, and satisfiability preserved per
assignment by brute force (for every assignment of the original variables, the fewest
unsatisfied clauses of the normalised formula over its fresh variables equals the original
formula's unsatisfied count; zero iff satisfied, i.e. equisatisfiable)."""
import itertools
import json
import os

import numpy as np
import pytest

from paper_2603_28796_b300 import _abi
from tests import _brute as bf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_appendix_example():
    with open(os.path.join(GOLDEN, "appendix_normalization_example.json")) as f:
        g = json.load(f)
    cp, lits = bf.csr_of(g["phi"]["clauses"])
    n2, cp2, lits2 = _abi.gs_tseitin3(g["phi"]["n_vars"], cp, lits)
    assert n2 == g["phi_prime"]["n_vars"]
    assert bf.clauses_of(cp2, lits2) == g["phi_prime"]["clauses"]


@pytest.mark.parametrize("seed", range(8))
def test_sizes_and_widths(seed):
    rng = np.random.default_rng(seed)
    clauses = bf.random_clauses(rng, 30, 200, 0, 12, distinct=bool(seed % 2))
    cp, lits = bf.csr_of(clauses)
    n2, cp2, lits2 = _abi.gs_tseitin3(30, cp, lits)
    u = np.array([len(c) for c in clauses])
    assert n2 == 30 + int(np.maximum(u - 3, 0).sum())
    assert cp2.size - 1 == int(np.maximum(u - 2, 1).sum())
    w = np.diff(cp2)
    assert set(np.unique(w)) <= {0, 3} and (w == 0).sum() == (u == 0).sum()
    assert np.abs(lits2).max(initial=0) <= n2
    # fresh variables are used in clause order, each by exactly two clauses (once plain, once negated)
    fresh = lits2[np.abs(lits2) > 30]
    if fresh.size:
        vals, counts = np.unique(np.abs(fresh), return_counts=True)
        assert np.array_equal(vals, np.arange(31, n2 + 1)) and np.all(counts == 2)


@pytest.mark.parametrize("seed", range(6))
def test_unsat_count_preserved_over_fresh_variables(seed):
    rng = np.random.default_rng(100 + seed)
    n = 5
    clauses = bf.random_clauses(rng, n, 7, 0, 6, distinct=False)
    cp, lits = bf.csr_of(clauses)
    n2, cp2, lits2 = _abi.gs_tseitin3(n, cp, lits)
    norm = bf.clauses_of(cp2, lits2)
    aux = n2 - n
    assert aux <= 12
    for x in itertools.product((0, 1), repeat=n):
        want = bf.count_unsat(clauses, x)
        best = min(bf.count_unsat(norm, x + z) for z in itertools.product((0, 1), repeat=aux))
        assert best == want


def test_rejects_bad_literals():
    with pytest.raises(_abi.GSError):
        _abi.gs_tseitin3(3, np.array([0, 2]), np.array([1, 7], dtype=np.int32))
