"""Pins of the oracle's candidate-pool and branching selections (no GPU): the appendix's printed
probabilities, and brute force over all subsets on tiny inputs."""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2603_28796_b300 import pool


def golden(name):
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        return json.load(f)


def logit(p):
    return math.log(p / (1.0 - p))


def test_appendix_probabilities_rank_confidence():
    """Appendix example: y = P(x = 1) = [0.7, 0.3, 0.2, 0.9] gives confidences max(y, 1 - y) =
    [0.7, 0.7, 0.8, 0.9]: the two most confident are x4, x3; the two least are x1, x2 (tied at
    0.7, the lower rows first); the hard assignment is the printed x_hat = [1, 0, 0, 1]."""
    g = golden("appendix_normalization_example.json")
    d = np.array([logit(p) for p in g["y_second_entries"]], dtype=np.float32)
    x, sel = oracle.pool_select(d, np.zeros((4, 1), dtype=np.float32), 2)
    assert list(x[0]) == g["x_hat"]
    assert list(sel[0]) == [2, 3]
    assert list(oracle.branch_select(d, 2)) == [0, 1]
    assert list(oracle.branch_select(d, 3)) == [0, 1, 2]


@pytest.mark.parametrize("seed", range(5))
def test_selection_maximises_total_confidence(seed):
    """The top-S set is the subset of size S with the largest total confidence sum of
    sigma(|z|), and among equal totals the lexicographically smallest rows (brute force)."""
    rng = np.random.default_rng(seed)
    n, N, S = 7, 3, 3
    d = rng.normal(size=n).astype(np.float32)
    l = rng.logistic(size=(n, N)).astype(np.float32)
    l[2, :] = l[5, :] = 0.0
    d[5] = d[2]                        # a tie between rows 2 and 5 in every sample
    x, sel = oracle.pool_select(d, l, S)
    z = (d[:, None] + l).astype(np.float32).astype(np.float64)
    conf = 1.0 / (1.0 + np.exp(-np.abs(z)))
    for k in range(N):
        best = max(itertools.combinations(range(n), S),
                   key=lambda c: (round(sum(conf[list(c), k]), 12), [-i for i in c]))
        assert list(sel[k]) == list(best)
        assert np.array_equal(x[k], (z[:, k] > 0).astype(np.uint8))
    b = oracle.branch_select(d, 2)
    best = min(itertools.combinations(range(n), 2), key=lambda c: (sum(np.abs(d[list(c)])), c))
    assert list(b) == list(best)


def test_select_candidate_policies():
    assert pool.select_candidate([3, 9, 1, 9]) == 1
    assert pool.select_candidate([3, 9, 1, 1], policy="min") == 2
    assert pool.selection_size(100_000) == 50 and pool.selection_size(10) == 1


def test_dimacs_writers():
    cp = np.array([0, 2, 5])
    lits = np.array([1, -2, 2, 3, -1])
    txt = pool.dimacs(3, cp, lits, [-3, 1], comment="x")
    lines = txt.strip().split("\n")
    assert lines[0] == "c x" and lines[1] == "p cnf 3 4"
    assert lines[2:] == ["1 -2 0", "2 3 -1 0", "-3 0", "1 0"]
    forms = pool.branch_formulas(3, cp, lits, [0, 2])
    assert len(forms) == 4
    units = [f.strip().split("\n")[-2:] for f in forms]
    assert units == [["-1 0", "-3 0"], ["1 0", "-3 0"], ["-1 0", "3 0"], ["1 0", "3 0"]]
    aug = pool.augmented_formulas(3, cp, lits, np.array([[1, 0, 1], [0, 0, 0]], dtype=np.uint8),
                                  np.array([[0, 1], [1, 2]]))
    assert aug[0].strip().split("\n")[-2:] == ["1 0", "-2 0"]
    assert aug[1].strip().split("\n")[-2:] == ["-2 0", "-3 0"]
