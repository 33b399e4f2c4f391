"""Pure-Python Boolean reference pieces for pinning the oracle (independent of oracle/)."""
from __future__ import annotations

import itertools

import numpy as np


def clauses_of(clause_ptr, lits):
    return [list(map(int, lits[clause_ptr[t]:clause_ptr[t + 1]])) for t in range(len(clause_ptr) - 1)]


def csr_of(clauses):
    cp = np.zeros(len(clauses) + 1, dtype=np.int64)
    for t, c in enumerate(clauses):
        cp[t + 1] = cp[t] + len(c)
    lits = np.array([l for c in clauses for l in c], dtype=np.int32)
    return cp, lits


def literal_true(lit: int, assignment) -> bool:
    v = abs(lit) - 1
    return bool(assignment[v]) if lit > 0 else not bool(assignment[v])


def count_unsat(clauses, assignment) -> int:
    return sum(1 for c in clauses if not any(literal_true(l, assignment) for l in c))


def all_assignments(n: int):
    return [tuple(bits) for bits in itertools.product((0, 1), repeat=n)]


def expected_unsat(clauses, n: int, p) -> float:
    """E_x[#unsat(x)] with x_v ~ Bernoulli(p_v) independent, by enumerating all 2^n points."""
    total = 0.0
    for x in all_assignments(n):
        w = 1.0
        for v in range(n):
            w *= p[v] if x[v] else (1.0 - p[v])
        total += w * count_unsat(clauses, x)
    return total


def boolean_gradient(clauses, n: int, assignment):
    """dL_unsat/dx_v at a Boolean point, from the counting rule: for every occurrence of v whose
    other literals are all false, a negated occurrence contributes +1 and a positive one -1."""
    g = [0] * n
    for c in clauses:
        for i, li in enumerate(c):
            others_false = all(not literal_true(lj, assignment) for j, lj in enumerate(c) if j != i)
            if others_false:
                g[abs(li) - 1] += 1 if li < 0 else -1
    return g


def random_clauses(rng, n: int, m: int, kmin: int, kmax: int, distinct: bool = True):
    out = []
    for _ in range(m):
        k = int(rng.integers(kmin, kmax + 1))
        if distinct:
            vs = rng.choice(n, size=min(k, n), replace=False)
        else:
            vs = rng.integers(0, n, size=k)
        signs = rng.integers(0, 2, size=len(vs))
        out.append([int(v + 1) if s else -int(v + 1) for v, s in zip(vs, signs)])
    return out
