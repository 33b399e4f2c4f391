"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test ties one oracle function to something other than itself: brute-force enumeration,
the paper's worked examples (tests/golden/), closed forms, finite differences, and torch's
autograd + torch.optim.Adam on the paper's own two-logit parameterisation.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from tests import _brute as bf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def logit(p):
    p = np.asarray(p, dtype=np.float64)
    return np.log(p) - np.log1p(-p)


# ---------------------------------------------------------------------------------------------
# P1: Boolean corners. At x in {0,1}^n every clause product is the indicator of the clause being
# unsatisfied (Eq. 2 at Boolean points), so L_unsat equals the brute-force count exactly and is
# zero iff x satisfies the formula.
@pytest.mark.parametrize("seed", range(4))
def test_boolean_corners_equal_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = 7
    clauses = bf.random_clauses(rng, n, 18, 1, 4, distinct=bool(seed % 2))
    cp, lits = bf.csr_of(clauses)
    pts = bf.all_assignments(n)
    x = np.array(pts, dtype=np.float64).T  # [n, 2^n]
    lu, lp = oracle.forward(n, cp, lits, x)
    counts = np.array([bf.count_unsat(clauses, a) for a in pts], dtype=np.float64)
    assert np.array_equal(lu, counts)
    assert np.array_equal(lp, counts - len(clauses))          # L_paper = -sum C_t = #unsat - m
    _, unsat, best = oracle.round_check(n, cp, lits, 2.0 * x - 1.0)
    assert np.array_equal(unsat, counts.astype(np.int32))
    assert best == int(np.argmin(counts))
    for j, a in enumerate(pts):
        assert (lu[j] == 0.0) == (bf.count_unsat(clauses, a) == 0)


# P2: multilinear expectation. With distinct variables per clause, the clause product equals
# Pr[clause unsatisfied] under independent x_v ~ Bernoulli(x_v), so L_unsat(x) = E[#unsat].
@pytest.mark.parametrize("seed", range(3))
def test_interior_equals_expected_unsat(seed):
    rng = np.random.default_rng(100 + seed)
    n = 8
    clauses = bf.random_clauses(rng, n, 20, 1, 5, distinct=True)
    cp, lits = bf.csr_of(clauses)
    B = 4
    x = rng.uniform(0.0, 1.0, size=(n, B))
    lu, _ = oracle.forward(n, cp, lits, x)
    for b in range(B):
        ref = bf.expected_unsat(clauses, n, x[:, b])
        assert abs(lu[b] - ref) <= 1e-12 * max(1.0, ref)
        assert lu[b] > 0.0   # strictly positive in the open cube


# P3: the soft-relaxation example of the paper: (x OR y) at 0.5, 0.5 gives C = 0.75.
def test_soft_relaxation_075():
    g = golden("soft_relaxation_075.json")
    cp, lits = bf.csr_of(g["clauses"])
    x = np.array(g["x"], dtype=np.float64).reshape(-1, 1)
    lu, lp = oracle.forward(g["n_vars"], cp, lits, x)
    assert lp[0] == -g["C"]
    assert lu[0] == 1.0 - g["C"]


# P4: the three-term inclusion-exclusion expansion printed in the appendix, and the printed
# expansions of the example's three clauses, at random real points.
def test_three_term_expansion_and_printed_clause_polynomials():
    rng = np.random.default_rng(7)
    for _ in range(50):
        x1, x2, x3, x4, z1 = rng.uniform(-0.5, 1.5, size=5)
        X = np.array([x1, x2, x3, x4, z1]).reshape(-1, 1)
        # a OR b OR c with literal values a, b, c
        for signs in ([1, 1, 1], [1, -1, 1], [-1, -1, -1]):
            clause = [s * (i + 1) for i, s in enumerate(signs)]
            cp, lits = bf.csr_of([clause])
            vals = [X[i, 0] if s > 0 else 1.0 - X[i, 0] for i, s in enumerate(signs)]
            a, b, c = vals
            expansion = a + b + c - a * b - b * c - c * a + a * b * c
            _, lp = oracle.forward(5, cp, lits, X)
            assert abs(-lp[0] - expansion) <= 1e-13
        g = golden("appendix_normalization_example.json")
        cp, lits = bf.csr_of(g["phi_prime"]["clauses"])
        # the appendix's printed expansions of C1, C2 (Eq. 7 reading) and C3
        C1 = x1 + (1 - x2) + z1 - x1 * (1 - x2) - (1 - x2) * z1 - z1 * x1 + x1 * (1 - x2) * z1
        C2 = (1 - z1) + x3 + x4 - (1 - z1) * x3 - x3 * x4 - x4 * (1 - z1) + (1 - z1) * x3 * x4
        C3 = (1 - x1) + x3 + x3 - (1 - x1) * x3 - (1 - x1) * x3 - x3 * x3 + (1 - x1) * x3 * x3
        for t, Ct in enumerate((C1, C2, C3)):
            cpt, lt = bf.csr_of([g["phi_prime"]["clauses"][t]])
            _, lp = oracle.forward(5, cpt, lt, X)
            assert abs(-lp[0] - Ct) <= 1e-12


# P5: the appendix's worked example end to end: y -> x_hat -> C -> L = -2.
@pytest.mark.parametrize("z1", [0.0, 1.0])
@pytest.mark.parametrize("variant", ["clauses", "printed_clause_2"])
def test_appendix_worked_example(z1, variant):
    g = golden("appendix_normalization_example.json")
    clauses = [list(c) for c in g["phi_prime"]["clauses"]]
    if variant == "printed_clause_2":
        clauses[1] = g["phi_prime"]["printed_clause_2"]
    cp, lits = bf.csr_of(clauses)
    y = np.array(g["y_second_entries"] + [0.9 if z1 else 0.1], dtype=np.float64)
    delta = logit(y).reshape(-1, 1)
    x_hat, unsat, _ = oracle.round_check(5, cp, lits, delta)
    assert list(x_hat[:4, 0]) == g["x_hat"]
    lu, lp = oracle.forward(5, cp, lits, x_hat.astype(np.float64))
    C = [1 - int(bf.count_unsat([c], x_hat[:, 0])) for c in clauses]
    assert C == g["C"]
    assert lp[0] == g["loss"]
    assert lu[0] == len(clauses) + g["loss"]
    assert unsat[0] == len(clauses) + g["loss"]
    # the original 4-variable formula under the same x_hat: second clause unsatisfied
    cp0, l0 = bf.csr_of(g["phi"]["clauses"])
    _, u0, _ = oracle.round_check(4, cp0, l0, delta[:4])
    assert u0[0] == 1
    # relaxed value of the duplicated clause (NOT x1 OR x3 OR x3) at y: 1 - 0.7 * 0.8^2
    cp3, l3 = bf.csr_of([clauses[2]])
    _, lp3 = oracle.forward(5, cp3, l3, y.reshape(-1, 1))
    assert abs(-lp3[0] - (1 - 0.7 * 0.8 * 0.8)) <= 1e-15


# P6: the related-work example.
def test_related_work_example():
    g = golden("related_work_example.json")
    cp, lits = bf.csr_of(g["clauses"])
    a = np.array(g["satisfying_assignment"], dtype=np.float64).reshape(-1, 1)
    _, unsat, _ = oracle.round_check(3, cp, lits, 2 * a - 1)
    assert unsat[0] == 0
    pts = bf.all_assignments(3)
    x = np.array(pts, dtype=np.float64).T
    _, unsat_all, _ = oracle.round_check(3, cp, lits, 2 * x - 1)
    assert int((unsat_all == 0).sum()) == 4   # brute force: 4 of the 8 assignments satisfy


# ---------------------------------------------------------------------------------------------
# P7: finite differences. L_unsat is a polynomial of degree <= (multiplicity of v in a clause)
# in each coordinate; with degree <= 2 the central difference is exact for any step.
@pytest.mark.parametrize("distinct", [True, False])
def test_backward_matches_central_differences(distinct):
    rng = np.random.default_rng(11 if distinct else 12)
    n = 9
    clauses = bf.random_clauses(rng, n, 30, 1, 4, distinct=distinct)
    if not distinct:   # keep multiplicity <= 2 per clause so the central difference stays exact
        clauses = [c for c in clauses if max(np.unique(np.abs(c), return_counts=True)[1]) <= 2]
        clauses.append([3, 3, -5])
    cp, lits = bf.csr_of(clauses)
    B = 3
    x = rng.uniform(0.0, 1.0, size=(n, B))
    g, scale = oracle.backward(n, cp, lits, x)
    h = 0.25
    for v in range(n):
        xp, xm = x.copy(), x.copy()
        xp[v] += h
        xm[v] -= h
        lp, _ = oracle.forward(n, cp, lits, xp)
        lm, _ = oracle.forward(n, cp, lits, xm)
        fd = (lp - lm) / (2 * h)
        assert np.all(np.abs(fd - g[v]) <= 1e-12 * np.maximum(1.0, scale[v]))


# P7b: integer gradients at Boolean points (exact at zeros: a division-based leave-one-out
# would produce 0/0 here).
@pytest.mark.parametrize("seed", range(3))
def test_backward_integer_at_boolean_points(seed):
    rng = np.random.default_rng(200 + seed)
    n = 6
    clauses = bf.random_clauses(rng, n, 25, 1, 4, distinct=bool(seed % 2))
    cp, lits = bf.csr_of(clauses)
    pts = bf.all_assignments(n)
    x = np.array(pts, dtype=np.float64).T
    g, _ = oracle.backward(n, cp, lits, x)
    for j, a in enumerate(pts):
        assert list(g[:, j]) == bf.boolean_gradient(clauses, n, a)


def test_empty_and_unit_clauses():
    # empty clause: U = 1 always, no gradient; unit clause: leave-one-out product 1
    clauses = [[], [2], [-1, 2]]
    cp, lits = bf.csr_of(clauses)
    x = np.array([[0.3], [0.6]])
    lu, _ = oracle.forward(2, cp, lits, x)
    assert abs(lu[0] - (1.0 + 0.4 + 0.3 * 0.4)) <= 1e-15
    g, _ = oracle.backward(2, cp, lits, x)
    assert abs(g[0, 0] - (+1.0 * 0.4)) <= 1e-15          # d/dx1 of x1*(1-x2)
    assert abs(g[1, 0] - (-1.0 - 0.3)) <= 1e-15          # d/dx2 of (1-x2) + x1*(1-x2)
    _, unsat, _ = oracle.round_check(2, cp, lits, np.array([[1.0], [1.0]]))
    assert unsat[0] == 1


# ---------------------------------------------------------------------------------------------
def test_relax_is_the_two_state_softmax():
    d = np.array([[-40.0, -3.0, 0.0, 1e-9, 2.5, 40.0]])
    x = oracle.relax(d, tau=1.0)
    for j, dv in enumerate(d[0]):
        e0, e1 = 0.0, dv   # softmax over the two logits (theta_0, theta_1) = (0, delta)
        ref = math.exp(e1 - max(e0, e1)) / (math.exp(e0 - max(e0, e1)) + math.exp(e1 - max(e0, e1)))
        assert abs(x[0, j] - ref) <= 1e-15
    x2 = oracle.relax(d, tau=2.0)
    assert abs(x2[0, 4] - 1.0 / (1.0 + math.exp(-1.25))) <= 1e-15


def test_round_ties_to_state_zero():
    cp, lits = bf.csr_of([[1], [2], [3]])
    d = np.array([[0.0], [-0.0], [1e-30]])
    x_hat, unsat, _ = oracle.round_check(3, cp, lits, d)
    assert list(x_hat[:, 0]) == [0, 0, 1]
    assert unsat[0] == 2


# P8: Adam's first step in closed form: m_hat = g, v_hat = g^2, so
# delta_1 = delta_0 - lr * g / (|g| + eps) with g the logit gradient.
def test_adam_first_step_closed_form():
    rng = np.random.default_rng(3)
    n, B = 5, 4
    d0 = rng.normal(size=(n, B))
    gx = rng.normal(size=(n, B))
    d1, m1, v1, x1 = oracle.adam(d0, np.zeros((n, B)), np.zeros((n, B)), gx, 1, lr=1.0, eps=1e-8, tau=1.0)
    s = 1.0 / (1.0 + np.exp(-d0))
    g = gx * s * (1.0 - s)
    assert np.allclose(d1, d0 - g / (np.abs(g) + 1e-8), rtol=0, atol=1e-14)
    assert np.allclose(m1, 0.1 * g, rtol=1e-14, atol=0)
    assert np.allclose(v1, 0.001 * g * g, rtol=1e-13, atol=0)
    assert np.allclose(x1, 1.0 / (1.0 + np.exp(-d1)), rtol=0, atol=1e-15)


# P8b: the paper's parameterisation, through an independent library. Two logits per variable
# (Theta in R^{B x n x 2}), y = softmax(Theta / tau)[..., 1] (Eq. 3 with g = 0), loss of Eq. 2 +
# Eq. 5 summed over the batch, torch autograd, torch.optim.Adam(lr = 0.5). The oracle runs
# forward -> backward -> adam on delta = theta_1 - theta_0 with lr = 1.0; both must agree.
@pytest.mark.parametrize("tau", [1.0, 0.7])
def test_oracle_step_equals_torch_adam_on_two_logits(tau):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    n, B, steps = 7, 3, 6
    clauses = bf.random_clauses(rng, n, 22, 1, 4, distinct=False)
    cp, lits = bf.csr_of(clauses)
    d0 = rng.normal(scale=1.5, size=(n, B))
    theta = torch.zeros((B, n, 2), dtype=torch.float64)
    theta[..., 1] = torch.from_numpy(d0.T.copy())
    theta.requires_grad_(True)
    opt = torch.optim.Adam([theta], lr=0.5)
    for _ in range(steps):
        opt.zero_grad()
        y = torch.softmax(theta / tau, dim=-1)[..., 1]          # [B, n]
        loss = 0.0
        for c in clauses:
            prod = torch.ones(B, dtype=torch.float64)
            for l in c:
                s = y[:, abs(l) - 1] if l > 0 else 1.0 - y[:, abs(l) - 1]
                prod = prod * (1.0 - s)
            loss = loss - (1.0 - prod)                            # L = -sum_t C_t
        loss.sum().backward()
        opt.step()
    d_torch = (theta[..., 1] - theta[..., 0]).detach().numpy().T
    d, m, v = d0.copy(), np.zeros((n, B)), np.zeros((n, B))
    for t in range(1, steps + 1):
        x = oracle.relax(d, tau)
        g, _ = oracle.backward(n, cp, lits, x)
        d, m, v, _ = oracle.adam(d, m, v, g, t, lr=1.0, tau=tau)
    assert np.allclose(d, d_torch, rtol=0, atol=1e-10)


def test_oracle_rejects_bad_literals():
    cp, lits = bf.csr_of([[1, 5]])
    with pytest.raises(ValueError):
        oracle.forward(3, cp, lits, np.zeros((3, 1)))
