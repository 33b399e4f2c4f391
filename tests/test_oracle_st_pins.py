"""Pins of the oracle's straight-through Gumbel pieces (no GPU): the counter-based generator
against its published known-answer vectors, the noise distribution against the logistic law,
and the straight-through step against torch autograd + torch.optim.Adam on the paper's two-logit
parameterisation."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from tests import _brute as bf

def test_philox_known_answer_vectors():
    """The generator against the known-answer vectors published with its reference
    implementation (tests/golden/philox4x32_10_kat.json)."""
    with open(os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.json")) as f:
        kat = json.load(f)
    for vec in kat["vectors"]:
        ctr = [int(x, 16) for x in vec["counter"]]
        key = [int(x, 16) for x in vec["key"]]
        out = [int(x, 16) for x in vec["out"]]
        assert [int(x) for x in oracle.philox4x32([ctr], [key])[0]] == out


def test_noise_layout_from_philox_words():
    n, B, seed, step = 3, 21, (7 << 32) | 12345, (1 << 33) + 4
    noise, k = oracle.logistic_noise(n, B, seed, step)
    for v in range(n):
        for b in range(B):
            ctr = [b // 4, v, step & 0xffffffff, step >> 32]
            r = oracle.philox4x32([ctr], [[seed & 0xffffffff, seed >> 32]])[0]
            assert k[v, b] == int(r[b % 4]) >> 9
            u = (k[v, b] + 0.5) / 2 ** 23
            assert noise[v, b] == math.log(u / (1.0 - u))


def test_logistic_noise_distribution():
    """l = g1 - g0 of two independent Gumbel(0,1) draws is Logistic(0,1): CDF 1/(1+e^-l),
    mean 0, variance pi^2/3."""
    noise, k = oracle.logistic_noise(512, 512, seed=2026, step=1)
    x = np.sort(noise.ravel())
    N = x.size
    cdf = 1.0 / (1.0 + np.exp(-x))
    ks = max(np.max(np.arange(1, N + 1) / N - cdf), np.max(cdf - np.arange(0, N) / N))
    assert ks < 1.63 / math.sqrt(N)                      # Kolmogorov-Smirnov at the 1 % level
    var = math.pi ** 2 / 3
    assert abs(x.mean()) < 4 * math.sqrt(var / N)
    assert abs(x.var() / var - 1) < 0.03
    assert k.max() < 2 ** 23
    # different steps and rows are different draws
    n2, _ = oracle.logistic_noise(512, 512, seed=2026, step=2)
    assert abs(np.corrcoef(noise.ravel(), n2.ravel())[0, 1]) < 0.01
    n3, _ = oracle.logistic_noise(511, 512, seed=2026, step=1, row0=1)
    assert np.array_equal(n3, noise[1:])


@pytest.mark.parametrize("tau", [1.0, 0.5])
def test_st_step_equals_torch_straight_through_adam(tau):
    """The paper's training step in torch: Theta in R^{B x n x 2}, Gumbel noise on each logit,
    y = softmax((Theta + G)/tau) (Eq. 3), hard one-hot argmax in the forward pass with the soft
    y's gradient (straight-through, Eq. 4), L = -sum_t C_t (Eq. 5), torch.optim.Adam(lr = 0.5).
    The oracle's step on delta = theta_1 - theta_0 with l = g_1 - g_0 and lr 1.0 must agree.

    Adam's eps is 1e-3 on both sides here: where the exact gradient cancels to 0 (a variable
    whose positive and negated occurrences balance at the hard point), torch's softmax backward
    leaves a 1e-17 residue (y_0 + y_1 rounds to 1 +- 1 ulp) that eps = 1e-8 would turn into a
    1e-9 move per step; the identity being checked holds for any eps."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    n, B, steps = 9, 4, 6
    clauses = bf.random_clauses(rng, n, 30, 1, 4, distinct=False)
    cp, lits = bf.csr_of(clauses)
    d0 = rng.normal(scale=1.0, size=(n, B))
    noises = [oracle.logistic_noise(n, B, seed=99, step=t)[0] for t in range(1, steps + 2)]
    g0 = rng.gumbel(size=(steps + 1, n, B))                  # any g_0; g_1 = g_0 + l
    theta = torch.zeros((B, n, 2), dtype=torch.float64)
    theta[..., 1] = torch.from_numpy(d0.T.copy())
    theta.requires_grad_(True)
    eps = 1e-3
    opt = torch.optim.Adam([theta], lr=0.5, eps=eps)
    hard_torch, unsat_torch = [], []
    for t in range(steps):
        opt.zero_grad()
        G = torch.zeros((B, n, 2), dtype=torch.float64)
        G[..., 0] = torch.from_numpy(g0[t].T.copy())
        G[..., 1] = torch.from_numpy((g0[t] + noises[t]).T.copy())
        y_soft = torch.softmax((theta + G) / tau, dim=-1)
        idx = torch.argmax(theta + G, dim=-1)
        y_hard = torch.nn.functional.one_hot(idx, 2).to(torch.float64)
        # straight-through: forward value exactly y_hard, gradient of y_soft. (The common form
        # y_hard - y_soft.detach() + y_soft rounds to within 1e-16 of y_hard; where the exact
        # gradient is 0 that residue, divided by Adam's eps, moves delta by ~1e-9 per step.)
        y = y_hard + (y_soft - y_soft.detach())
        loss = 0.0
        unsat = torch.zeros(B, dtype=torch.float64)
        for c in clauses:
            prod = torch.ones(B, dtype=torch.float64)
            for l in c:
                s = y[:, abs(l) - 1, 1] if l > 0 else y[:, abs(l) - 1, 0]
                prod = prod * (1.0 - s)
            loss = loss - (1.0 - prod)
            unsat = unsat + prod.detach()
        loss.sum().backward()
        opt.step()
        hard_torch.append(idx.numpy().T.copy())
        unsat_torch.append(np.rint(unsat.numpy()).astype(np.int32))
    d_torch = (theta[..., 1] - theta[..., 0]).detach().numpy().T
    d, m, v = d0.copy(), np.zeros((n, B)), np.zeros((n, B))
    for t in range(1, steps + 1):
        r = oracle.st_step(n, cp, lits, d, m, v, noises[t - 1], noises[t], t, lr=1.0, eps=eps, tau=tau)
        assert np.array_equal(r["x_hat"], hard_torch[t - 1])
        assert np.array_equal(r["unsat"], unsat_torch[t - 1])
        d, m, v = r["delta"], r["m"], r["v"]
    assert np.allclose(d, d_torch, rtol=0, atol=1e-10)


def test_st_gradient_is_the_boolean_counting_rule():
    """At the hard point the straight-through gradient dL/dx is the integer counting rule (P7b)."""
    rng = np.random.default_rng(4)
    n, B = 10, 6
    clauses = bf.random_clauses(rng, n, 45, 1, 5)
    cp, lits = bf.csr_of(clauses)
    d = rng.normal(size=(n, B))
    noise, _ = oracle.logistic_noise(n, B, seed=5, step=1)
    r = oracle.st_step(n, cp, lits, d, np.zeros((n, B)), np.zeros((n, B)), noise, noise, 1)
    for b in range(B):
        assert list(r["grad"][:, b].astype(int)) == bf.boolean_gradient(clauses, n, r["x_hat"][:, b])
        assert r["unsat"][b] == bf.count_unsat(clauses, r["x_hat"][:, b])
