"""FP64 CPU oracle for the GaloisSAT differentiable solving stage (arXiv 2603.28796).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import this package. The CUDA library never calls it, shares no code with it,
and must fail loudly rather than fall back to it.

Each function converts its inputs to float64 (exact for float32/bfloat16/float16 values) and
calls the plain C implementation in ``oracle.c``; see that file for the equations each step
follows (Eq. 1-5 and the experiment-setup hyper-parameters of the paper).

Arrays of candidate values are var-major, shape ``[n, B]``: row v holds variable v of every
candidate. Parity status: all functions pinned (``tests/test_oracle_pins.py``,
``tests/test_oracle_st_pins.py``, ``tests/test_oracle_pool_pins.py``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (gcc, -O2, IEEE arithmetic, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.run(
            ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
             "-std=c11", _SRC, "-o", tmp, "-lm"],
            check=True,
        )
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        i64, i32, dp = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
        d = ctypes.c_double
        lib.o_threads.restype = ctypes.c_int
        lib.o_relax.argtypes = [i64, i64, dp, d, dp]
        lib.o_forward.argtypes = [i64, i64, dp, dp, i64, dp, dp, dp]
        lib.o_backward.argtypes = [i64, i64, dp, dp, i64, dp, dp, dp]
        lib.o_adam.argtypes = [i64, i64, dp, dp, dp, dp, i64, d, d, d, d, d, dp, dp, dp, dp]
        lib.o_round_check.argtypes = [i64, i64, dp, dp, i64, dp, dp, dp, dp]
        u64 = ctypes.c_uint64
        lib.o_philox4x32.argtypes = [i64, dp, dp, dp]
        lib.o_logistic_noise.argtypes = [i64, i64, u64, i64, i64, dp, dp]
        lib.o_st_adam.argtypes = [i64, i64, dp, dp, dp, dp, dp, i64, d, d, d, d, d, dp, dp, dp]
        for f in (lib.o_relax, lib.o_forward, lib.o_backward, lib.o_adam, lib.o_round_check, lib.o_philox4x32,
                  lib.o_logistic_noise, lib.o_st_adam):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _cnf(clause_ptr, lits):
    cp = np.ascontiguousarray(clause_ptr, dtype=np.int64)
    lt = np.ascontiguousarray(lits, dtype=np.int32)
    if lt.size == 0:
        lt = np.zeros(1, dtype=np.int32)
    return cp, lt


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _check(rc, name):
    if rc != 0:
        raise ValueError("oracle %s failed with status %d" % (name, rc))


def threads() -> int:
    """OpenMP threads the oracle uses."""
    return int(_load().o_threads())


def relax(delta, tau: float = 1.0):
    """x = sigma(delta / tau), Eq. 3 with two states and no noise."""
    d = _f64(delta)
    n, B = d.shape
    x = np.empty_like(d)
    _check(_load().o_relax(n, B, _ptr(d), float(tau), _ptr(x)), "relax")
    return x


def forward(n_vars, clause_ptr, lits, x):
    """Returns (unsat_loss[B], paper_loss[B]): sum_t prod(1 - s_i) and -sum_t C_t (Eq. 2, 5)."""
    cp, lt = _cnf(clause_ptr, lits)
    xx = _f64(x)
    B = xx.shape[1]
    lu = np.empty(B)
    lp = np.empty(B)
    _check(_load().o_forward(int(n_vars), cp.size - 1, _ptr(cp), _ptr(lt), B, _ptr(xx), _ptr(lu), _ptr(lp)),
           "forward")
    return lu, lp


def backward(n_vars, clause_ptr, lits, x):
    """Returns (grad[n, B], scale[n, B]): dL_unsat/dx and the sum of |leave-one-out products|."""
    cp, lt = _cnf(clause_ptr, lits)
    xx = _f64(x)
    B = xx.shape[1]
    g = np.empty((int(n_vars), B))
    s = np.empty((int(n_vars), B))
    _check(_load().o_backward(int(n_vars), cp.size - 1, _ptr(cp), _ptr(lt), B, _ptr(xx), _ptr(g), _ptr(s)),
           "backward")
    return g, s


def adam(delta, m, v, grad_x, step, lr=1.0, beta1=0.9, beta2=0.999, eps=1e-8, tau=1.0):
    """One Adam step on delta from dL/dx; returns (delta', m', v', x' = sigma(delta'/tau))."""
    d, mm, vv, g = _f64(delta), _f64(m), _f64(v), _f64(grad_x)
    n, B = d.shape
    d1, m1, v1, x1 = (np.empty_like(d) for _ in range(4))
    _check(_load().o_adam(n, B, _ptr(d), _ptr(mm), _ptr(vv), _ptr(g), int(step), float(lr), float(beta1),
                          float(beta2), float(eps), float(tau), _ptr(d1), _ptr(m1), _ptr(v1), _ptr(x1)), "adam")
    return d1, m1, v1, x1


def round_check(n_vars, clause_ptr, lits, delta):
    """Returns (x_hat[n, B] uint8, unsat[B] int32, best int): Eq. 4 rounding and exact clause check."""
    cp, lt = _cnf(clause_ptr, lits)
    d = _f64(delta)
    B = d.shape[1]
    xh = np.empty((int(n_vars), B), dtype=np.uint8)
    un = np.empty(B, dtype=np.int32)
    best = np.zeros(1, dtype=np.int32)
    _check(_load().o_round_check(int(n_vars), cp.size - 1, _ptr(cp), _ptr(lt), B, _ptr(d), _ptr(xh), _ptr(un),
                                 _ptr(best)), "round_check")
    return xh, un, int(best[0])


def step(n_vars, clause_ptr, lits, delta, m, v, x, t, lr=1.0, beta1=0.9, beta2=0.999, eps=1e-8, tau=1.0):
    """One training step of the hot path at stored values x: forward loss, gradient, Adam.

    Returns dict(loss, grad, scale, delta, m, v, x).
    """
    lu, _ = forward(n_vars, clause_ptr, lits, x)
    g, s = backward(n_vars, clause_ptr, lits, x)
    d1, m1, v1, x1 = adam(delta, m, v, g, t, lr, beta1, beta2, eps, tau)
    return dict(loss=lu, grad=g, scale=s, delta=d1, m=m1, v=v1, x=x1)


# ---------------------------------------------------------------------------------------------
# Straight-through Gumbel training (Eq. 3 with noise, Eq. 4 in the forward pass); see oracle.c.
def philox4x32(counter, key):
    """Philox4x32-10 blocks: counter [..., 4] uint32, key [..., 2] uint32 -> [..., 4] uint32."""
    c = np.ascontiguousarray(counter, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    if k.shape[0] == 1 and c.shape[0] > 1:
        k = np.ascontiguousarray(np.repeat(k, c.shape[0], axis=0))
    out = np.empty_like(c)
    _check(_load().o_philox4x32(c.shape[0], _ptr(c), _ptr(k), _ptr(out)), "philox4x32")
    return out.reshape(np.shape(counter))


def logistic_noise(n, B, seed, step, row0=0):
    """(l [n, B] float64, k [n, B] uint32): the logistic noise of one step and its 23-bit draws."""
    noise = np.empty((int(n), int(B)))
    k23 = np.empty((int(n), int(B)), dtype=np.uint32)
    _check(_load().o_logistic_noise(int(n), int(B), int(seed) & (2 ** 64 - 1), int(step), int(row0), _ptr(noise),
                                    _ptr(k23)), "logistic_noise")
    return noise, k23


def st_adam(delta, m, v, grad_x, noise, step, lr=1.0, beta1=0.9, beta2=0.999, eps=1e-8, tau=1.0):
    """Adam on delta with the straight-through chain y(1 - y)/tau, y = sigma((delta + noise)/tau)."""
    d, mm, vv, g, ns = _f64(delta), _f64(m), _f64(v), _f64(grad_x), _f64(noise)
    n, B = d.shape
    d1, m1, v1 = (np.empty_like(d) for _ in range(3))
    _check(_load().o_st_adam(n, B, _ptr(d), _ptr(mm), _ptr(vv), _ptr(g), _ptr(ns), int(step), float(lr),
                             float(beta1), float(beta2), float(eps), float(tau), _ptr(d1), _ptr(m1), _ptr(v1)),
           "st_adam")
    return d1, m1, v1


def st_step(n_vars, clause_ptr, lits, delta, m, v, noise, noise_next, t, lr=1.0, beta1=0.9, beta2=0.999,
            eps=1e-8, tau=1.0):
    """One straight-through Gumbel step at logits delta with this step's noise and the next's.

    x_hat = [delta + noise > 0] (Eq. 4 on the noisy logits); loss = number of clauses false
    under x_hat (L_unsat at a Boolean point); grad = dL/dx at x_hat (integers); Adam with the
    chain through y = sigma((delta + noise)/tau); x_hat_next = [delta' + noise_next > 0].
    Returns dict(x_hat, unsat, grad, delta, m, v, x_hat_next, unsat_next).
    """
    d = _f64(delta)
    z = d + _f64(noise)
    x_hat, unsat, _ = round_check(n_vars, clause_ptr, lits, z)
    g, _ = backward(n_vars, clause_ptr, lits, x_hat.astype(np.float64))
    d1, m1, v1 = st_adam(d, m, v, g, noise, t, lr, beta1, beta2, eps, tau)
    x_next, unsat_next, _ = round_check(n_vars, clause_ptr, lits, d1 + _f64(noise_next))
    return dict(x_hat=x_hat, unsat=unsat, grad=g, delta=d1, m=m1, v=v1, x_hat_next=x_next, unsat_next=unsat_next)


# ---------------------------------------------------------------------------------------------
# Candidate pool (Sec. "Partial Assignment Extraction for SAT Instances", Eq. 9) and branching
# variables (Sec. "Guided Branching for UNSAT Instances"), written as plain sorts.
def pool_select(delta_col, noise, S):
    """Samples and selections around one candidate.

    delta_col float32 [n] (the candidate's logits), noise float32 [n, N] (one logistic draw per
    variable and sample). z = delta + l in float32 (one rounding, as the kernels add), sample
    x^(k) = [z > 0] (Eq. 4 on the noisy logits), confidence c = sigma(|z| / tau) = max_j y_j,
    ranked by |z| (sigma is increasing), ties to the lower row; the S highest per sample.
    Returns (x uint8 [N, n], sel int32 [N, S], rows ascending)."""
    d = np.asarray(delta_col, dtype=np.float32).reshape(-1, 1)
    z = (d + np.asarray(noise, dtype=np.float32)).astype(np.float32)
    n, N = z.shape
    x = (z > 0).astype(np.uint8).T
    rows = np.arange(n)
    sel = np.empty((N, int(S)), dtype=np.int32)
    for k in range(N):
        order = np.lexsort((rows, -np.abs(z[:, k]).astype(np.float64)))
        sel[k] = np.sort(order[: int(S)])
    return x, sel


def branch_select(delta_col, d):
    """The d variables of lowest confidence sigma(|delta| / tau), i.e. smallest |delta|, ties to the
    lower row; rows ascending."""
    a = np.abs(np.asarray(delta_col, dtype=np.float32)).astype(np.float64)
    order = np.lexsort((np.arange(a.size), a))
    return np.sort(order[: int(d)]).astype(np.int32)
