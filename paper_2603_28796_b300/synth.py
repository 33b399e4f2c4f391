"""Seeded synthetic inputs: planted CNF formulas and initial candidate logits.

This module only generates inputs; it holds none of the method's arithmetic. Both the CUDA
library and the FP64 oracle (test infrastructure) consume what it produces. The CNF generators
are the plain C code of ``csrc/synth.c`` (xoshiro256** streams); candidate values come from
numpy's PCG64 generator.

The paper evaluates on SAT Competition 2024 instances, which are not available here; the
generators below stand in for them with the structure the workloads name: planted uniform
random 3-SAT / 4-SAT, mixed-width clauses with power-law variable occurrences, uneven batches
of many instances, and community-structured formulas.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from . import build as _build

_lib = None


def _synth():
    global _lib
    if _lib is None:
        path = _build.build_synth()
        L = ctypes.CDLL(path)
        L.gs_synth_widths.restype = ctypes.c_int64
        L.gs_synth_widths.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_double, ctypes.c_void_p]
        L.gs_synth_lits.restype = ctypes.c_int32
        L.gs_synth_lits.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int32,
                                    ctypes.c_double, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
        _lib = L
    return _lib


@dataclass
class CNF:
    """A formula in CSR form with DIMACS literals, plus the hidden planted assignment."""

    n_vars: int
    clause_ptr: np.ndarray   # int64 [m + 1]
    lits: np.ndarray         # int32 [nnz]
    xstar: Optional[np.ndarray] = None   # uint8 [n_vars], satisfies every clause
    name: str = ""

    @property
    def n_clauses(self) -> int:
        return int(self.clause_ptr.size - 1)

    @property
    def nnz(self) -> int:
        return int(self.clause_ptr[-1])

    def clause(self, t: int) -> np.ndarray:
        return self.lits[self.clause_ptr[t]:self.clause_ptr[t + 1]]

    def to_dimacs(self) -> str:
        out = ["p cnf %d %d" % (self.n_vars, self.n_clauses)]
        for t in range(self.n_clauses):
            out.append(" ".join(str(int(x)) for x in self.clause(t)) + " 0")
        return "\n".join(out) + "\n"


@dataclass
class Batch:
    """Many independent instances; instance i's literals are local (1..n_vars[i])."""

    n_vars: np.ndarray       # int64 [n_inst]
    n_clauses: np.ndarray    # int64 [n_inst]
    clause_ptr: np.ndarray   # int64 [sum m + 1], one CSR over all clauses
    lits: np.ndarray         # int32
    xstar: np.ndarray        # uint8 [sum n]
    name: str = ""

    @property
    def n_inst(self) -> int:
        return int(self.n_vars.size)

    def instance(self, i: int) -> CNF:
        c0, c1 = int(self.n_clauses[:i].sum()), int(self.n_clauses[:i + 1].sum())
        v0 = int(self.n_vars[:i].sum())
        cp = self.clause_ptr[c0:c1 + 1] - self.clause_ptr[c0]
        lt = self.lits[self.clause_ptr[c0]:self.clause_ptr[c1]]
        return CNF(int(self.n_vars[i]), cp.copy(), lt.copy(), self.xstar[v0:v0 + int(self.n_vars[i])].copy())


_WIDTH_FIXED, _WIDTH_GEOMETRIC, _WIDTH_UNIFORM = 0, 1, 2
_VARS_UNIFORM, _VARS_POWERLAW, _VARS_COMMUNITY = 0, 1, 2


def _generate(n, m, seed, width_law, kmin, kmax, q, var_law, alpha=0.0, n_comm=1, p_in=0.0, name="") -> CNF:
    L = _synth()
    cp = np.empty(m + 1, dtype=np.int64)
    nnz = L.gs_synth_widths(seed, m, width_law, kmin, kmax, q, cp.ctypes.data)
    if nnz < 0:
        raise ValueError("bad clause-width parameters")
    lits = np.empty(max(int(nnz), 1), dtype=np.int32)
    xs = np.empty(n, dtype=np.uint8)
    rc = L.gs_synth_lits(seed, n, m, cp.ctypes.data, var_law, alpha, n_comm, p_in, xs.ctypes.data, lits.ctypes.data)
    if rc != 0:
        raise ValueError("CNF generation failed (status %d)" % rc)
    return CNF(n, cp, lits[:int(nnz)], xs, name)


def planted_ksat(n: int, m: int, k: int = 3, seed: int = 0) -> CNF:
    """Planted uniform random k-SAT: k distinct uniform variables per clause, signs uniform over
    the patterns the hidden assignment satisfies."""
    return _generate(n, m, seed, _WIDTH_FIXED, k, k, 0.0, _VARS_UNIFORM, name="planted-%d-SAT n=%d m=%d" % (k, n, m))


def mixed_powerlaw(n: int, m: int, kmin: int = 2, kmax: int = 12, q: float = 0.6, alpha: float = 2.5,
                   seed: int = 0) -> CNF:
    """Mixed widths P(k) proportional to q^(k-kmin) on [kmin, kmax]; variable weights
    (r+1)^(-1/(alpha-1)) over random ranks (occurrence tail exponent alpha); planted."""
    return _generate(n, m, seed, _WIDTH_GEOMETRIC, kmin, kmax, q, _VARS_POWERLAW, alpha=alpha,
                     name="mixed-width power-law n=%d m=%d" % (n, m))


def community(n: int, m: int, n_comm: int, kmin: int = 2, kmax: int = 8, p_in: float = 0.9,
              seed: int = 0) -> CNF:
    """Community-structured planted SAT: n_comm contiguous blocks, clause widths uniform on
    [kmin, kmax], each literal inside the clause's home block with probability p_in."""
    return _generate(n, m, seed, _WIDTH_UNIFORM, kmin, kmax, 0.0, _VARS_COMMUNITY, n_comm=n_comm, p_in=p_in,
                     name="community n=%d m=%d blocks=%d" % (n, m, n_comm))


def uneven_batch(n_inst: int = 512, n_min: int = 1000, n_max: int = 200000, seed: int = 0) -> Batch:
    """Half planted 3-SAT (ratio uniform in [4.0, 4.26]), half planted 4-SAT (ratio 9.5), with
    n uniform in [n_min, n_max], in a seeded shuffled order."""
    rng = np.random.default_rng(seed)
    kinds = np.array([3] * (n_inst // 2) + [4] * (n_inst - n_inst // 2))
    rng.shuffle(kinds)
    parts: List[CNF] = []
    for i, k in enumerate(kinds):
        n = int(rng.integers(n_min, n_max + 1))
        ratio = float(rng.uniform(4.0, 4.26)) if k == 3 else 9.5
        m = int(round(ratio * n))
        parts.append(planted_ksat(n, m, int(k), seed=seed * 100003 + i + 1))
    return concat(parts, name="uneven batch of %d" % n_inst)


def concat(parts: List[CNF], name: str = "") -> Batch:
    nv = np.array([p.n_vars for p in parts], dtype=np.int64)
    nc = np.array([p.n_clauses for p in parts], dtype=np.int64)
    nnz = np.array([p.nnz for p in parts], dtype=np.int64)
    cp = np.empty(int(nc.sum()) + 1, dtype=np.int64)
    cp[0] = 0
    off_c, off_l = 0, 0
    for p in parts:
        cp[off_c + 1:off_c + p.n_clauses + 1] = p.clause_ptr[1:] + off_l
        off_c += p.n_clauses
        off_l += p.nnz
    lits = np.concatenate([p.lits for p in parts]) if parts else np.zeros(0, np.int32)
    xs = np.concatenate([p.xstar if p.xstar is not None else np.zeros(p.n_vars, np.uint8) for p in parts]) \
        if parts else np.zeros(0, np.uint8)
    return Batch(nv, nc, cp, lits.astype(np.int32), xs, name)


# ------------------------------------------------------------------------------------------
# Candidate initialisation: each candidate independently and randomly initialised. x0 is drawn
# uniformly on (0, 1) at float32 resolution ((k + 1/2) / 2^24), and the logit difference is
# delta0 = log(x0 / (1 - x0)) evaluated in float64, rounded to float32.
def init_delta(n: int, B: int, seed: int, ldB: Optional[int] = None, rows: Optional[slice] = None) -> np.ndarray:
    """float32 [n, ldB] (columns >= B are 0)."""
    ldB = B if ldB is None else ldB
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x6a5d]))
    k = rng.integers(0, 1 << 24, size=(n, B), dtype=np.int64)
    x0 = (k.astype(np.float64) + 0.5) * (1.0 / (1 << 24))
    out = np.zeros((n, ldB), dtype=np.float32)
    out[:, :B] = (np.log(x0) - np.log1p(-x0)).astype(np.float32)
    return out


def uniform_values(n: int, B: int, seed: int, ldB: Optional[int] = None, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """float32 [n, ldB] uniform on [lo, hi) (columns >= B are 0): generic relaxed-value inputs."""
    ldB = B if ldB is None else ldB
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x17]))
    out = np.zeros((n, ldB), dtype=np.float32)
    out[:, :B] = rng.uniform(lo, hi, size=(n, B)).astype(np.float32)
    return out


def normal_values(n: int, B: int, seed: int, scale: float = 1.0, ldB: Optional[int] = None) -> np.ndarray:
    """float32 [n, ldB] normal(0, scale) (columns >= B are 0): generic gradient / moment inputs."""
    ldB = B if ldB is None else ldB
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x29]))
    out = np.zeros((n, ldB), dtype=np.float32)
    out[:, :B] = (scale * rng.standard_normal(size=(n, B))).astype(np.float32)
    return out


def padded_ld(B: int, elem_bytes: int = 4) -> int:
    """Row stride (elements) rounding B up to 16-byte rows (and to 8 elements for 16-bit data)."""
    mult = max(16 // elem_bytes, 8)
    return max(mult, ((B + mult - 1) // mult) * mult)


# ------------------------------------------------------------------------------------------
# The benchmark workloads (seeded stand-ins for the paper's benchmark instances).
WORKLOADS = {
    "plain": dict(desc="planted uniform random 3-SAT, n=200, m=852 (ratio 4.26), B=64, FP32, 1000 steps",
                  n=200, m=852, B=64, dtype="f32", steps=1000),
    "differentiation": dict(desc="planted uniform random 3-SAT, n=100000, m=426000, B=1024, FP32",
                            n=100_000, m=426_000, B=1024, dtype="f32"),
    "precision": dict(desc="mixed-width planted k-SAT, k in 2..12 with P(k) ~ 0.6^(k-2), power-law occurrences "
                           "(exponent 2.5), n=2000000, m=8000000, B=256, BF16 storage vs FP32",
                      n=2_000_000, m=8_000_000, B=256, dtype="bf16"),
    "batching": dict(desc="512 uneven planted instances (half 3-SAT ratio U[4.0,4.26], half 4-SAT ratio 9.5), "
                          "n uniform in [1000, 200000], B=64 each", n_inst=512, B=64, dtype="f32"),
    "structured": dict(desc="community-structured planted SAT, n=10000000 in 1000 blocks, m=42000000, k uniform "
                            "2..8, 90% of literals in-block, B=32, BF16 storage", n=10_000_000, m=42_000_000,
                       n_comm=1000, B=32, dtype="bf16"),
}


def workload_cnf(name: str, seed: int = 0, scale: float = 1.0):
    """The CNF (or Batch) of a named workload; ``scale`` < 1 shrinks n and m proportionally."""
    w = WORKLOADS[name]
    if name in ("plain", "differentiation"):
        n = max(8, int(w["n"] * scale))
        m = max(8, int(round(w["m"] * scale)))
        return planted_ksat(n, m, 3, seed)
    if name == "precision":
        return mixed_powerlaw(max(16, int(w["n"] * scale)), max(16, int(w["m"] * scale)), seed=seed)
    if name == "structured":
        n_comm = max(1, int(w["n_comm"] * scale))
        block = 10_000 if scale >= 1.0 else max(16, int(10_000 * scale ** 0.5))
        n = n_comm * block
        m = int(round(4.2 * n))
        return community(n, m, n_comm, seed=seed)
    if name == "batching":
        n_inst = max(2, int(w["n_inst"] * scale))
        return uneven_batch(n_inst, seed=seed, n_max=max(1000, int(200_000 * min(1.0, scale * 4))))
    raise KeyError(name)
