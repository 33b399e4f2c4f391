"""From trained candidates to CNF formulas for CPU solvers (Sec. "GaloisSAT Solving Flow").

SAT side (Sec. "Partial Assignment Extraction for SAT Instances", the pool of Eq. 9): pick one
trained candidate theta_sel, draw N noisy hard samples around it, keep each sample's |S| most
confident variables and add them to the formula as unit clauses, one augmented formula per sample.
UNSAT side (Sec. "Guided Branching for UNSAT Instances", Lemma 1): pick the d least confident
variables of theta_sel and emit the 2^d formulas that fix them to every sign pattern.

The sampling and both selections run on the GPU (``gs_pool_sample``, ``gs_branch_vars``); this
module chooses theta_sel and writes DIMACS text.
"""
from __future__ import annotations

import math
from typing import Iterable, List, Optional, Sequence

import numpy as np

from . import _abi

# Sec. "Experiment Setup": N = 100 samples, the top 0.05 % most confident variables, d = 7.
DEFAULT_N = 100
DEFAULT_FRACTION = 0.0005
DEFAULT_D = 7


def select_candidate(scores, policy: str = "max") -> int:
    """theta_sel: the candidate with the largest loss ("max", the most uncertain batch, used for
    exploration in the SAT flow) or the smallest ("min"); ties to the lowest index. ``scores`` is
    one value per candidate (unsat counts or losses)."""
    s = np.asarray(scores).ravel()
    if s.size == 0:
        raise ValueError("no candidates")
    if policy == "max":
        return int(np.flatnonzero(s == s.max())[0])
    if policy == "min":
        return int(np.flatnonzero(s == s.min())[0])
    raise ValueError("policy must be 'max' or 'min'")


def selection_size(n_vars: int, fraction: float = DEFAULT_FRACTION) -> int:
    """|S| for a fraction of the variables (at least one)."""
    return max(1, int(math.ceil(fraction * n_vars)))


def sample_pool(prob: _abi.Problem, delta, b_sel: int, N: int = DEFAULT_N, S: Optional[int] = None,
                seed: int = 0, n_vars: Optional[int] = None, noise=None):
    """N samples around candidate b_sel of delta and each sample's S most confident variables.

    n_vars: number of original variables (the rows before any chain variables); defaults to all.
    Returns host arrays (samples uint8 [N, n_vars], sel int32 [N, S] of 0-based rows, ascending).
    """
    nv = prob.n_vars if n_vars is None else int(n_vars)
    S = selection_size(nv) if S is None else int(S)
    bits, sel = _abi.gs_pool_sample(prob, delta, b_sel, N, S, seed=seed, n_rows=nv, noise=noise)
    words = bits.cpu().numpy().view(np.uint64)[:nv]
    samples = np.zeros((N, nv), dtype=np.uint8)
    for k in range(N):
        samples[k] = ((words[:, k // 64] >> np.uint64(k % 64)) & np.uint64(1)).astype(np.uint8)
    return samples, sel.cpu().numpy()


def branch_variables(prob: _abi.Problem, delta, b_sel: int, d: int = DEFAULT_D, n_vars: Optional[int] = None):
    """The d least confident variables (0-based rows, ascending) of candidate b_sel."""
    nv = prob.n_vars if n_vars is None else int(n_vars)
    return _abi.gs_branch_vars(prob, delta, b_sel, d, n_rows=nv).cpu().numpy()


def unit_clauses(rows: Iterable[int], values: Sequence[int]) -> List[int]:
    """DIMACS unit literals: x_{v+1} where the value is 1, -x_{v+1} where it is 0."""
    return [(int(v) + 1) if values[int(v)] else -(int(v) + 1) for v in rows]


def cube_units(rows: Sequence[int], alpha: int) -> List[int]:
    """Units of branch alpha (bit r of alpha is the value of rows[r]), Lemma 1."""
    return [(int(v) + 1) if (alpha >> r) & 1 else -(int(v) + 1) for r, v in enumerate(rows)]


def dimacs(n_vars: int, clause_ptr, lits, units: Sequence[int] = (), comment: str = "") -> str:
    """DIMACS CNF text of the formula plus one unit clause per literal in ``units``."""
    cp = np.asarray(clause_ptr, dtype=np.int64)
    lt = np.asarray(lits, dtype=np.int64)
    m = cp.size - 1
    out = []
    if comment:
        out.extend("c " + line for line in comment.splitlines())
    out.append("p cnf %d %d" % (n_vars, m + len(units)))
    for t in range(m):
        out.append(" ".join(str(x) for x in lt[cp[t]:cp[t + 1]]) + " 0")
    for u in units:
        out.append("%d 0" % u)
    return "\n".join(out) + "\n"


def augmented_formulas(n_vars: int, clause_ptr, lits, samples, sel) -> List[str]:
    """phi_aug^(k) = phi AND the unit clauses of sample k's selected variables, k = 1..N."""
    return [dimacs(n_vars, clause_ptr, lits, unit_clauses(sel[k], samples[k]),
                   "candidate-pool sample %d: %d confident variables fixed" % (k, sel.shape[1]))
            for k in range(sel.shape[0])]


def branch_formulas(n_vars: int, clause_ptr, lits, rows: Sequence[int]) -> List[str]:
    """The 2^d cubes of Lemma 1 on the branching rows: phi AND the units of each sign pattern."""
    d = len(rows)
    return [dimacs(n_vars, clause_ptr, lits, cube_units(rows, a), "branch %d of %d" % (a, 2 ** d))
            for a in range(2 ** d)]
