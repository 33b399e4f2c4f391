"""Candidate and instance sharding across ranks (one process per GPU).

Candidates are independent: a candidate's loss, gradient, update, rounding and check involve no
other candidate (Eq. 2 and Eq. 5 are per-candidate sums; the batch objective is their sum). So
the batch is partitioned by candidate: every rank loads the same formula, owns its own B
candidates (global candidate id = rank * B + b) and steps them with no per-step collective.

The one exchange is at the end of a run: the ranks agree on the best candidate (fewest
unsatisfied clauses; ties to the lowest global id, matching the single-GPU check) and the
winning rank broadcasts its rounded assignment (Eq. 4), e.g. for the hand-off to a CPU solver.
A batch of many instances (gs_load_batch) can instead be partitioned by instance: every rank
loads a sub-batch of whole instances, chosen so that the ranks' literal counts (the work of a
step is proportional to nnz * B) are balanced, and steps all B candidates of each; at the end
the ranks exchange one row per instance (fewest unsatisfied clauses and the candidate reaching
it). Everything here is host-side plumbing over ``torch.distributed``; it works with gloo on CPU
tensors and with NCCL on device tensors.
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import torch
import torch.distributed as dist


def rank_seed(base: int, rank: int) -> int:
    """Seed of a rank's candidate initialisation: distinct per rank, fixed per (base, rank)."""
    return 1000 * int(rank) + int(base)


def global_candidate(rank: int, B: int, b: int) -> int:
    return int(rank) * int(B) + int(b)


def max_over_ranks(value: float, device=None, group=None) -> float:
    """Maximum of a per-rank scalar (e.g. elapsed time) over all ranks; identity without a
    process group."""
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def unpack_assignment(bits: torch.Tensor, n: int, b: int) -> torch.Tensor:
    """Rounded assignment of candidate b as uint8 [n] from bit-packed [n, >= ceil(B/64)] int64
    words (bit b % 64 of word b // 64)."""
    w = bits[:n, b // 64]
    return ((w >> (b % 64)) & 1).to(torch.uint8)


def global_best(unsat: torch.Tensor, best: torch.Tensor, bits: torch.Tensor, n: int, inst: int = 0,
                group=None) -> Tuple[int, int, int, torch.Tensor]:
    """Agree on the best candidate of instance ``inst`` over all ranks and fetch its assignment.

    unsat: [n_inst, B] int32 per-candidate unsatisfied-clause counts of this rank; best: [n_inst]
    int32 lowest local candidate with the fewest; bits: this rank's bit-packed rounded
    assignments. Returns (rank, local candidate, unsat count, uint8 [n] assignment), identical on
    every rank. Without a process group the local best is returned.
    """
    b_loc = int(best[inst].item())
    u_loc = int(unsat[inst, b_loc].item())
    assignment = unpack_assignment(bits, n, b_loc)
    if not (dist.is_available() and dist.is_initialized()):
        return 0, b_loc, u_loc, assignment
    world = dist.get_world_size(group)
    mine = torch.tensor([u_loc, b_loc], dtype=torch.int64, device=unsat.device)
    allv = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(allv, mine, group=group)
    pairs = [(int(t[0].item()), r, int(t[1].item())) for r, t in enumerate(allv)]
    u_best, r_best, b_best = min(pairs)   # fewest unsat, then lowest rank (= lowest global id)
    out = assignment if dist.get_rank(group) == r_best else torch.zeros(n, dtype=torch.uint8, device=unsat.device)
    src = dist.get_global_rank(group, r_best) if group is not None else r_best
    dist.broadcast(out, src=src, group=group)
    return r_best, b_best, u_best, out


def partition_instances(nnz: Sequence[int], world: int) -> List[List[int]]:
    """Split instances over ``world`` ranks by literal count: largest instance first, each to the
    rank with the smallest load so far (ties to the lowest rank). Returns each rank's instance
    ids in ascending order. Deterministic; every instance goes to exactly one rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(nnz)), key=lambda i: (-int(nnz[i]), i))
    load = [0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += int(nnz[i])
    return [sorted(p) for p in parts]


def sub_batch(n_vars, n_clauses, clause_ptr, lits, ids: Sequence[int]):
    """The CSR arrays (n_vars, n_clauses, clause_ptr, lits) of the instances ``ids`` of a batch
    (instance-local literals are kept; clause_ptr is rebased), ready for gs_load_batch."""
    import numpy as np

    n_vars = np.asarray(n_vars, dtype=np.int64)
    n_clauses = np.asarray(n_clauses, dtype=np.int64)
    c_off = np.concatenate([[0], np.cumsum(n_clauses)])
    cps, lts = [np.zeros(1, dtype=np.int64)], []
    base = 0
    for i in ids:
        c0, c1 = int(c_off[i]), int(c_off[i + 1])
        a, b = int(clause_ptr[c0]), int(clause_ptr[c1])
        cps.append(np.asarray(clause_ptr[c0 + 1:c1 + 1], dtype=np.int64) - a + base)
        lts.append(np.asarray(lits[a:b], dtype=np.int32))
        base += b - a
    ids = list(ids)
    return (n_vars[ids].copy(), n_clauses[ids].copy(), np.concatenate(cps),
            np.concatenate(lts) if lts else np.zeros(0, dtype=np.int32))


def global_best_instances(inst_ids: Sequence[int], unsat: torch.Tensor, best: torch.Tensor, n_inst: int,
                          cand_offset: int = 0, group=None) -> torch.Tensor:
    """Per-instance best candidate over all ranks of an instance-partitioned batch.

    inst_ids: the global ids of this rank's instances (row i of unsat / best is instance
    inst_ids[i]); unsat: [len(inst_ids), B] int32 counts; best: [len(inst_ids)] int32 lowest local
    candidate with the fewest; cand_offset: global id of this rank's candidate 0 (0 when every
    instance lives on one rank; rank * B when ranks also split the candidates of an instance).
    Returns int64 [n_inst, 3] = (unsat, global candidate, rank) per instance, identical on every
    rank: fewest unsatisfied clauses, ties to the lowest global candidate then the lowest rank;
    (-1, -1, -1) for an instance no rank holds."""
    rows = []
    for i, g in enumerate(inst_ids):
        b = int(best[i].item())
        rows.append((int(g), int(unsat[i, b].item()), int(cand_offset) + b))
    rank = dist.get_rank(group) if (dist.is_available() and dist.is_initialized()) else 0
    mine = torch.tensor([[g, u, c, rank] for g, u, c in rows] or [[-1, 0, 0, 0]], dtype=torch.int64)
    if dist.is_available() and dist.is_initialized():
        world = dist.get_world_size(group)
        dev = unsat.device
        cnt = torch.tensor([mine.shape[0]], dtype=torch.int64, device=dev)
        cnts = [torch.zeros_like(cnt) for _ in range(world)]
        dist.all_gather(cnts, cnt, group=group)
        mx = int(max(int(c.item()) for c in cnts))
        pad = torch.full((mx, 4), -1, dtype=torch.int64)
        pad[:mine.shape[0]] = mine
        pad = pad.to(dev)
        allv = [torch.zeros_like(pad) for _ in range(world)]
        dist.all_gather(allv, pad, group=group)
        table = torch.cat([a.cpu() for a in allv])
    else:
        table = mine
    out = torch.full((int(n_inst), 3), -1, dtype=torch.int64)
    best_key = {}
    for g, u, c, r in table.tolist():
        if g < 0:
            continue
        key = (u, c, r)
        if g not in best_key or key < best_key[g]:
            best_key[g] = key
    for g, (u, c, r) in best_key.items():
        out[g] = torch.tensor([u, c, r])
    return out


def init_from_env(backend: Optional[str] = None) -> Tuple[int, int, int]:
    """(rank, world, local_rank) from the torchrun environment; initialises the default process
    group when WORLD_SIZE > 1 (NCCL if CUDA is available, else gloo)."""
    import os

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and not dist.is_initialized():
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return rank, world, local
