"""Candidate sharding across ranks (one process per GPU).

Candidates are independent: a candidate's loss, gradient, update, rounding and check involve no
other candidate (Eq. 2 and Eq. 5 are per-candidate sums; the batch objective is their sum). So
the batch is partitioned by candidate: every rank loads the same formula, owns its own B
candidates (global candidate id = rank * B + b) and steps them with no per-step collective.

The one exchange is at the end of a run: the ranks agree on the best candidate (fewest
unsatisfied clauses; ties to the lowest global id, matching the single-GPU check) and the
winning rank broadcasts its rounded assignment (Eq. 4), e.g. for the hand-off to a CPU solver.
Everything here is host-side plumbing over ``torch.distributed``; it works with gloo on CPU
tensors and with NCCL on device tensors.
"""
from __future__ import annotations

from typing import Optional, Tuple

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
