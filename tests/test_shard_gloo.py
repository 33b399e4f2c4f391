"""Candidate sharding over ranks: world_size-2 gloo process groups on CPU (no GPU).

Each rank owns its own candidates; the only cross-rank operations are the max-over-ranks
timing reduction and the final agreement on the best candidate with the broadcast of its
rounded assignment."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2603_28796_b300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _pack(bits01):
    """[n, B] 0/1 -> [n, ceil(B/64)] int64 words, bit b % 64 of word b // 64."""
    n, B = bits01.shape
    words = np.zeros((n, (B + 63) // 64), dtype=np.uint64)
    for b in range(B):
        words[:, b // 64] |= bits01[:, b].astype(np.uint64) << np.uint64(b % 64)
    return torch.from_numpy(words.view(np.int64))


def _case(rank, n, B, seed):
    rng = np.random.default_rng(seed + rank)
    x = rng.integers(0, 2, size=(n, B))
    unsat = rng.integers(3, 50, size=(2, B)).astype(np.int32)
    return x, unsat


def _worker(rank, world, port, n, B, mins, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    r, w, _ = shard.init_from_env("gloo")
    assert (r, w) == (rank, world)
    x, unsat = _case(rank, n, B, 5)
    # plant this rank's minimum (instance 1) at a known candidate; several at the minimum
    u_min, where = mins[rank]
    for b in where:
        unsat[1, b] = u_min
    best = torch.from_numpy(np.argmin(unsat, axis=1).astype(np.int32))
    res = shard.global_best(torch.from_numpy(unsat), best, _pack(x), n, inst=1)
    t = shard.max_over_ranks(10.0 + rank)
    torch.save({"res": (res[0], res[1], res[2], res[3].numpy()), "t": t}, os.path.join(out_dir, "r%d.pt" % rank))
    torch.distributed.destroy_process_group()


@pytest.mark.parametrize("mins", [
    [(1, [7, 20]), (0, [3])],      # rank 1 holds the unique minimum
    [(2, [9, 4]), (2, [0])],       # tie across ranks: lowest rank wins, lowest local index there
])
def test_global_best_world2(tmp_path, mins):
    n, B = 97, 130
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n, B, mins, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    outs = [torch.load(os.path.join(tmp_path, "r%d.pt" % r), weights_only=False) for r in range(2)]
    # expected: fewest unsat over both ranks, ties to the lowest global candidate id
    cands = []
    for r in range(2):
        x, unsat = _case(r, n, B, 5)
        for b in mins[r][1]:
            unsat[1, b] = mins[r][0]
        for b in range(B):
            cands.append((int(unsat[1, b]), shard.global_candidate(r, B, b), r, b, x[:, b]))
    u, _, r_exp, b_exp, a_exp = min(cands, key=lambda c: (c[0], c[1]))
    for o in outs:
        r, b, uu, a = o["res"]
        assert (r, b, uu) == (r_exp, b_exp, u)
        assert np.array_equal(a, a_exp.astype(np.uint8))
        assert o["t"] == 11.0      # max over ranks of 10 + rank


def test_single_process_fallbacks():
    x = np.random.default_rng(0).integers(0, 2, size=(10, 70))
    unsat = torch.tensor([[5] * 70], dtype=torch.int32)
    unsat[0, 66] = 1
    r, b, u, a = shard.global_best(unsat, torch.tensor([66], dtype=torch.int32), _pack(x), 10)
    assert (r, b, u) == (0, 66, 1) and np.array_equal(a.numpy(), x[:, 66].astype(np.uint8))
    assert shard.max_over_ranks(3.5) == 3.5
    assert len({shard.rank_seed(1, r) for r in range(8)}) == 8


# ---------------------------------------------------------------------------------------------
# Instance sharding of a batch of many instances: greedy split by literal count, sub-batch
# extraction, and the per-instance best exchange.
def test_partition_instances_covers_and_balances():
    rng = np.random.default_rng(3)
    nnz = rng.integers(3_000, 2_000_000, size=512)
    for world in (1, 2, 3, 8):
        parts = shard.partition_instances(nnz, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(nnz.size))
        assert all(p == sorted(p) for p in parts)
        loads = [int(nnz[p].sum()) for p in parts]
        # largest-first greedy: the heaviest rank exceeds the lightest by at most one instance
        assert max(loads) - min(loads) <= int(nnz.max())
    assert shard.partition_instances([5, 5, 5, 5], 2) == [[0, 2], [1, 3]]
    with pytest.raises(ValueError):
        shard.partition_instances([1], 0)


def test_sub_batch_equals_selected_instances():
    from paper_2603_28796_b300 import synth

    parts = [synth.planted_ksat(50 + 10 * i, 200 + 40 * i, 3 + i % 2, seed=i) for i in range(5)]
    batch = synth.concat(parts)
    ids = [1, 3, 4]
    nv, nc, cp, lits = shard.sub_batch(batch.n_vars, batch.n_clauses, batch.clause_ptr, batch.lits, ids)
    ref = synth.concat([parts[i] for i in ids])
    assert np.array_equal(nv, ref.n_vars) and np.array_equal(nc, ref.n_clauses)
    assert np.array_equal(cp, ref.clause_ptr) and np.array_equal(lits, ref.lits)
    nv, nc, cp, lits = shard.sub_batch(batch.n_vars, batch.n_clauses, batch.clause_ptr, batch.lits, [])
    assert nv.size == 0 and cp.tolist() == [0] and lits.size == 0


def _inst_case(n_inst, B, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(2, 40, size=(n_inst, B)).astype(np.int32)


def _inst_worker(rank, world, port, n_inst, B, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    shard.init_from_env("gloo")
    nnz = np.arange(1, n_inst + 1) * 1000
    ids = shard.partition_instances(nnz, world)[rank]
    full = _inst_case(n_inst, B, 11)
    unsat = full[ids]
    best = torch.from_numpy(np.argmin(unsat, axis=1).astype(np.int32))
    table = shard.global_best_instances(ids, torch.from_numpy(unsat), best, n_inst)
    torch.save(table, os.path.join(out_dir, "i%d.pt" % rank))
    torch.distributed.destroy_process_group()


def test_global_best_instances_world2(tmp_path):
    n_inst, B = 9, 70
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_inst_worker, args=(r, 2, port, n_inst, B, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    tables = [torch.load(os.path.join(tmp_path, "i%d.pt" % r)) for r in range(2)]
    assert torch.equal(tables[0], tables[1])
    full = _inst_case(n_inst, B, 11)
    owner = {}
    for r, ids in enumerate(shard.partition_instances(np.arange(1, n_inst + 1) * 1000, 2)):
        for i in ids:
            owner[i] = r
    for i in range(n_inst):
        b = int(np.argmin(full[i]))
        assert tables[0][i].tolist() == [int(full[i, b]), b, owner[i]]


def test_global_best_instances_single_process_and_ties():
    unsat = torch.tensor([[4, 2, 2], [7, 7, 1]], dtype=torch.int32)
    best = torch.tensor([1, 2], dtype=torch.int32)
    t = shard.global_best_instances([3, 0], unsat, best, 5, cand_offset=10)
    assert t[3].tolist() == [2, 11, 0] and t[0].tolist() == [1, 12, 0]
    assert t[1].tolist() == [-1, -1, -1]
