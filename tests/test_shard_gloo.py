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
