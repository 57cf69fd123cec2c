"""Sharding a batch of independent races across ranks, on CPU: the
partition assigns every race to exactly one rank and balances the work, and
two gloo ranks that plan their shares (with a deterministic CPU stand-in for
the planner: a function of the race alone) and gather them reassemble
exactly the one-process batch."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2607_25388_b300 import shard as SH

L = 3


def shapes(n=37, seed=5):
    rng = np.random.default_rng(seed)
    return [(int(rng.integers(2, 11)), int(rng.integers(30, 81))) for _ in range(n)]


def stand_in_plan(r, n_v, T):
    """Plan of race r as a deterministic function of the race alone."""
    rng = np.random.default_rng(1000 + r)
    return (rng.standard_normal(n_v * (T + 1) * 4).astype(np.float32),
            rng.integers(0, 4096, (L + 1) * n_v + 1).astype(np.int32),
            rng.standard_normal(n_v * T * 2).astype(np.float32))


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_partition_assigns_every_race_once_and_balances_work(world):
    sh = shapes()
    parts = SH.partition(sh, world, L)
    flat = sorted(r for p in parts for r in p)
    assert flat == list(range(len(sh)))
    work = [sum(SH.race_work(*sh[r], L) for r in p) for p in parts]
    biggest = max(SH.race_work(n, T, L) for n, T in sh)
    assert max(work) - min(work) <= biggest               # LPT: within one race's work
    assert SH.partition(sh, world, L) == parts             # deterministic


def test_more_ranks_than_races_leaves_ranks_idle():
    parts = SH.partition([(2, 30), (3, 40)], 4, L)
    assert sorted(r for p in parts for r in p) == [0, 1] and sum(1 for p in parts if not p) == 2


def test_race_slices_follow_the_batch_layout():
    sl = SH.race_slices([(2, 30), (10, 80)], L)
    assert sl[0] == ((0, 2 * 31 * 4), (0, 4 * 2 + 1), (0, 2 * 30 * 2))
    assert sl[1][0] == (248, 248 + 10 * 81 * 4) and sl[1][1] == (9, 9 + 41) and sl[1][2] == (120, 120 + 1600)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sh = shapes()
    mine = SH.partition(sh, world, L)[rank]
    parts = {r: stand_in_plan(r, *sh[r]) for r in mine}
    merged = SH.gather_to_rank0(parts, rank, world)
    if rank == 0:
        xi, ks, U = SH.reassemble(merged, sh, L)
        q.put((xi.tobytes(), ks.tobytes(), U.tobytes(), sorted(merged)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reassemble_the_one_process_batch():
    sh = shapes()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    xi, ks, U, races = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = SH.reassemble({r: stand_in_plan(r, *sh[r]) for r in range(len(sh))}, sh, L)
    assert races == list(range(len(sh)))
    assert xi == ref[0].tobytes() and ks == ref[1].tobytes() and U == ref[2].tobytes()


def test_reassemble_rejects_missing_races():
    sh = [(2, 30), (3, 30)]
    with pytest.raises(ValueError, match="without a plan"):
        SH.reassemble({0: stand_in_plan(0, 2, 30)}, sh, L)
