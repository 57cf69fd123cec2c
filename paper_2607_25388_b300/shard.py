"""Sharding a batch of independent races across GPUs (one process per GPU).

Races are independent problems (every planning call is its own Alg. 1), so
a batch splits across ranks with no exchange in the data path: each rank
plans its share of the races as one batch on its own GPU, and only timing
(or, for checking, the plans themselves) is gathered afterwards.  A race
keeps its global index as the `race` word of its noise counters, so its plan
does not depend on which rank plans it or on the other races in that
rank's batch: the reassembled plans equal those of the one-GPU batch bit
for bit.

Partition: longest-processing-time first over the races' work,
((L + 1) n_v + 1) best responses of T steps each at the batch's K (the same
for every race), each race to the rank with the least work so far, ties to
the lower rank; every race is assigned to exactly one rank.
"""
from __future__ import annotations

import numpy as np


def race_work(n_v: int, T: int, L: int) -> int:
    """Rollout steps per sample of one race's planning call."""
    return ((L + 1) * n_v + 1) * T


def partition(shapes, world: int, L: int):
    """Assign races with shapes [(n_v, T), ...] to `world` ranks; returns one
    ascending list of race indices per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    work = [race_work(n_v, T, L) for n_v, T in shapes]
    order = sorted(range(len(shapes)), key=lambda r: (-work[r], r))
    load = [0] * world
    out = [[] for _ in range(world)]
    for r in order:
        k = min(range(world), key=lambda q: (load[q], q))
        out[k].append(r)
        load[k] += work[r]
    return [sorted(x) for x in out]


def race_slices(shapes, L: int):
    """Per race, the element ranges of its outputs in a batch of these races
    in this order: xi (n_v (T+1) 4), k_star ((L+1) n_v + 1), U (n_v T 2)."""
    xo = ko = uo = 0
    out = []
    for n_v, T in shapes:
        nx, nk, nu = n_v * (T + 1) * 4, (L + 1) * n_v + 1, n_v * T * 2
        out.append(((xo, xo + nx), (ko, ko + nk), (uo, uo + nu)))
        xo += nx; ko += nk; uo += nu
    return out


def plan_share(races, ids, K: int, L: int, params, seed: int, device="cuda"):
    """Plan races[ids] as one batch on this process's GPU, each race tagged
    with its global index.  Returns {race index: (xi, k_star, U)} as numpy
    arrays and the launch's time in ms (CUDA events)."""
    import torch

    from .planner import Batch, Track
    if not ids:
        return {}, 0.0
    sub = [races[r] for r in ids]
    trk = Track.from_many([sc.track for sc in sub])
    b = Batch(trk, [dict(track_id=q, n_v=sc.X0.shape[0], T=sc.T, ego=sc.ego, race_tag=r)
                    for q, (r, sc) in enumerate(zip(ids, sub))], K=K, L=L)
    X0 = torch.as_tensor(np.concatenate([sc.X0 for sc in sub])).to(device)
    U = torch.as_tensor(np.concatenate([sc.U0.reshape(-1) for sc in sub])).to(device)
    vs = torch.as_tensor(np.concatenate([sc.vref_scale for sc in sub])).to(device)
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    out = b.plan(params, X0, U, vs, seed=seed)
    e.record()
    torch.cuda.synchronize()
    if out["status"].item() != 0:
        raise RuntimeError(f"batch plan status {out['status'].item()}")
    xi, ks, Uo = out["xi"].cpu().numpy(), out["k_star"].cpu().numpy(), U.cpu().numpy()
    res = {}
    for r, ((x0, x1), (k0, k1), (u0, u1)) in zip(ids, race_slices([(sc.X0.shape[0], sc.T) for sc in sub], L)):
        res[r] = (xi[x0:x1], ks[k0:k1], Uo[u0:u1])
    return res, a.elapsed_time(e)


def reassemble(parts, shapes, L: int):
    """Concatenate per-race results {race: (xi, k_star, U)} (the union of all
    ranks' shares) in global race order, the layout of the one-GPU batch."""
    missing = [r for r in range(len(shapes)) if r not in parts]
    if missing:
        raise ValueError(f"races without a plan: {missing[:10]}")
    xi = np.concatenate([parts[r][0] for r in range(len(shapes))])
    ks = np.concatenate([parts[r][1] for r in range(len(shapes))])
    U = np.concatenate([parts[r][2] for r in range(len(shapes))])
    return xi, ks, U


def gather_to_rank0(parts: dict, rank: int, world: int):
    """Collect every rank's {race: result} on rank 0 (torch.distributed
    object gather; used to check the sharded plans, not in the timed path).
    Returns the merged dict on rank 0 and None elsewhere."""
    import torch.distributed as dist
    if world == 1:
        return dict(parts)
    got = [None] * world if rank == 0 else None
    dist.gather_object(parts, got, dst=0)
    if rank != 0:
        return None
    merged = {}
    for p in got:
        dup = set(merged) & set(p)
        if dup:
            raise ValueError(f"races planned twice: {sorted(dup)[:10]}")
        merged.update(p)
    return merged
