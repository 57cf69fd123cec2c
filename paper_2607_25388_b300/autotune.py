"""Launch-shape autotuner of the persistent plan kernel.

The search space is the launch shape of ``sgtp_launch_opts``: the build
(128-thread CTAs with one to three samples per thread at once, or the
256-thread builds with one), samples per thread (0 = chosen per round),
resident CTAs per SM and the schedule (lock-step rounds or per-race
progression from the device queue).  Block and samples per thread fix the
tile, block x samples per thread consecutive samples, and with it the
number of CTA work items per best response, ceil(K / tile); the entries
record it.  Every shape computes each sample with the same code and selects
by an exact integer minimum, so the plan must be bit-identical across
shapes; the tuner checks that on every candidate and refuses a shape that
differs.  (There is no 512-thread build: its one CTA per SM would hold the
registers of three 128-thread CTAs with less latency hiding per thread.)

Results are cached in a JSON file keyed by (horizon bucket, opponent bucket,
K, L, SM count, device name) for single races and by (races, vehicles,
longest horizon, largest race, K, L, SM count, device name) for batches;
``lookup`` / ``lookup_batch`` return the cached shape (``ibr_plan`` and
``Batch.plan`` use them with ``opts="auto"``), ``tune`` / ``tune_batch``
measure and store it.  The cache path is ``$SGTP_AUTOTUNE_CACHE`` or
``~/.cache/sgtp/autotune.json``; it is read once per path and process.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np
import torch

from . import scenario as S
from .planner import SCHEDULE_LOCKSTEP, SCHEDULE_QUEUE, Track, ibr_plan, launch_opts

# (block, samples per thread): the 128-thread build with 0 (per round), 1, 2
# or 3 samples per thread, the 256-thread builds with one
SHAPES = ((128, 0), (128, 1), (128, 2), (128, 3), (256, 1))
CTAS = (0, 1, 2, 3)              # 0 = the occupancy limit; larger values are capped by the library
SCHEDULES = (SCHEDULE_LOCKSTEP, SCHEDULE_QUEUE)


def cache_path() -> str:
    return os.environ.get("SGTP_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "sgtp",
                                                                "autotune.json"))


def _t_bucket(T: int) -> int:
    return (T + 15) // 16 * 16


def _o_bucket(n_opp: int) -> int:
    return 1 if n_opp <= 1 else 3 if n_opp <= 3 else 9 if n_opp <= 9 else 15


def device_info(device=None):
    """(SM count, device name) of the current (or given) CUDA device."""
    d = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    props = torch.cuda.get_device_properties(d)
    return props.multi_processor_count, props.name


def key(n_v: int, T: int, K: int, L: int, info=None) -> str:
    sms, name = info if info is not None else device_info()
    return f"T{_t_bucket(T)}-o{_o_bucket(n_v - 1)}-K{K}-L{L}-sm{sms}-{name}"


_CACHE = {}


def _load(path, fresh=False):
    if not fresh and path in _CACHE:
        return _CACHE[path]
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        d = {}
    _CACHE[path] = d
    return d


def lookup(n_v: int, T: int, K: int, L: int, path: str | None = None, info=None):
    """Cached launch options for this problem shape, or None."""
    return _opts(_load(path or cache_path()).get(key(n_v, T, K, L, info)))


def _opts(ent):
    if not ent:
        return None
    return launch_opts(block=ent["block"], samples_per_thread=ent.get("samples_per_thread", 0),
                       ctas_per_sm=ent["ctas_per_sm"], schedule=ent.get("schedule", 0))


def _tiles(K: int, block: int, spt: int):
    """Work items (tiles) per best response of a fixed shape (None when the
    library chooses samples per thread, and with it the tile, per round)."""
    if block == 0 or (block == 128 and spt == 0):
        return None
    return -(-K // (block * max(spt, 1)))


def _candidates():
    for block, spt in SHAPES:
        for ctas in CTAS:
            for sched in SCHEDULES:
                yield block, spt, ctas, sched


def key_batch(batch, info=None) -> str:
    """Cache key of a batch of races: its size and shape extremes."""
    sms, name = info if info is not None else device_info()
    T_max = max(int(r["T"]) for r in batch.races)
    nv_max = max(int(r["n_v"]) for r in batch.races)
    return (f"batch{len(batch.races)}-a{batch.agents}-T{_t_bucket(T_max)}-o{_o_bucket(nv_max - 1)}-K{batch.K}"
            f"-L{batch.L}-sm{sms}-{name}")


def lookup_batch(batch, path: str | None = None, info=None):
    """Cached launch options for this batch's shape, or None."""
    return _opts(_load(path or cache_path()).get(key_batch(batch, info)))


def _time_plan(trk, params, sc, K, L, opts, reps, warmup):
    X0, vs = torch.as_tensor(sc.X0).cuda(), torch.as_tensor(sc.vref_scale).cuda()
    U0 = torch.as_tensor(sc.U0).cuda()
    U = U0.clone()
    out = None
    for w in range(warmup):
        U.copy_(U0)
        out = ibr_plan(trk, params, X0, U, vs, sc.T, K, L, ego=sc.ego, seed=w, opts=opts, out=out)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    ts = []
    for r in range(reps):
        U.copy_(U0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        ibr_plan(trk, params, X0, U, vs, sc.T, K, L, ego=sc.ego, seed=r, opts=opts, out=out)
        b.record(s)
        ts.append((a, b))
    torch.cuda.synchronize()
    # result of a fixed seed, for the invariance check
    U.copy_(U0)
    res = ibr_plan(trk, params, X0, U, vs, sc.T, K, L, ego=sc.ego, seed=12345, opts=opts, want_hist=True)
    torch.cuda.synchronize()
    digest = tuple(v.cpu().numpy().tobytes() for k, v in sorted(res.items()) if k != "status") + (
        U.cpu().numpy().tobytes(),)
    return float(np.median([a.elapsed_time(b) for a, b in ts])), digest


def store(n_v: int, T: int, K: int, L: int, entry: dict, path: str | None = None, info=None):
    """Write one cache entry (atomic replace of the JSON file)."""
    _store(key(n_v, T, K, L, info), entry, path)


def _store(k: str, entry: dict, path: str | None = None):
    p = path or cache_path()
    os.makedirs(os.path.dirname(p) or ".", exist_ok=True)
    cache = dict(_load(p, fresh=True))
    cache[k] = entry
    tmp = p + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, p)
    _CACHE[p] = cache


def tune(n_v: int, T: int, K: int, L: int, params=None, reps=10, warmup=3, track_seed=777, path: str | None = None,
         log=None):
    """Time every candidate shape on a synthetic race of this shape (seeded
    Fourier track, two-wide grid), check bit-identical plans, store and
    return the fastest as a dict {block, samples_per_thread, ctas_per_sm,
    schedule, tiles_per_response, ms, default_ms}."""
    params = params or S.params_fullscale()
    sc = S.grid_race(S.fourier_track(track_seed), n_v, T, K, L, track_seed + 1)
    trk = Track.from_data(sc.track)
    base_ms, base_digest = _time_plan(trk, params, sc, K, L, launch_opts(), reps, warmup)
    best = dict(block=0, samples_per_thread=0, ctas_per_sm=0, schedule=0, ms=base_ms)
    for block, spt, ctas, sched in _candidates():
        opts = launch_opts(block=block, samples_per_thread=spt, ctas_per_sm=ctas, schedule=sched)
        ms, digest = _time_plan(trk, params, sc, K, L, opts, reps, warmup)
        if digest != base_digest:
            raise RuntimeError(f"launch shape block={block} samples/thread={spt} ctas_per_sm={ctas} "
                               f"schedule={sched} changed the plan")
        if log:
            log(f"block {block:3d} samples/thread {spt} ctas/SM {ctas} schedule {sched}: {ms:.4f} ms")
        if ms < best["ms"]:
            best = dict(block=block, samples_per_thread=spt, ctas_per_sm=ctas, schedule=sched, ms=ms)
    best["tiles_per_response"] = _tiles(K, best["block"], best["samples_per_thread"])
    best["default_ms"] = base_ms
    best["tuned_at"] = time.strftime("%Y-%m-%dT%H:%M:%S")
    store(n_v, T, K, L, best, path)
    return best


def _time_batch(batch, params, X0, U0, vs, opts, reps, warmup):
    U = U0.clone()
    out = None
    for w in range(warmup):
        U.copy_(U0)
        out = batch.plan(params, X0, U, vs, seed=w, opts=opts, out=out)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    ts = []
    for r in range(reps):
        U.copy_(U0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        batch.plan(params, X0, U, vs, seed=r, opts=opts, out=out)
        b.record(s)
        ts.append((a, b))
    torch.cuda.synchronize()
    U.copy_(U0)
    res = batch.plan(params, X0, U, vs, seed=12345, opts=opts, want_hist=True)
    torch.cuda.synchronize()
    digest = tuple(v.cpu().numpy().tobytes() for k, v in sorted(res.items()) if k != "status") + (
        U.cpu().numpy().tobytes(),)
    return float(np.median([a.elapsed_time(b) for a, b in ts])), digest


def tune_batch(batch, params, X0, U0, vs, reps=5, warmup=2, path: str | None = None, log=None):
    """Time every candidate shape on this batch's own inputs (device tensors;
    U0 is not modified), check bit-identical plans, store and return the
    fastest as a dict {block, samples_per_thread, ctas_per_sm, schedule,
    tiles_per_response, ms, default_ms}."""
    base_ms, base_digest = _time_batch(batch, params, X0, U0, vs, launch_opts(), reps, warmup)
    best = dict(block=0, samples_per_thread=0, ctas_per_sm=0, schedule=0, ms=base_ms)
    for block, spt, ctas, sched in _candidates():
        opts = launch_opts(block=block, samples_per_thread=spt, ctas_per_sm=ctas, schedule=sched)
        ms, digest = _time_batch(batch, params, X0, U0, vs, opts, reps, warmup)
        if digest != base_digest:
            raise RuntimeError(f"launch shape block={block} samples/thread={spt} ctas_per_sm={ctas} "
                               f"schedule={sched} changed the batch's plans")
        if log:
            log(f"batch block {block:3d} samples/thread {spt} ctas/SM {ctas} schedule {sched}: {ms:.4f} ms")
        if ms < best["ms"]:
            best = dict(block=block, samples_per_thread=spt, ctas_per_sm=ctas, schedule=sched, ms=ms)
    best["tiles_per_response"] = _tiles(batch.K, best["block"], best["samples_per_thread"])
    best["default_ms"] = base_ms
    best["tuned_at"] = time.strftime("%Y-%m-%dT%H:%M:%S")
    _store(key_batch(batch), best, path)
    return best
